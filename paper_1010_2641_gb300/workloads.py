"""Seeded synthetic inputs shaped like the paper's workloads.

This module only builds INPUTS: atom positions (lattice units), species
indices, occupancies, scattering-factor coefficient sets and reciprocal-space
sampling (grids, lists).  It evaluates nothing of the scattering method
itself, so the FP64 oracle and the GPU library can both consume it without
sharing any arithmetic.  numpy only; every generator takes an explicit seed
(PCG64 via ``numpy.random.default_rng``).

Workloads (sizes and shapes of the paper's examples, Sections 2.2-4.3):
  simple_cubic        perfect parallelepiped at integer coordinates (Sec. 4.1)
  linear_chain        periodic chain 0..N-1 for the accuracy test (Sec. 2.3)
  fcc_sphere          strained spherical nanocrystal, core/shell species
  strained_cube       fcc block with a sinusoidal strain (differentiation)
  truncated_pyramid   epitaxial island for grazing incidence (Sec. 4.3)
  ewald_batch         many small crystals, each with its own curved
                      Ewald-sphere slice of S points (non-grid lists)
  random_sweep        random atoms and random S, the speed test of Sec. 2.2
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

#: Cubic reference lattice parameter (Angstrom) used by every workload (Si).
LATTICE_A = 5.43
#: 10 keV X-ray wavelength (Angstrom), the energy of the paper's example.
WAVELENGTH_10KEV = 1.2398

# Basis of the face-centred cubic lattice (lattice units).
_FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])


# --------------------------------------------------------------------------
# Scattering-factor coefficient sets
# --------------------------------------------------------------------------

def species_coefficients(Z: float, fp: float = 0.0, fpp: float = 0.0, b_dw: float = 0.0) -> np.ndarray:
    """Synthetic 4-Gaussian + constant coefficients with f0(0) = Z.

    The tabulated analytic coefficients the paper takes from cctbx are not
    available, so a fixed, smooth stand-in of the same form is used:
    a_i = Z * (0.42, 0.30, 0.18, 0.07), c = 0.03 Z,
    b_i = (0.6, 3.5, 14, 45) Angstrom^2.
    Returns the 12-vector (a0..a3, b0..b3, c, f', f'', B_dw).
    """
    a = Z * np.array([0.42, 0.30, 0.18, 0.07])
    b = np.array([0.6, 3.5, 14.0, 45.0])
    return np.concatenate([a, b, [0.03 * Z, fp, fpp, b_dw]]).astype(np.float64)


def unit_species() -> np.ndarray:
    """f == 1 (the paper's speed test evaluates no scattering factor)."""
    return np.array([0, 0, 0, 0, 0, 0, 0, 0, 1.0, 0, 0, 0], dtype=np.float64)


def si_ge_species() -> np.ndarray:
    """Two species: Si-like core (Z=14) and Ge-like shell (Z=32, with f', f'')."""
    return np.stack([species_coefficients(14.0, 0.1, 0.2, 0.5),
                     species_coefficients(32.0, -1.6, 0.9, 0.6)])


# --------------------------------------------------------------------------
# Reciprocal-space sampling
# --------------------------------------------------------------------------

def linspace_axis(center: float, n: int, step: float | None = None, half_width: float | None = None) -> np.ndarray:
    """n points centred on `center`, either with a step or spanning +-half_width inclusive."""
    if step is not None:
        return center + (np.arange(n) - 0.5 * (n - 1)) * step
    if n == 1:
        return np.array([float(center)])
    return np.linspace(center - half_width, center + half_width, n)


def grid_points(axes) -> np.ndarray:
    """Flatten a grid (three 1-D axes) to [M,3], first axis slowest."""
    a0, a1, a2 = (np.asarray(a, dtype=np.float64) for a in axes)
    g = np.stack(np.meshgrid(a0, a1, a2, indexing="ij"), axis=-1)
    return g.reshape(-1, 3)


# --------------------------------------------------------------------------
# Crystals
# --------------------------------------------------------------------------

def simple_cubic(n=(10, 10, 10), origin=(0, 0, 0)) -> np.ndarray:
    """One atom per cell at integer coordinates origin + (0..n-1), x fastest."""
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xyz = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float64)
    return xyz + np.asarray(origin, dtype=np.float64)


def example_cube_100(strained: bool = False) -> np.ndarray:
    """The first worked example of Section 4: a simple cubic crystal of
    100 x 100 x 100 cells, one atom per cell at x, y in [-50, 50), z in
    [0, 100) (lattice units, f = 1).  strained=True adds the displacement
    field of the same example along z, u_z = 1e-6 z (x^2 + y^2) (at most
    ~0.5 cells at the corners).  1,000,000 atoms."""
    xyz = simple_cubic((100, 100, 100), origin=(-50, -50, 0))
    if strained:
        xyz[:, 2] += 1e-6 * xyz[:, 2] * (xyz[:, 0] ** 2 + xyz[:, 1] ** 2)
    return xyz


def example_cube_axes():
    """Its map around (004): h = -0.1 ... 0.099 and l = 3.9 ... 4.099 in steps
    of 0.001 (200 values each), k = 0: a 200 x 1 x 200 grid (40,000 points)."""
    i = np.arange(200, dtype=np.float64)
    return [-0.1 + 0.001 * i, np.zeros(1), 3.9 + 0.001 * i]


def linear_chain(n: int, sigma: float = 0.0, seed: int = 0) -> np.ndarray:
    """Atoms at x = 0..n-1 (Section 2.3), optionally with Gaussian noise of std sigma."""
    xyz = np.zeros((n, 3))
    xyz[:, 0] = np.arange(n)
    if sigma:
        xyz[:, 0] += np.random.default_rng(seed).normal(0.0, sigma, n)
    return xyz


def _fcc_sites(lo, hi) -> np.ndarray:
    r = [np.arange(lo[i], hi[i]) for i in range(3)]
    cells = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 1, 3)
    return (cells + _FCC_BASIS[None]).reshape(-1, 3).astype(np.float64)


@dataclasses.dataclass
class Crystal:
    xyz: np.ndarray            # [N,3] float64 lattice units
    species: np.ndarray        # [N] int32
    coef: np.ndarray           # [n_species, 12]
    occ: np.ndarray | None = None


def fcc_sphere(radius_cells: float = 20.0, shell_cells: float = 3.0, strain: float = 0.02,
               strain_length_cells: float = 15.0, sigma_angstrom: float = 0.05,
               seed: int = 2000, lattice_a: float = LATTICE_A) -> Crystal:
    """Strained spherical fcc nanocrystal (core Z=14, shell Z=32).

    Sites of an fcc lattice within |r| <= radius (cells).  Radial displacement
    u = strain * r * exp(-|r|^2 / L^2) with L = strain_length_cells (i.e.
    15 a), plus independent Gaussian displacements of sigma_angstrom per
    component.  Atoms with |r| > radius - shell_cells are species 1.
    """
    R = float(radius_cells)
    k = int(math.ceil(R)) + 1
    sites = _fcc_sites((-k, -k, -k), (k + 1, k + 1, k + 1))
    r2 = np.einsum("ij,ij->i", sites, sites)
    sites = sites[r2 <= R * R + 1e-9]
    r2 = np.einsum("ij,ij->i", sites, sites)
    species = (np.sqrt(r2) > R - shell_cells).astype(np.int32)
    rng = np.random.default_rng(seed)
    u = strain * sites * np.exp(-r2 / strain_length_cells ** 2)[:, None]
    u += rng.normal(0.0, sigma_angstrom / lattice_a, sites.shape)
    return Crystal(sites + u, species, si_ge_species())


def strained_cube(n=(40, 40, 16), amplitude: float = 0.01, sigma_cells: float = 0.01,
                  seed: int = 4000) -> Crystal:
    """fcc block of n cells with u_z = (amplitude*nx/2pi) sin(2 pi x/nx) + noise.

    The sinusoid's largest strain du_z/dx is `amplitude`.
    """
    nx, ny, nz = n
    sites = _fcc_sites((0, 0, 0), (nx, ny, nz))
    sites -= np.array([nx / 2, ny / 2, nz / 2])
    rng = np.random.default_rng(seed)
    uz = amplitude * nx / (2 * np.pi) * np.sin(2 * np.pi * sites[:, 0] / nx)
    sites[:, 2] += uz
    sites += rng.normal(0.0, sigma_cells, sites.shape)
    return Crystal(sites, np.zeros(len(sites), np.int32), si_ge_species()[:1])


def perturbed_copy(c: Crystal, sigma_cells: float = 0.02, seed: int = 4001) -> Crystal:
    """The same crystal with extra Gaussian displacements (source of I_obs)."""
    rng = np.random.default_rng(seed)
    return Crystal(c.xyz + rng.normal(0.0, sigma_cells, c.xyz.shape), c.species.copy(), c.coef.copy(), c.occ)


def truncated_pyramid(base_cells: int = 120, height_cells: int = 40, top_cells: int = 30,
                      mismatch: float = 0.04, vertical_spacing: float = 1.04,
                      two_species: bool = True) -> Crystal:
    """Epitaxial fcc island: a truncated square pyramid on a flat substrate.

    Cell layer z (0..height-1) is a centred square of side
    round(base - (base-top) z/(height-1)) cells; its in-plane lattice is
    expanded by mismatch*z/(height-1) (fully strained at the interface,
    relaxed at the top) and cells are stacked with `vertical_spacing`.
    With two_species, the upper half is species 1 (Ge-like).
    """
    parts, spec = [], []
    for z in range(height_cells):
        side = int(round(base_cells - (base_cells - top_cells) * z / (height_cells - 1)))
        scale = 1.0 + mismatch * z / (height_cells - 1)
        s = _fcc_sites((0, 0, z), (side, side, z + 1))
        s[:, 0] = (s[:, 0] - side / 2) * scale
        s[:, 1] = (s[:, 1] - side / 2) * scale
        s[:, 2] = s[:, 2] * vertical_spacing
        parts.append(s)
        spec.append(np.full(len(s), 1 if (two_species and z >= height_cells // 2) else 0, np.int32))
    coef = si_ge_species() if two_species else si_ge_species()[:1]
    return Crystal(np.concatenate(parts), np.concatenate(spec), coef)


def below_surface(c: Crystal, depth_cells: float) -> Crystal:
    """The same crystal moved into the substrate: its top at depth_cells
    below the surface plane z = 0 (every z <= -depth_cells)."""
    xyz = c.xyz.copy()
    xyz[:, 2] -= xyz[:, 2].max() + depth_cells
    return Crystal(xyz, c.species.copy(), c.coef.copy(), c.occ)


def gid_axes(n_h: int = 512, n_k: int = 512, n_af: int = 32):
    """Grazing-incidence map around in-plane (400): h in [3.80, 4.05],
    k in [-0.125, 0.125] (inclusive) and alpha_f = (i+1)/32 degrees."""
    h = np.linspace(3.80, 4.05, n_h)
    k = np.linspace(-0.125, 0.125, n_k)
    af = np.deg2rad((np.arange(n_af) + 1) / 32.0)
    return h, k, af


GID_ALPHA_I = float(np.deg2rad(0.2))
GID_DELTA = 1e-5
GID_BETA = 1e-7


# --------------------------------------------------------------------------
# Batches on curved Ewald-sphere slices
# --------------------------------------------------------------------------

def _rotation(axis, angle):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def ewald_slice(n_points: int, hkl=(1, 1, 1), lattice_a: float = LATTICE_A,
                wavelength: float = WAVELENGTH_10KEV, window_deg: float = 1.0,
                rocking_deg: float = 0.0, seed: int = 0) -> np.ndarray:
    """S points (r.l.u.) seen by a detector window around the Bragg direction.

    The crystal's reflection `hkl` is put in Bragg condition; the exit
    directions k_f are sampled uniformly in a +-window_deg x +-window_deg
    patch around the Bragg exit direction and S = (k_f - k_i) * a, |k| = 1/lambda
    (1/Angstrom).  `rocking_deg` tilts k_i off the Bragg condition.
    """
    rng = np.random.default_rng(seed)
    g = np.asarray(hkl, float) / lattice_a           # 1/Angstrom
    n = g / np.linalg.norm(g)
    sin_t = wavelength * np.linalg.norm(g) / 2.0
    cos_t = math.sqrt(1.0 - sin_t ** 2)
    p = np.cross(n, [1.0, 0.0, 0.0])
    if np.linalg.norm(p) < 1e-6:
        p = np.cross(n, [0.0, 1.0, 0.0])
    p /= np.linalg.norm(p)
    q = np.cross(n, p)
    ki = (-sin_t * n + cos_t * p) / wavelength
    kf0 = (sin_t * n + cos_t * p) / wavelength
    ki = _rotation(q, math.radians(rocking_deg)) @ ki
    e1 = np.cross(kf0, q)
    e1 /= np.linalg.norm(e1)
    a1 = np.deg2rad(rng.uniform(-window_deg, window_deg, n_points))
    a2 = np.deg2rad(rng.uniform(-window_deg, window_deg, n_points))
    # exit directions: kf0 tilted by a1 about q, then by a2 about e1 (Rodrigues)
    kf = _rotate_many(np.broadcast_to(kf0, (n_points, 3)), q, a1)
    kf = _rotate_many(kf, e1, a2)
    return (kf - ki) * lattice_a


def _rotate_many(v, axis, angles):
    k = np.asarray(axis, float) / np.linalg.norm(axis)
    c, s = np.cos(angles)[:, None], np.sin(angles)[:, None]
    kv = np.cross(np.broadcast_to(k, v.shape), v)
    return v * c + kv * s + k[None, :] * (v @ k)[:, None] * (1.0 - c)


def ewald_batch(n_instances: int = 64, n_atoms_range=(1e3, 2e5), n_s_range=(1e4, 1e6),
                seed: int = 3000):
    """Uneven batch: fcc spheres with log-uniform atom counts, each with its
    own log-uniform number of Ewald-slice S points near (1,1,1).

    Returns (xyz [sum N,3], species [sum N], coef, S [sum M,3], atom_off, s_off).
    """
    rng = np.random.default_rng(seed)
    n_atoms = np.exp(rng.uniform(np.log(n_atoms_range[0]), np.log(n_atoms_range[1]), n_instances))
    n_s = np.exp(rng.uniform(np.log(n_s_range[0]), np.log(n_s_range[1]), n_instances)).astype(np.int64)
    xyzs, specs, Ss = [], [], []
    for b in range(n_instances):
        radius = (3.0 * n_atoms[b] / (16.0 * math.pi)) ** (1.0 / 3.0)  # 4 atoms per cell
        c = fcc_sphere(radius_cells=radius, shell_cells=min(3.0, 0.3 * radius), seed=seed + 1 + b)
        xyzs.append(c.xyz)
        specs.append(c.species)
        Ss.append(ewald_slice(int(n_s[b]), rocking_deg=float(rng.uniform(-0.05, 0.05)),
                              seed=seed + 1000 + b))
    atom_off = np.concatenate([[0], np.cumsum([len(x) for x in xyzs])]).astype(np.int64)
    s_off = np.concatenate([[0], np.cumsum([len(s) for s in Ss])]).astype(np.int64)
    return (np.concatenate(xyzs), np.concatenate(specs), si_ge_species(), np.concatenate(Ss),
            atom_off, s_off)


def random_sweep(n_atoms: int, n_s: int, seed: int = 0, box: float = 100.0, center=(0, 0, 4)):
    """Random atoms in a box^3 (lattice units) and random S within +-0.5 of center."""
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(0.0, box, (n_atoms, 3))
    S = np.asarray(center, float) + rng.uniform(-0.5, 0.5, (n_s, 3))
    return xyz, S


@dataclasses.dataclass
class BlockModel:
    """Eq. 4 input: blocks of atoms on a lattice, displaced (r_j^0 + u_j).

    origins : [n_blocks, 3] displaced block origins (lattice units)
    types   : [n_blocks] block type (0 or 1)
    content : [n_types] list of [n_atoms_in_block, 3] atom offsets in a block
    species : [n_types] list of per-atom species indices of each block type
    """
    origins: np.ndarray
    types: np.ndarray
    content: list
    species: list


def fcc_cell_blocks(n=(12, 12, 8), frac_type1: float = 0.3, amplitude: float = 0.05, sigma: float = 0.01,
                    seed: int = 5001) -> BlockModel:
    """A lattice of one-cell fcc blocks (4 atoms each), the block type drawn
    at random (type 0: Si-like atoms, type 1: Ge-like atoms), displaced by a
    smooth field u_z = amplitude sin(2 pi x / n_x) plus seeded noise: the
    continuum-elasticity picture of Section 2.1 at one-cell resolution."""
    rng = np.random.default_rng(seed)
    cells = np.stack(np.meshgrid(*[np.arange(k, dtype=np.float64) for k in n], indexing="ij"), -1).reshape(-1, 3)
    cells -= 0.5 * (np.asarray(n, dtype=np.float64) - 1.0)
    u = np.zeros_like(cells)
    u[:, 2] = amplitude * np.sin(2.0 * np.pi * cells[:, 0] / n[0])
    u += rng.normal(0.0, sigma, cells.shape)
    types = (rng.uniform(size=len(cells)) < frac_type1).astype(np.int32)
    cell = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]], dtype=np.float64)
    return BlockModel(origins=cells + u, types=types, content=[cell, cell],
                      species=[np.zeros(4, np.int32), np.ones(4, np.int32)])


def ge_dot(base_radius_cells: float = 50.0, height_cells: float = 20.0, seed: int = 6001) -> Crystal:
    """The germanium quantum dot of the paper's grazing-incidence example
    (Section 4.3): a spherical cap of base radius 50 cells and height 20
    cells standing on the substrate (z >= 0), diamond lattice (8 atoms per
    cell, Si/Ge), Ge fraction rising linearly from 0.2 at the bottom to 0.8
    at the top (species drawn per atom, seeded), and the in-plane relaxation
    eps_xx = eps_yy = 0.005 + z 0.002 (1 + sqrt(x^2 + y^2) / 50) of the
    substrate lattice, applied as the dilation x -> x (1 + eps), y -> y (1 + eps)
    (x, y, z fractional coordinates of the substrate lattice)."""
    R, h = float(base_radius_cells), float(height_cells)
    Rs = (R * R + h * h) / (2.0 * h)          # radius of the sphere the cap is cut from
    zc = h - Rs                               # its centre (below the base plane)
    n = int(np.ceil(R)) + 1
    cells = np.stack(np.meshgrid(np.arange(-n, n + 1), np.arange(-n, n + 1), np.arange(0, int(np.ceil(h)) + 1),
                                 indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    fcc = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    basis = np.concatenate([fcc, fcc + 0.25])                 # diamond
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    x, y, z = sites[:, 0], sites[:, 1], sites[:, 2]
    keep = (z >= 0) & (z <= h) & (x * x + y * y + (z - zc) ** 2 <= Rs * Rs)
    sites = sites[keep]
    x, y, z = sites[:, 0], sites[:, 1], sites[:, 2]
    eps = 0.005 + z * 0.002 * (1.0 + np.sqrt(x * x + y * y) / 50.0)
    xyz = np.stack([x * (1.0 + eps), y * (1.0 + eps), z], 1)
    rng = np.random.default_rng(seed)
    ge = rng.uniform(size=len(xyz)) < 0.2 + 0.6 * z / h
    return Crystal(xyz=xyz, species=ge.astype(np.int32), coef=si_ge_species())


def ge_dot_axes(n_h: int = 512, n_af: int = 128):
    """(h, k, alpha_f) axes of the dot's map: h across (400), k = 0, alpha_f in (0, 1 deg]."""
    h = np.linspace(3.70, 4.10, n_h)
    k = np.array([0.0])
    af = np.deg2rad((np.arange(n_af) + 1) * (1.0 / n_af))
    return h, k, af
