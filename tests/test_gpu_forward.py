"""GPU parity of the forward paths (generic FP32/MUFU and plain FP64) against
the FP64 oracle and closed forms, through the C ABI.

Tolerance (stated by the method's precision targets): relative L2 over each
map <= 1e-4 for the FP32 paths; the FP64 kernel accumulates in double and
rounds its output to complex64, so <= 1e-6 there.
"""
import ctypes

import numpy as np
import pytest
import torch

import __graft_entry__
import oracle
from closed_forms import parallelepiped_closed_form, rel_l2
from paper_1010_2641_gb300 import api
from paper_1010_2641_gb300 import binding as B
from paper_1010_2641_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4
TOL_FP64 = 1e-6
A_LAT = W.LATTICE_A


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def dev(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda:0")


def run(plan, xyz, occ=None):
    A = plan.amplitude(dev(xyz), None if occ is None else dev(occ, torch.float32))
    plan.check()
    return A.cpu().numpy().astype(np.complex128)


def unit():
    return W.unit_species()[None]


# ---------------------------------------------------------------------------
# tiny configuration: perfect 10^3 cube, 32^3 grid around (004)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("path", ["generic", "fp64"])
def test_tiny_cube_dirichlet(path):
    xyz = W.simple_cubic((10, 10, 10))
    axes = [W.linspace_axis(c, 32, half_width=0.5) for c in (0.0, 0.0, 4.0)]
    S = W.grid_points(axes)
    plan = api.Plan(unit(), A_LAT, len(xyz), axes=axes, path=path)
    A = run(plan, xyz)
    closed = parallelepiped_closed_form((10, 10, 10), S)
    ref = oracle.amplitude(xyz, S, unit(), A_LAT)
    tol = TOL_FP32 if path == "generic" else TOL_FP64
    assert rel_l2(A, ref) < tol
    assert rel_l2(A, closed) < tol
    # the Bragg node (0,0,4) is not on this grid; the largest |A| must still
    # match the closed form's largest |A|
    assert abs(np.abs(A).max() - np.abs(closed).max()) < 10 * tol * np.abs(closed).max()


# ---------------------------------------------------------------------------
# lists with species, occupancies, ragged sizes, several tiles
# ---------------------------------------------------------------------------

def _random_case(seed, n_atoms, n_s, spread=0.3, box=12.0, offset=(0, 0, 0)):
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(-box, box, (n_atoms, 3)) + np.asarray(offset, float)
    sp = rng.integers(0, 2, n_atoms).astype(np.int32)
    occ = rng.uniform(0.3, 1.0, n_atoms)
    S = np.array([0.0, 0.0, 4.0]) + rng.uniform(-spread, spread, (n_s, 3))
    return xyz, sp, occ, W.si_ge_species(), S


@pytest.mark.parametrize("n_atoms,n_s", [(1000, 3001), (77, 513), (2049, 257)])
def test_list_species_occupancy(n_atoms, n_s):
    xyz, sp, occ, coef, S = _random_case(1, n_atoms, n_s)
    plan = api.Plan(coef, A_LAT, n_atoms, s_list=S, atom_species=sp)
    A = run(plan, xyz, occ)
    ref = oracle.amplitude(xyz, S, coef, A_LAT, species=sp, occ=occ.astype(np.float32))
    assert rel_l2(A, ref) < TOL_FP32
    I = plan.intensity(dev(xyz), dev(occ, torch.float32)).cpu().numpy()
    assert np.allclose(I, np.abs(A) ** 2, rtol=1e-5, atol=1e-6 * np.abs(A).max() ** 2)


@pytest.mark.parametrize("threads,R,split", [(128, 4, 1), (256, 8, 3), (256, 16, 2), (128, 16, 7), (256, 4, 64)])
def test_tilings_agree(threads, R, split):
    xyz, sp, occ, coef, S = _random_case(2, 3000, 2000)
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, threads=threads,
                    points_per_thread=R, split_k=split)
    info = plan.info()
    assert (info["threads"], info["points_per_thread"], info["split_k"]) == (threads, R, split)
    A = run(plan, xyz, occ)
    ref = oracle.amplitude(xyz, S, coef, A_LAT, species=sp, occ=occ.astype(np.float32))
    assert rel_l2(A, ref) < TOL_FP32


@pytest.mark.parametrize("kind", ["list", "grid"])
def test_off_centre_crystal_translation(kind):
    """A crystal far from the origin: the per-call integer centring t must be
    undone exactly by the translation phase e^{2 pi i s.t}."""
    xyz, sp, occ, coef, S = _random_case(3, 1500, 1000, box=6.0, offset=(137.3, -212.8, 55.1))
    if kind == "list":
        plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp)
    else:
        axes = [W.linspace_axis(0.02, 5, step=0.013), W.linspace_axis(-0.01, 7, step=0.011),
                W.linspace_axis(3.97, 13, step=0.009)]
        S = W.grid_points(axes)
        plan = api.Plan(coef, A_LAT, len(xyz), axes=axes, atom_species=sp, path="generic")
    A = run(plan, xyz, occ)
    assert plan.info()["shift"] == [137.0, -213.0, 55.0]
    ref = oracle.amplitude(xyz, S, coef, A_LAT, species=sp, occ=occ.astype(np.float32))
    assert rel_l2(A, ref) < TOL_FP32


@pytest.mark.parametrize("shape", [(5, 7, 13), (1, 1, 1), (3, 2, 9), (16, 16, 64)])
def test_grid_ragged(shape):
    c = W.fcc_sphere(radius_cells=4.3, seed=9)
    axes = [W.linspace_axis(0.0, shape[0], step=0.004), W.linspace_axis(0.0, shape[1], step=0.004),
            W.linspace_axis(4.0, shape[2], step=0.004)]
    S = W.grid_points(axes)
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, path="generic")
    A = run(plan, c.xyz)
    ref = oracle.amplitude(c.xyz, S, c.coef, A_LAT, species=c.species)
    assert A.shape == (np.prod(shape),)
    assert rel_l2(A, ref) < TOL_FP32


def test_fp64_path_list():
    xyz, sp, occ, coef, S = _random_case(4, 700, 900)
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, path="fp64")
    A = run(plan, xyz, occ)
    ref = oracle.amplitude(xyz, S, coef, A_LAT, species=sp, occ=occ.astype(np.float32))
    assert rel_l2(A, ref) < TOL_FP64


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_single_atom_single_point():
    xyz = np.array([[0.25, -1.5, 3.125]])
    S = np.array([[0.1, 0.2, 4.3]])
    coef = W.si_ge_species()[1:]
    plan = api.Plan(coef, A_LAT, 1, s_list=S)
    A = run(plan, xyz)
    ref = oracle.amplitude(xyz, S, coef, A_LAT)
    assert abs(A[0] - ref[0]) < 1e-5 * abs(ref[0])


def test_no_atoms_gives_zeros():
    S = np.array([[0.0, 0.0, 4.0], [0.1, 0.0, 4.0]])
    plan = api.Plan(unit(), A_LAT, 0, s_list=S)
    A = plan.amplitude(torch.empty(0, 3, dtype=torch.float64, device="cuda:0"))
    assert torch.all(A == 0)


def test_no_points():
    plan = api.Plan(unit(), A_LAT, 3, s_list=np.zeros((0, 3)))
    A = plan.amplitude(dev(np.zeros((3, 3))))
    assert A.numel() == 0


def test_zero_occupancy_removes_atoms():
    xyz, sp, occ, coef, S = _random_case(5, 300, 200)
    occ[::2] = 0.0
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp)
    A = run(plan, xyz, occ)
    keep = occ != 0
    ref = oracle.amplitude(xyz[keep], S, coef, A_LAT, species=sp[keep], occ=occ[keep].astype(np.float32))
    assert rel_l2(A, ref) < TOL_FP32


def test_nonfinite_position_reported():
    xyz, sp, occ, coef, S = _random_case(6, 100, 64)
    xyz[17, 1] = np.nan
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp)
    plan.amplitude(dev(xyz))
    with pytest.raises(B.ScatterError) as e:
        plan.check()
    assert e.value.status == B.SCATTER_ERR_NUMERIC
    xyz[17, 1] = 0.0
    plan.amplitude(dev(xyz))
    plan.check()  # cleared


def test_host_pointer_rejected():
    xyz, sp, occ, coef, S = _random_case(7, 10, 10)
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp)
    host = np.ascontiguousarray(xyz)
    out = torch.empty(10, dtype=torch.complex64, device="cuda:0")
    st = B.lib().scatter_amplitude(plan.handle, host.ctypes.data, None, out.data_ptr(), None)
    assert st == B.SCATTER_ERR_INVALID_ARG


def test_plan_reuse_and_destroy_twice():
    xyz, sp, occ, coef, S = _random_case(8, 200, 100)
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp)
    A1 = run(plan, xyz, occ)
    A2 = run(plan, xyz + 0.1, occ)
    A3 = run(plan, xyz, occ)
    assert np.array_equal(A1, A3) and not np.array_equal(A1, A2)
    plan.close()
    plan.close()


def test_autotune_cache(tmp_path):
    c = W.fcc_sphere(radius_cells=5.0, seed=3)
    axes = [W.linspace_axis(0.0, 24, step=0.01), W.linspace_axis(0.0, 24, step=0.01), W.linspace_axis(4.0, 32, step=0.01)]
    cache = tmp_path / "tune.jsonl"
    p1 = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, autotune=True, tune_cache=str(cache),
                  path="generic")
    assert cache.exists() and cache.read_text().count("\n") == 1
    p2 = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, autotune=True, tune_cache=str(cache),
                  path="generic")
    assert cache.read_text().count("\n") == 1
    i1, i2 = p1.info(), p2.info()
    assert (i1["threads"], i1["points_per_thread"], i1["split_k"]) == (i2["threads"], i2["points_per_thread"], i2["split_k"])
    A = run(p2, c.xyz)
    ref = oracle.amplitude(c.xyz, W.grid_points(axes), c.coef, A_LAT, species=c.species)
    assert rel_l2(A, ref) < TOL_FP32


def test_error_bound_covers_diffuse_map():
    """A disordered crystal gives a diffuse map whose per-pair errors are
    uncorrelated: the measured error must sit below the stated model."""
    rng = np.random.default_rng(12)
    xyz = rng.uniform(-20, 20, (4000, 3))
    S = np.array([0.0, 0.0, 4.0]) + rng.uniform(-0.25, 0.25, (2000, 3))
    plan = api.Plan(unit(), A_LAT, len(xyz), s_list=S)
    A = run(plan, xyz)
    ref = oracle.amplitude(xyz, S, unit(), A_LAT)
    per_pair, rel = plan.error_bound(radius=20.0 * np.sqrt(3))
    assert rel_l2(A, ref) < rel
    assert rel < TOL_FP32


# ---------------------------------------------------------------------------
# full-size strained sphere (134,009 atoms x 256x256x64 grid) on samples
# ---------------------------------------------------------------------------

def test_strained_sphere_full_size_sampled():
    c = W.fcc_sphere()
    axes = [W.linspace_axis(0.0, 256, step=0.002), W.linspace_axis(0.0, 256, step=0.002),
            W.linspace_axis(4.0, 64, step=0.002)]
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, path="generic")
    A = run(plan, c.xyz)
    assert A.shape == (256 * 256 * 64,)
    rng = np.random.default_rng(0)
    idx = rng.choice(A.shape[0], 768, replace=False)
    idx[:8] = np.argsort(np.abs(A))[-8:]  # include the brightest points
    S = W.grid_points(axes)[idx]
    ref = oracle.amplitude(c.xyz, S, c.coef, A_LAT, species=c.species)
    assert rel_l2(A[idx], ref) < TOL_FP32
    assert np.all(np.isfinite(A))
