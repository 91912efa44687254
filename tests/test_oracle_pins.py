"""Pins of the FP64 oracle to results fixed by the paper and by mathematics.

None of these tests re-evaluates the oracle's own code path: each compares
it with a closed form (geometric series of a parallelepiped, Section 2.3),
an invariant of Eq. 2 (Friedel, translation, species factoring, occupancy,
permutation), a high-precision brute force on tiny inputs, textbook Fresnel
coefficients or wave-vector kinematics (Section 4.3), or an independent
route to the gradient.  CPU only.
"""
import math

import numpy as np
import pytest

import oracle
from closed_forms import dirichlet, parallelepiped_closed_form
from paper_1010_2641_gb300 import workloads as W

A_LAT = W.LATTICE_A


def unit_coef():
    return W.unit_species()[None, :]


# ----------------------------------------------------------------------------
# Eq. 2 against closed forms
# ----------------------------------------------------------------------------

def test_dirichlet_cube_tiny_config():
    """10x10x10 simple cubic, f=1, 32^3 grid spanning +-0.5 around (0,0,4)."""
    xyz = W.simple_cubic((10, 10, 10))
    ax = [W.linspace_axis(c, 32, half_width=0.5) for c in (0.0, 0.0, 4.0)]
    S = W.grid_points(ax)
    A = oracle.amplitude(xyz, S, unit_coef(), A_LAT)
    ref = parallelepiped_closed_form((10, 10, 10), S)
    assert np.max(np.abs(A - ref)) < 1e-9 * 1000
    assert np.linalg.norm(A - ref) / np.linalg.norm(ref) < 1e-12


@pytest.mark.parametrize("n", [(3, 5, 7), (1, 4, 9)])
def test_dirichlet_box_random_S(n):
    rng = np.random.default_rng(7)
    xyz = W.simple_cubic(n)
    S = rng.uniform(-3.0, 3.0, (500, 3))
    S[:20] = np.rint(S[:20])  # exact reciprocal-lattice nodes: |A| = N
    A = oracle.amplitude(xyz, S, unit_coef(), A_LAT)
    ref = parallelepiped_closed_form(n, S)
    assert np.max(np.abs(A - ref)) < 1e-11 * np.prod(n)
    assert np.allclose(np.abs(A[:20]), np.prod(n), rtol=1e-13)


@pytest.mark.parametrize("N", [1000, 10000, 100000])
@pytest.mark.parametrize("offset", [0.0, 0.00037])
def test_linear_chain_accuracy_test(N, offset):
    """Section 2.3: chain at 0..N-1, H every 0.001 r.l.u. around H=1, versus
    sin(pi N H)/sin(pi H) in full complex form (the paper's grid puts every
    point but the peak on a zero of the kernel; the offset grid does not)."""
    xyz = W.linear_chain(N)
    H = 0.95 + offset + 0.001 * np.arange(100)
    S = np.stack([H, np.zeros_like(H), np.zeros_like(H)], 1)
    A = oracle.amplitude(xyz, S, unit_coef(), A_LAT)
    ref = dirichlet(N, H)
    # phases reach 1e5 cycles: FP64 keeps ~1e-11 rad per term
    assert np.max(np.abs(A - ref)) < 1e-9 * N
    peak = np.argmin(np.abs(H - 1.0))
    if offset == 0.0:
        assert abs(abs(A[peak]) - N) < 1e-9 * N


# ----------------------------------------------------------------------------
# High-precision brute force on tiny inputs
# ----------------------------------------------------------------------------

def test_brute_force_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(11)
    n_atoms, n_s = 9, 15
    xyz = rng.uniform(-6, 6, (n_atoms, 3))
    species = rng.integers(0, 2, n_atoms).astype(np.int32)
    occ = rng.uniform(0.2, 1.5, n_atoms)
    coef = np.stack([W.species_coefficients(14, 0.3, 0.7, 0.4), W.species_coefficients(32, -1.2, 2.5, 0.9)])
    coef[1, 4:8] = [0.2, 1.7, 9.0, 30.0]
    S = rng.uniform(-5, 5, (n_s, 3))
    A = oracle.amplitude(xyz, S, coef, A_LAT, species=species, occ=occ)
    for m in range(n_s):
        Sm = [mp.mpf(float(v)) for v in S[m]]
        # Bragg's law: d = a / |hkl|, sin(theta)/lambda = 1 / (2 d)
        d = mp.mpf(A_LAT) / mp.sqrt(sum(v * v for v in Sm))
        s2 = (1 / (2 * d)) ** 2
        tot = mp.mpc(0)
        for j in range(n_atoms):
            c = coef[species[j]]
            f0 = sum(mp.mpf(float(c[i])) * mp.e ** (-mp.mpf(float(c[4 + i])) * s2) for i in range(4)) + mp.mpf(float(c[8]))
            f = (f0 + mp.mpf(float(c[9])) + 1j * mp.mpf(float(c[10]))) * mp.e ** (-mp.mpf(float(c[11])) * s2)
            x = sum(Sm[i] * mp.mpf(float(xyz[j, i])) for i in range(3))
            tot += mp.mpf(float(occ[j])) * f * mp.expjpi(2 * x)
        ref = complex(tot)
        assert abs(A[m] - ref) < 1e-12 * max(1.0, abs(ref))


# ----------------------------------------------------------------------------
# Invariants of Eq. 2
# ----------------------------------------------------------------------------

def _random_problem(seed, n_atoms=200, n_s=300, real_f=False):
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(-8, 8, (n_atoms, 3))
    species = rng.integers(0, 2, n_atoms).astype(np.int32)
    occ = rng.uniform(0.5, 1.0, n_atoms)
    coef = W.si_ge_species()
    if real_f:
        coef[:, 10] = 0.0
    S = rng.uniform(-4, 4, (n_s, 3))
    return xyz, species, occ, coef, S


def test_friedel_symmetry():
    xyz, sp, occ, coef, S = _random_problem(1, real_f=True)
    A = oracle.amplitude(xyz, S, coef, A_LAT, sp, occ)
    Am = oracle.amplitude(xyz, -S, coef, A_LAT, sp, occ)
    assert np.max(np.abs(Am - np.conj(A))) < 1e-11 * np.max(np.abs(A))


def test_friedel_broken_by_anomalous_term():
    """With f'' != 0 Friedel's law must fail: a check that the imaginary
    part of f enters at all."""
    xyz, sp, occ, coef, S = _random_problem(1, real_f=False)
    A = oracle.amplitude(xyz, S, coef, A_LAT, sp, occ)
    Am = oracle.amplitude(xyz, -S, coef, A_LAT, sp, occ)
    assert np.max(np.abs(Am - np.conj(A))) > 1e-3 * np.max(np.abs(A))


def test_translation_phase():
    xyz, sp, occ, coef, S = _random_problem(2)
    t = np.array([0.3, -1.7, 2.25])
    A = oracle.amplitude(xyz, S, coef, A_LAT, sp, occ)
    At = oracle.amplitude(xyz + t, S, coef, A_LAT, sp, occ)
    assert np.max(np.abs(At - np.exp(2j * math.pi * (S @ t)) * A)) < 1e-11 * np.max(np.abs(A))


def test_species_factoring():
    """A = sum_s f_s(|S|) * sum_{j in s} w_j exp(2 i pi S.r_j)  (Section 4.2).
    f_s(|S|) is obtained as the amplitude of one atom of species s at the
    origin, and the per-species sums with f = 1."""
    xyz, sp, occ, coef, S = _random_problem(3)
    A = oracle.amplitude(xyz, S, coef, A_LAT, sp, occ)
    tot = np.zeros_like(A)
    for s in range(coef.shape[0]):
        f_s = oracle.amplitude(np.zeros((1, 3)), S, coef[s:s + 1], A_LAT)
        m = sp == s
        tot += f_s * oracle.amplitude(xyz[m], S, unit_coef(), A_LAT, occ=occ[m])
    assert np.max(np.abs(A - tot)) < 1e-11 * np.max(np.abs(A))


def test_form_factor_values():
    c = W.species_coefficients(32.0, -1.6, 0.9, 0.6)
    f0 = oracle.form_factor(c, 0.0)
    assert abs(f0 - complex(32.0 - 1.6, 0.9)) < 1e-13
    # single Gaussian, exp(-b s^2) at the (004) reflection: Bragg's law
    # d = a/4, sin(theta)/lambda = 1/(2d)
    g = np.zeros(12)
    g[0], g[4] = 1.0, 2.5
    S = np.array([[0.0, 0.0, 4.0]])
    s = 1.0 / (2.0 * A_LAT / 4.0)
    A = oracle.amplitude(np.zeros((1, 3)), S, g[None], A_LAT)
    assert abs(A[0] - math.exp(-2.5 * s * s)) < 1e-14
    # Debye-Waller alone
    g = np.zeros(12)
    g[8], g[11] = 1.0, 0.7
    A = oracle.amplitude(np.zeros((1, 3)), S, g[None], A_LAT)
    assert abs(A[0] - math.exp(-0.7 * s * s)) < 1e-14


def test_occupancy():
    xyz, sp, occ, coef, S = _random_problem(4, n_atoms=50)
    w = occ.copy()
    w[7] = 2.0
    w[9] = 0.0
    A = oracle.amplitude(xyz, S, coef, A_LAT, sp, w)
    keep = np.ones(len(xyz), bool)
    keep[9] = False
    xyz2 = np.concatenate([xyz[keep], xyz[7:8]])
    sp2 = np.concatenate([sp[keep], sp[7:8]])
    w2 = np.concatenate([w[keep], [1.0]])
    w2[list(np.nonzero(keep)[0]).index(7)] = 1.0
    A2 = oracle.amplitude(xyz2, S, coef, A_LAT, sp2, w2)
    assert np.max(np.abs(A - A2)) < 1e-11 * np.max(np.abs(A))


def test_permutation_invariance():
    xyz, sp, occ, coef, S = _random_problem(5)
    p = np.random.default_rng(0).permutation(len(xyz))
    A = oracle.amplitude(xyz, S, coef, A_LAT, sp, occ)
    Ap = oracle.amplitude(xyz[p], S, coef, A_LAT, sp[p], occ[p])
    assert np.max(np.abs(A - Ap)) < 1e-11 * np.max(np.abs(A))


# ----------------------------------------------------------------------------
# Fresnel coefficients and the four-beam DWBA sum (Section 4.3)
# ----------------------------------------------------------------------------

def fresnel_textbook(alpha, delta, beta):
    """s-polarised Fresnel reflection with angles from the surface normal:
    r = (cos ti - n cos tt) / (cos ti + n cos tt), Snell sin ti = n sin tt."""
    n = 1.0 - delta + 1j * beta
    ti = math.pi / 2 - alpha
    cos_tt = np.sqrt(1.0 - (math.sin(ti) / n) ** 2 + 0j)
    if (n * cos_tt).imag < 0:  # wave decaying into the substrate
        cos_tt = -cos_tt
    r = (math.cos(ti) - n * cos_tt) / (math.cos(ti) + n * cos_tt)
    return r, 1.0 + r


@pytest.mark.parametrize("alpha_deg", [0.01, 0.1, 0.2, 0.25, 0.3, 1.0, 5.0])
def test_fresnel_textbook(alpha_deg):
    a = math.radians(alpha_deg)
    R, T = oracle.fresnel(a, 1e-5, 1e-7)
    r_ref, t_ref = fresnel_textbook(a, 1e-5, 1e-7)
    assert abs(R - r_ref) < 1e-9
    assert abs(T - (1 + R)) < 1e-15
    assert abs(T - t_ref) < 1e-9


def test_fresnel_limits():
    delta = 1e-5
    a_c = math.acos(1.0 - delta)  # cos(alpha_c) = n for beta = 0
    for a in (0.1 * a_c, 0.5 * a_c, 0.99 * a_c):
        R, _ = oracle.fresnel(a, delta, 0.0)
        assert abs(abs(R) - 1.0) < 1e-12  # total external reflection
    for a in (1.01 * a_c, 2 * a_c):
        R, _ = oracle.fresnel(a, delta, 0.0)
        assert abs(R) < 1.0 - 1e-6 and abs(R.imag) < 1e-12
    R, _ = oracle.fresnel(1e-9, delta, 1e-7)
    assert abs(R + 1.0) < 1e-3  # grazing limit R -> -1
    a = math.radians(5.0)
    R, _ = oracle.fresnel(a, delta, 1e-7)
    asym = (delta - 1e-7j) / (2 * math.sin(a) ** 2)
    assert abs(R - asym) < 2e-2 * abs(asym)


def _kin_S(h, k, alpha_i, alpha_f, lam, a, inc_reflected, exit_reflected):
    """S (r.l.u.) of one DWBA beam from wave vectors (|k| = 1/lambda).
    The substrate mirrors the z component of a wave."""
    ki_z = -math.sin(alpha_i) / lam
    kf_z = math.sin(alpha_f) / lam
    if inc_reflected:
        ki_z = -ki_z
    if exit_reflected:
        kf_z = -kf_z
    return np.array([h, k, (kf_z - ki_z) * a])


def test_dwba_reduces_to_kinematic_without_substrate():
    rng = np.random.default_rng(21)
    xyz = rng.uniform(-5, 5, (60, 3))
    coef = W.si_ge_species()[:1]
    lam, ai = W.WAVELENGTH_10KEV, W.GID_ALPHA_I
    pts = np.stack([rng.uniform(3.8, 4.1, 40), rng.uniform(-0.1, 0.1, 40),
                    np.radians(rng.uniform(0.05, 1.0, 40))], 1)
    A = oracle.dwba(xyz, pts, coef, A_LAT, lam, ai, 0.0, 0.0)
    S1 = np.array([_kin_S(p[0], p[1], ai, p[2], lam, A_LAT, False, False) for p in pts])
    ref = oracle.amplitude(xyz, S1, coef, A_LAT)
    assert np.max(np.abs(A - ref)) < 1e-11 * np.max(np.abs(ref))


def test_dwba_four_beams():
    rng = np.random.default_rng(22)
    xyz = rng.uniform(-5, 5, (60, 3))
    xyz[:, 2] = np.abs(xyz[:, 2])
    sp = rng.integers(0, 2, 60).astype(np.int32)
    coef = W.si_ge_species()
    lam, ai, d, b = W.WAVELENGTH_10KEV, W.GID_ALPHA_I, 3e-5, 2e-6
    pts = np.stack([rng.uniform(3.8, 4.1, 30), rng.uniform(-0.1, 0.1, 30),
                    np.radians(rng.uniform(0.02, 1.0, 30))], 1)
    A = oracle.dwba(xyz, pts, coef, A_LAT, lam, ai, d, b, species=sp)
    Ri, _ = fresnel_textbook(ai, d, b)
    for m, p in enumerate(pts):
        Rf, _ = fresnel_textbook(p[2], d, b)
        beams = [(False, False, 1.0), (True, False, Ri), (False, True, Rf), (True, True, Ri * Rf)]
        tot = 0j
        for inc_r, exit_r, wgt in beams:
            S = _kin_S(p[0], p[1], ai, p[2], lam, A_LAT, inc_r, exit_r)[None]
            tot += wgt * oracle.amplitude(xyz, S, coef, A_LAT, species=sp)[0]
        assert abs(A[m] - tot) < 1e-9 * max(1.0, abs(tot))


def test_buried_dwba_without_substrate_is_the_kinematic_sum():
    """delta = beta = 0: T = 1, no refraction: the buried reading reduces to
    Eq. 2 at the vacuum beam S_1 (atoms below the surface plane)."""
    rng = np.random.default_rng(23)
    xyz = rng.uniform(-5, 5, (50, 3))
    xyz[:, 2] = -np.abs(xyz[:, 2])
    sp = rng.integers(0, 2, 50).astype(np.int32)
    coef = W.si_ge_species()
    lam, ai = W.WAVELENGTH_10KEV, W.GID_ALPHA_I
    pts = np.stack([rng.uniform(3.8, 4.1, 25), rng.uniform(-0.1, 0.1, 25), np.radians(rng.uniform(0.05, 1, 25))], 1)
    A = oracle.dwba_buried(xyz, pts, coef, A_LAT, lam, ai, 0.0, 0.0, species=sp)
    S1 = np.stack([_kin_S(p[0], p[1], ai, p[2], lam, A_LAT, False, False) for p in pts])
    ref = oracle.amplitude(xyz, S1, coef, A_LAT, species=sp)
    # sqrt(1 - cos^2 a) against sin a at a ~ 4e-3 rad: ~1e-11 relative in sigma
    assert np.allclose(A, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_buried_dwba_surface_atom_takes_both_transmission_coefficients():
    """One atom in the surface plane: |A| = |T_i T_f f|, with T from the
    textbook s-polarised transmission 2 k_z / (k_z + k_z') (not 1 + R)."""
    lam, ai, d, b = W.WAVELENGTH_10KEV, W.GID_ALPHA_I, 2e-5, 4e-7
    xyz = np.array([[0.3, -0.7, 0.0]])
    coef = W.unit_species()[None]
    pts = np.array([[4.0, 0.0, np.radians(a)] for a in (0.05, 0.15, 0.26, 0.5, 1.0)])
    A = oracle.dwba_buried(xyz, pts, coef, A_LAT, lam, ai, d, b)
    n = 1 - d + 1j * b

    def T(alpha):
        kz = np.sin(alpha)
        kzp = np.sqrt(n * n - np.cos(alpha) ** 2)
        return 2 * kz / (kz + kzp)

    for m, p in enumerate(pts):
        assert abs(abs(A[m]) - abs(T(ai) * T(p[2]))) < 1e-12
        phase = np.exp(2j * np.pi * (p[0] * xyz[0, 0] + p[1] * xyz[0, 1]))
        assert abs(A[m] - T(ai) * T(p[2]) * phase) < 1e-12


def test_buried_dwba_evanescent_decay_below_the_critical_angle():
    """beta = 0 and both angles below the critical angle sqrt(2 delta): total
    reflection, the waves are evanescent, and an atom at depth D scatters
    |T_i T_f| exp(-(2 pi a / lambda)(kappa_i + kappa_f) D) with kappa =
    sqrt(cos^2 a - (1 - delta)^2) (Snell's law with cos a > n)."""
    lam, d = W.WAVELENGTH_10KEV, 1e-5
    ac = np.sqrt(2 * d)
    ai = 0.5 * ac
    coef = W.unit_species()[None]
    pts = np.array([[4.0, 0.0, f * ac] for f in (0.3, 0.6, 0.9)])
    _, Ti = fresnel_textbook(ai, d, 0.0)
    for D in (0.0, 3.0, 40.0, 250.0):
        A = oracle.dwba_buried(np.array([[0.0, 0.0, -D]]), pts, coef, A_LAT, lam, ai, d, 0.0)
        for m, p in enumerate(pts):
            _, Tf = fresnel_textbook(p[2], d, 0.0)
            kap = [np.sqrt(np.cos(a) ** 2 - (1 - d) ** 2) for a in (ai, p[2])]
            want = abs(Ti * Tf) * np.exp(-2 * np.pi * A_LAT / lam * (kap[0] + kap[1]) * D)
            assert abs(abs(A[m]) - want) <= 1e-10 * abs(Ti * Tf)


# ----------------------------------------------------------------------------
# Misfit gradient: two routes and closed forms
# ----------------------------------------------------------------------------

def test_gradient_two_atoms_closed_form():
    """Two atoms, f = 1: |A|^2 = 2 + 2 cos(2 pi S.(r1 - r2)), so
    dL/dr1 = sum_S 2 (|A|^2 - I) (-2 sin(2 pi S.(r1-r2))) 2 pi S."""
    rng = np.random.default_rng(31)
    xyz = np.array([[0.3, -0.2, 1.1], [1.4, 0.9, -0.6]])
    S = rng.uniform(-2, 2, (64, 3))
    I_obs = rng.uniform(0, 4, 64)
    L, g = oracle.loss_grad(xyz, S, I_obs, unit_coef(), A_LAT)
    ph = 2 * math.pi * (S @ (xyz[0] - xyz[1]))
    I = 2 + 2 * np.cos(ph)
    assert abs(L - np.sum((I - I_obs) ** 2)) < 1e-10 * L
    g1 = (2 * (I - I_obs) * (-2 * np.sin(ph)) * 2 * math.pi) @ S
    assert np.allclose(g[0], g1, rtol=1e-11, atol=1e-9)
    assert np.allclose(g[1], -g1, rtol=1e-11, atol=1e-9)


def test_gradient_vs_finite_differences():
    rng = np.random.default_rng(32)
    c = W.fcc_sphere(radius_cells=2.6, seed=5)
    S = W.grid_points([W.linspace_axis(0.0, 6, step=0.05), W.linspace_axis(0.0, 6, step=0.05),
                       W.linspace_axis(4.0, 8, step=0.05)])
    pert = W.perturbed_copy(c, 0.03, seed=6)
    I_obs = np.abs(oracle.amplitude(pert.xyz, S, c.coef, A_LAT, pert.species)) ** 2
    occ = rng.uniform(0.5, 1.0, len(c.xyz))
    L, g = oracle.loss_grad(c.xyz, S, I_obs, c.coef, A_LAT, c.species, occ)
    sel = rng.choice(len(c.xyz), 12, replace=False)
    for h in (1e-5, 5e-6):
        fd = oracle.fd_grad(c.xyz, S, I_obs, c.coef, A_LAT, sel, h=h, species=c.species, occ=occ)
        assert np.max(np.abs(fd - g[sel])) < 1e-6 * np.max(np.abs(g[sel]))


def test_gradient_from_a_given_map_two_atoms_closed_form():
    """The selected-atom gradient from a map the caller already has (used for
    maps too large to sum twice) against the two-atom closed form."""
    rng = np.random.default_rng(34)
    xyz = np.array([[0.3, -0.2, 1.1], [1.4, 0.9, -0.6]])
    S = rng.uniform(-2, 2, (64, 3))
    I_obs = rng.uniform(0, 4, 64)
    A = oracle.amplitude(xyz, S, unit_coef(), A_LAT)
    L, g = oracle.loss_grad_atoms(xyz, S, A, I_obs, unit_coef(), A_LAT, atoms=[1, 0])
    ph = 2 * math.pi * (S @ (xyz[0] - xyz[1]))
    I = 2 + 2 * np.cos(ph)
    assert abs(L - np.sum((I - I_obs) ** 2)) < 1e-10 * L
    g1 = (2 * (I - I_obs) * (-2 * np.sin(ph)) * 2 * math.pi) @ S
    assert np.allclose(g[1], g1, rtol=1e-11, atol=1e-9)
    assert np.allclose(g[0], -g1, rtol=1e-11, atol=1e-9)


def test_gradient_from_a_given_map_vs_finite_differences():
    """Both given-map routes (analytic and central differences) agree, with
    species and occupancy, at two step sizes."""
    rng = np.random.default_rng(35)
    c = W.fcc_sphere(radius_cells=2.6, seed=8)
    S = rng.uniform(-0.2, 0.2, (400, 3)) + np.array([0, 0, 4.0])
    pert = W.perturbed_copy(c, 0.03, seed=9)
    I_obs = np.abs(oracle.amplitude(pert.xyz, S, c.coef, A_LAT, pert.species)) ** 2
    occ = rng.uniform(0.5, 1.0, len(c.xyz))
    A = oracle.amplitude(c.xyz, S, c.coef, A_LAT, c.species, occ)
    sel = rng.choice(len(c.xyz), 10, replace=False)
    L, g = oracle.loss_grad_atoms(c.xyz, S, A, I_obs, c.coef, A_LAT, sel, species=c.species, occ=occ)
    assert abs(L - np.sum((np.abs(A) ** 2 - I_obs) ** 2)) < 1e-12 * L
    for h in (1e-5, 5e-6):
        fd = oracle.fd_grad(c.xyz, S, I_obs, c.coef, A_LAT, sel, h=h, species=c.species, occ=occ, A=A)
        assert np.max(np.abs(fd - g)) < 1e-6 * np.max(np.abs(g))


def test_gradient_translation_invariance():
    """L depends on |A|^2 only, which a global translation leaves unchanged,
    so the gradients of all atoms sum to zero."""
    c = W.fcc_sphere(radius_cells=2.6, seed=7)
    rng = np.random.default_rng(33)
    S = rng.uniform(-0.3, 0.3, (150, 3)) + np.array([0, 0, 4.0])
    I_obs = rng.uniform(0, 1e4, 150)
    L, g = oracle.loss_grad(c.xyz, S, I_obs, c.coef, A_LAT, c.species)
    assert np.max(np.abs(g.sum(0))) < 1e-10 * np.sum(np.abs(g))


# --- Eq. 4: blocks of atoms with per-(type, S) structure factors ------------

def _fcc_block():
    """The four atoms of an fcc cell, in lattice units (the block's content)."""
    return np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]], dtype=np.float64)


def test_table_of_form_factors_reproduces_eq2():
    """Single-atom 'blocks' with F_t(S) = f_t(|S|): Eq. 4 is Eq. 2.  Two types
    and a spread of |S| catch a transposed table index or a swapped product."""
    rng = np.random.default_rng(40)
    xyz = rng.uniform(-6, 6, (97, 3))
    types = (rng.uniform(size=97) < 0.4).astype(np.int32)
    S = rng.uniform(-3, 3, (33, 3)) + np.array([0, 0, 4.0])
    coef = W.si_ge_species()
    q = np.linalg.norm(S, axis=1) / W.LATTICE_A
    table = np.array([[oracle.form_factor(coef[t], qq) for qq in q] for t in range(2)])
    got = oracle.amplitude_table(xyz, S, table, types=types)
    ref = oracle.amplitude(xyz, S, coef, W.LATTICE_A, species=types)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_blocks_of_fcc_cells_equal_the_atom_sum():
    """A displaced lattice of fcc-cell blocks (two block types with different
    content weights) against Eq. 2 over every atom of every block: the block
    structure factor F_t(S) = sum_a f e^{2 i pi S.rho_a} makes Eq. 4 exact."""
    rng = np.random.default_rng(41)
    cells = np.stack(np.meshgrid(np.arange(4), np.arange(3), np.arange(5), indexing="ij"), -1).reshape(-1, 3)
    R = cells + rng.normal(0, 0.03, cells.shape)          # r_j^0 + u_j
    btype = (rng.uniform(size=len(R)) < 0.3).astype(np.int32)
    rho = _fcc_block()
    S = rng.uniform(-0.5, 0.5, (41, 3)) + np.array([1.0, 1.0, 3.0])
    coef = W.si_ge_species()
    q = np.linalg.norm(S, axis=1) / W.LATTICE_A
    f = np.array([[oracle.form_factor(coef[t], qq) for qq in q] for t in range(2)])       # [type, M]
    geo = np.exp(2j * np.pi * (S @ rho.T))                                                 # [M, 4]
    table = f * geo.sum(1)[None, :]
    got = oracle.amplitude_table(R, S, table, types=btype)
    atoms = (R[:, None, :] + rho[None, :, :]).reshape(-1, 3)
    species = np.repeat(btype, len(rho))
    ref = oracle.amplitude(atoms, S, coef, W.LATTICE_A, species=species)
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_block_gradient_is_the_sum_of_its_atoms_gradients():
    """A rigid block moves all its atoms together, so dL/d(origin) of Eq. 4
    (F_t = sum_a f e^{2 i pi S.rho_a} held fixed) equals the sum of Eq. 2's
    dL/dr over the block's atoms: two independent routes to the gradient."""
    rng = np.random.default_rng(43)
    cells = np.stack(np.meshgrid(np.arange(3), np.arange(3), np.arange(2), indexing="ij"), -1).reshape(-1, 3)
    R = cells + rng.normal(0, 0.04, cells.shape)
    btype = (rng.uniform(size=len(R)) < 0.4).astype(np.int32)
    rho = _fcc_block()
    S = rng.uniform(-0.4, 0.4, (60, 3)) + np.array([1.0, 1.0, 3.0])
    coef = W.si_ge_species()
    q = np.linalg.norm(S, axis=1) / W.LATTICE_A
    f = np.array([[oracle.form_factor(coef[t], qq) for qq in q] for t in range(2)])
    table = f * np.exp(2j * np.pi * (S @ rho.T)).sum(1)[None, :]
    atoms = (R[:, None, :] + rho[None, :, :]).reshape(-1, 3)
    species = np.repeat(btype, len(rho))
    I_obs = rng.uniform(0, 1, len(S)) * np.abs(oracle.amplitude(atoms, S, coef, W.LATTICE_A, species=species)) ** 2
    L_blk, g_blk = oracle.loss_grad_table(R, S, I_obs, table, types=btype)
    L_at, g_at = oracle.loss_grad(atoms, S, I_obs, coef, W.LATTICE_A, species=species)
    assert abs(L_blk - L_at) < 1e-10 * L_at
    g_sum = g_at.reshape(len(R), len(rho), 3).sum(1)
    assert np.allclose(g_blk, g_sum, rtol=1e-9, atol=1e-9 * np.abs(g_sum).max())


def test_table_gradient_of_form_factors_is_eq2_gradient():
    """Single-atom blocks with F_t(S) = f_t(|S|) and occupancies: the Eq. 4
    gradient is Eq. 2's."""
    rng = np.random.default_rng(44)
    xyz = rng.uniform(-5, 5, (40, 3))
    types = (rng.uniform(size=40) < 0.5).astype(np.int32)
    occ = rng.uniform(0.3, 1.0, 40)
    S = rng.uniform(-2, 2, (25, 3)) + np.array([0, 0, 4.0])
    coef = W.si_ge_species()
    q = np.linalg.norm(S, axis=1) / W.LATTICE_A
    table = np.array([[oracle.form_factor(coef[t], qq) for qq in q] for t in range(2)])
    I_obs = rng.uniform(0, 50, len(S))
    L1, g1 = oracle.loss_grad_table(xyz, S, I_obs, table, types=types, occ=occ)
    L2, g2 = oracle.loss_grad(xyz, S, I_obs, coef, W.LATTICE_A, species=types, occ=occ)
    assert abs(L1 - L2) < 1e-11 * L2
    assert np.allclose(g1, g2, rtol=1e-10, atol=1e-10 * np.abs(g2).max())


def test_table_occupancy_and_duplication():
    rng = np.random.default_rng(42)
    xyz = rng.uniform(-4, 4, (20, 3))
    S = rng.uniform(-1, 1, (9, 3))
    table = rng.normal(size=(1, 9)) + 1j * rng.normal(size=(1, 9))
    w = np.ones(20)
    w[3] = 2.0
    w[7] = 0.0
    dup = np.concatenate([xyz, xyz[3:4]])
    keep = np.ones(21, dtype=bool)
    keep[7] = False
    a = oracle.amplitude_table(xyz, S, table, occ=w)
    b = oracle.amplitude_table(dup[keep], S, table)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12)


# --- Eq. 5/6: the FFT approximation (atoms on grid nodes, (S-H).u dropped) --

def _grid_crystal(seed, sigma):
    rng = np.random.default_rng(seed)
    nodes = np.stack(np.meshgrid(np.arange(6), np.arange(5), np.arange(4), indexing="ij"), -1).reshape(-1, 3) * 0.5
    return nodes + rng.normal(0, sigma, nodes.shape), nodes


def test_fft_approx_exact_on_the_nodes():
    """u_j = 0: nothing is dropped, Eq. 5/6 is Eq. 2 (any S, not only the FFT grid)."""
    xyz, _ = _grid_crystal(50, 0.0)
    S = np.random.default_rng(51).uniform(-0.4, 0.4, (23, 3)) + np.array([0, 0, 4.0])
    coef = W.si_ge_species()
    sp = (np.arange(len(xyz)) % 3 == 0).astype(np.int32)
    got = oracle.fft_approx(xyz, S, coef, W.LATTICE_A, [0, 0, 4], 0.5, [0, 0, 0], species=sp)
    ref = oracle.amplitude(xyz, S, coef, W.LATTICE_A, species=sp)
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_fft_approx_without_reference_is_eq2_on_the_nodes():
    """H = 0: the phase is S.R_j, Eq. 2 of the snapped positions (catches r used for R)."""
    xyz, nodes = _grid_crystal(52, 0.06)
    S = np.random.default_rng(53).uniform(-0.4, 0.4, (19, 3))
    coef = W.si_ge_species()
    got = oracle.fft_approx(xyz, S, coef, W.LATTICE_A, [0, 0, 0], 0.5, [0, 0, 0])
    ref = oracle.amplitude(nodes, S, coef, W.LATTICE_A)
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_fft_approx_error_within_the_dropped_phase_bound():
    """|A_approx - A| <= sum_j |w_j f_j| 2 pi |(S - H).u_j| (|e^{ix} - 1| <= |x|), pointwise;
    a wrong H term (H.R for H.r) breaks it at H = (0, 0, 4)."""
    xyz, nodes = _grid_crystal(54, 0.03)
    H = np.array([0.0, 0.0, 4.0])
    S = H + np.random.default_rng(55).uniform(-0.05, 0.05, (31, 3))
    coef = W.unit_species()
    got = oracle.fft_approx(xyz, S, coef, W.LATTICE_A, H, 0.5, [0, 0, 0])
    ref = oracle.amplitude(xyz, S, coef, W.LATTICE_A)
    u = xyz - nodes
    bound = 2 * np.pi * np.abs((S - H) @ u.T).sum(1)
    assert np.all(np.abs(got - ref) <= bound * (1 + 1e-9) + 1e-12)
    assert np.abs(got - ref).max() > 0  # the approximation is not silently exact
