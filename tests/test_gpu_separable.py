"""GPU parity of the separable tensor-core path (tcgen05, split-f16 products)
on axis-aligned grids against the FP64 oracle and closed forms.

Tolerance: relative L2 <= 1e-3 per map (the stated bound for split
tensor-core paths); the measured error is also required to stay within the
plan's own error model."""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle
from closed_forms import parallelepiped_closed_form, rel_l2
from paper_1010_2641_gb300 import api
from paper_1010_2641_gb300 import workloads as W

pytestmark = pytest.mark.gpu
A_LAT = W.LATTICE_A
TOL_TC = 1e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def run(plan, xyz, occ=None):
    A = plan.amplitude(torch.tensor(xyz, dtype=torch.float64, device="cuda:0"),
                       None if occ is None else torch.tensor(occ, dtype=torch.float32, device="cuda:0"))
    plan.check()
    return A.cpu().numpy().astype(np.complex128)


def test_tiny_cube_dirichlet():
    xyz = W.simple_cubic((10, 10, 10))
    axes = [W.linspace_axis(c, 32, half_width=0.5) for c in (0.0, 0.0, 4.0)]
    S = W.grid_points(axes)
    plan = api.Plan(W.unit_species()[None], A_LAT, len(xyz), axes=axes, path="separable")
    A = run(plan, xyz)
    assert rel_l2(A, parallelepiped_closed_form((10, 10, 10), S)) < TOL_TC
    assert rel_l2(A, oracle.amplitude(xyz, S, W.unit_species()[None], A_LAT)) < TOL_TC


# n0 sets the M tiles (2 n0 rows of 128): 130 -> 3 tiles in 2 pairs (the
# CTA-pair kernel with a zero padding tile), 200 -> 2 full pairs, 300 -> 5
# tiles in 3 pairs and 384 -> 3 full pairs (two on the CTA-pair kernel, the
# last on the one-CTA kernel), 520 -> 9 tiles in 5 pairs
@pytest.mark.parametrize("shape,split", [((16, 16, 64), 0), ((5, 7, 13), 0), ((70, 3, 37), 2), ((1, 1, 1), 0),
                                         ((33, 9, 30), 5), ((130, 5, 11), 0), ((200, 4, 9), 3),
                                         ((300, 3, 7), 0), ((384, 2, 9), 2), ((520, 2, 5), 0)])
def test_sphere_grids(shape, split):
    c = W.fcc_sphere(radius_cells=4.3, seed=9)
    occ = np.random.default_rng(3).uniform(0.5, 1.0, len(c.xyz)).astype(np.float32)
    axes = [W.linspace_axis(0.0, shape[0], step=0.004), W.linspace_axis(0.0, shape[1], step=0.004),
            W.linspace_axis(4.0, shape[2], step=0.004)]
    S = W.grid_points(axes)
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, path="separable", split_k=split)
    A = run(plan, c.xyz, occ)
    ref = oracle.amplitude(c.xyz, S, c.coef, A_LAT, species=c.species, occ=occ)
    err = rel_l2(A, ref)
    assert err < TOL_TC
    _, model = plan.error_bound(radius=6.0)
    assert err < max(model, 1e-5) * 10


@pytest.mark.parametrize("n0", [200, 130])
def test_in_kernel_a_tiles_equal_the_table_route(n0):
    """A grid of one N tile (every A tile read by one cluster) forms its A
    tiles inside the CTA-pair kernel; a wider grid keeps the A table.  The
    two forms compute the same A values in the same order, so the points the
    two grids share agree bit for bit (same atom chunks).  n0 = 130 has a
    zero padding tile in its second M-tile pair."""
    c = W.fcc_sphere(radius_cells=6.2, seed=27)
    occ = np.random.default_rng(28).uniform(0.5, 1.0, len(c.xyz)).astype(np.float32)
    ax0 = W.linspace_axis(0.0, n0, step=0.004)
    ax2 = W.linspace_axis(4.0, 9, step=0.004)
    ax1_wide = W.linspace_axis(0.0, 64, step=0.004)
    ax1_narrow = ax1_wide[:4]
    narrow = api.Plan(c.coef, A_LAT, len(c.xyz), axes=[ax0, ax1_narrow, ax2], atom_species=c.species,
                      path="separable", split_k=3)
    wide = api.Plan(c.coef, A_LAT, len(c.xyz), axes=[ax0, ax1_wide, ax2], atom_species=c.species,
                    path="separable", split_k=3)
    An = run(narrow, c.xyz, occ).reshape(n0, 4, 9)
    Aw = run(wide, c.xyz, occ).reshape(n0, 64, 9)
    assert np.array_equal(An.view(np.float64), Aw[:, :4, :].copy().view(np.float64))
    S = W.grid_points([ax0, ax1_narrow, ax2])
    idx = np.sort(np.random.default_rng(29).choice(len(S), 512, replace=False))
    ref = oracle.amplitude(c.xyz, S[idx], c.coef, A_LAT, species=c.species, occ=occ)
    assert rel_l2(An.reshape(-1)[idx], ref) < TOL_TC


def test_off_centre_and_generic_agree():
    c = W.fcc_sphere(radius_cells=3.5, seed=19)
    xyz = c.xyz + np.array([31.2, -17.9, 8.4])
    axes = [W.linspace_axis(0.01, 20, step=0.006), W.linspace_axis(-0.02, 12, step=0.006),
            W.linspace_axis(3.98, 40, step=0.006)]
    S = W.grid_points(axes)
    ps = api.Plan(c.coef, A_LAT, len(xyz), axes=axes, atom_species=c.species, path="separable")
    pg = api.Plan(c.coef, A_LAT, len(xyz), axes=axes, atom_species=c.species, path="generic")
    As, Ag = run(ps, xyz), run(pg, xyz)
    ref = oracle.amplitude(xyz, S, c.coef, A_LAT, species=c.species)
    assert rel_l2(As, ref) < TOL_TC
    assert rel_l2(Ag, ref) < 1e-4
    assert ps.info()["shift"] == [31.0, -18.0, 8.0]


@pytest.mark.parametrize("n0", [2, 200, 300])
def test_no_atoms(n0):
    """An empty crystal gives a zero map on the one-CTA kernel (n0 = 2),
    on the CTA pair forming its own A tiles (n0 = 200: two M-tile pairs, one
    N tile) and on the CTA pair with the one-CTA kernel beside it (n0 = 300:
    three pairs)."""
    axes = [W.linspace_axis(0.0, n0, step=0.01), np.array([0.0]), np.array([4.0, 4.1, 4.2])]
    plan = api.Plan(W.unit_species()[None], A_LAT, 0, axes=axes, path="separable")
    A = plan.amplitude(torch.empty(0, 3, dtype=torch.float64, device="cuda:0"))
    plan.check()
    assert A.shape == (n0 * 3,)
    assert torch.all(A == 0)


def test_list_plans_rejected():
    from paper_1010_2641_gb300 import binding as B
    with pytest.raises(B.ScatterError) as e:
        api.Plan(W.unit_species()[None], A_LAT, 10, s_list=np.zeros((5, 3)), path="separable")
    assert e.value.status == B.SCATTER_ERR_UNSUPPORTED


def test_strained_sphere_full_size_sampled():
    c = W.fcc_sphere()
    axes = [W.linspace_axis(0.0, 256, step=0.002), W.linspace_axis(0.0, 256, step=0.002),
            W.linspace_axis(4.0, 64, step=0.002)]
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, path="separable")
    A = run(plan, c.xyz)
    assert np.all(np.isfinite(A))
    rng = np.random.default_rng(0)
    idx = rng.choice(A.shape[0], 768, replace=False)
    idx[:8] = np.argsort(np.abs(A))[-8:]
    ref = oracle.amplitude(c.xyz, W.grid_points(axes)[idx], c.coef, A_LAT, species=c.species)
    assert rel_l2(A[idx], ref) < TOL_TC


def test_wide_grid_takes_the_reduced_phase_path():
    """A k axis spanning +-3 r.l.u. over a crystal of radius 8.5 cells puts
    |s_b y'| near 27 cycles, above the limit under which B phases skip the
    exact mod-1 reduction: this map exercises the reduced branch."""
    c = W.fcc_sphere(radius_cells=8.5, shell_cells=2.0, seed=71)
    axes = [np.linspace(-0.05, 0.05, 5), np.linspace(-3.0, 3.0, 61), np.linspace(3.9, 4.1, 17)]
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, path="separable")
    A = plan.amplitude(torch.tensor(c.xyz, dtype=torch.float64, device="cuda:0")).cpu().numpy().reshape(-1)
    plan.check()
    ref = oracle.amplitude(c.xyz, W.grid_points(axes), c.coef, A_LAT, species=c.species)
    assert rel_l2(A, ref) < 1e-4


def test_repeated_calls_are_bitwise_identical():
    """Chunks of more than 256 steps read the accumulators out several times
    (a store, then L2 reductions in program order): the map, and the
    tensor-core gradient on the same plan, repeat bit for bit."""
    c = W.fcc_sphere(radius_cells=8.0, seed=77)
    axes = [W.linspace_axis(0.0, 40, step=0.004), W.linspace_axis(0.0, 9, step=0.004),
            W.linspace_axis(4.0, 33, step=0.004)]
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, path="separable", split_k=1)
    assert plan.info()["n_atoms_padded"] // 16 > 2 * 256  # several read-outs per chunk
    x = torch.tensor(c.xyz, dtype=torch.float64, device="cuda:0")
    a1 = plan.amplitude(x).clone()
    a2 = plan.amplitude(x)
    plan.check()
    assert torch.equal(a1, a2)
    I_obs = (a1.abs() ** 2 * 1.02).float()
    _, g1 = plan.backward(x, a1, I_obs)
    g1 = g1.clone()
    _, g2 = plan.backward(x, a1, I_obs)
    plan.check()
    assert torch.equal(g1, g2)
    S = W.grid_points(axes)
    idx = np.random.default_rng(5).choice(len(S), 256, replace=False)
    ref = oracle.amplitude(c.xyz, S[idx], c.coef, A_LAT, species=c.species)
    assert rel_l2(a1.cpu().numpy().astype(np.complex128)[idx], ref) < TOL_TC
