"""GPU parity of the FFT approximation (Eq. 5/6) against its FP64 oracle
(the same approximation as a direct sum), and its relation to the exact sum
(Eq. 2) under the validity metric of Eq. 7.  Tolerance: relative L2 <= 1e-5
against the oracle (FP32 transform)."""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle
from closed_forms import rel_l2
from paper_1010_2641_gb300 import api
from paper_1010_2641_gb300 import binding as B
from paper_1010_2641_gb300 import workloads as W

pytestmark = pytest.mark.gpu
A_LAT = W.LATTICE_A


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def dev(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda:0")


def fft_case(c, n=(24, 26, 32), step=0.5, origin=None, occ=None):
    origin = np.floor(c.xyz.min(0)) - 1.0 if origin is None else np.asarray(origin, float)
    plan = api.FFTPlan(c.coef, A_LAT, len(c.xyz), center=(0, 0, 4), step=step, origin=origin, n=n)
    A = plan.amplitude(dev(c.xyz), dev(c.species, torch.int32), None if occ is None else dev(occ, torch.float32))
    return plan, origin, A.cpu().numpy().astype(np.complex128).reshape(-1)


def test_fft_vs_oracle_strained_sphere():
    c = W.fcc_sphere(radius_cells=4.6, shell_cells=1.0, seed=31)
    occ = np.random.default_rng(32).uniform(0.4, 1.0, len(c.xyz))
    plan, origin, A = fft_case(c, occ=occ)
    S = W.grid_points(plan.axes())
    ref = oracle.fft_approx(c.xyz, S, c.coef, A_LAT, (0, 0, 4), 0.5, origin, species=c.species, occ=occ)
    assert rel_l2(A, ref) < 1e-5
    m, outside = plan.validity()
    assert outside == 0
    u = c.xyz - (origin + 0.5 * np.rint((c.xyz - origin) / 0.5))
    qmax = np.array([(k // 2) / (k * 0.5) for k in plan.n])
    assert abs(m - (np.abs(u) @ qmax).max()) < 1e-5 * max(m, 1e-6)


def test_fft_on_the_nodes_equals_the_exact_sum():
    """Undisplaced fcc atoms sit on the nodes of the 0.5-step grid: nothing is
    dropped, and the map equals Eq. 2 (oracle and the GPU's direct sum)."""
    xyz = W.simple_cubic((6, 5, 4)).astype(np.float64) * 1.0
    xyz = np.concatenate([xyz, xyz + [0.5, 0.5, 0], xyz + [0.5, 0, 0.5], xyz + [0, 0.5, 0.5]])
    c = W.Crystal(xyz=xyz, species=np.zeros(len(xyz), np.int32), coef=W.si_ge_species()[:1])
    plan, origin, A = fft_case(c, n=(16, 16, 16))
    assert plan.validity()[0] < 1e-6
    S = W.grid_points(plan.axes())
    ref = oracle.amplitude(xyz, S, c.coef, A_LAT)
    assert rel_l2(A, ref) < 1e-5
    direct = api.Plan(c.coef, A_LAT, len(xyz), axes=plan.axes(), path="generic").amplitude(dev(xyz)).cpu().numpy()
    assert rel_l2(A, direct) < 1e-5


def test_dropped_phase_bound_against_the_exact_sum():
    """|A_fft - A| <= sum_j |w f| 2 pi |(S-H).u_j| pointwise, and the error
    grows with the displacements (Eq. 7)."""
    errs = []
    for sigma in (0.005, 0.05):
        rng = np.random.default_rng(33)
        base = W.fcc_sphere(radius_cells=3.6, seed=34, strain=0.0, sigma_angstrom=0.0)
        xyz = base.xyz + rng.normal(0, sigma, base.xyz.shape)
        c = W.Crystal(xyz=xyz, species=np.zeros(len(xyz), np.int32), coef=W.unit_species())
        plan, origin, A = fft_case(c, n=(20, 20, 20))
        assert plan.validity()[1] == 0
        S = W.grid_points(plan.axes())
        exact = oracle.amplitude(xyz, S, c.coef, A_LAT)
        u = xyz - (origin + 0.5 * np.rint((xyz - origin) / 0.5))
        bound = 2 * np.pi * np.abs((S - np.array([0, 0, 4.0])) @ u.T).sum(1)
        assert np.all(np.abs(A - exact) <= bound * (1 + 1e-4) + 1e-3)
        errs.append(rel_l2(A, exact))
    assert errs[1] > 5 * errs[0]


def test_outside_atoms_counted_and_bad_species_reported():
    c = W.fcc_sphere(radius_cells=3.0, seed=35)
    origin = np.floor(c.xyz.min(0)) - 1.0
    xyz = np.concatenate([c.xyz, [[origin[0] - 5.0, 0.0, 0.0]]])
    plan = api.FFTPlan(c.coef, A_LAT, len(xyz), center=(0, 0, 4), step=0.5, origin=origin, n=(24, 24, 24))
    plan.amplitude(dev(xyz), dev(np.append(c.species, 0), torch.int32))
    assert plan.validity()[1] == 1
    bad = np.append(c.species, 0).astype(np.int32)
    bad[0] = 7  # an atom inside the grid (atoms outside are dropped before their species is read)
    plan.amplitude(dev(xyz), dev(bad, torch.int32))
    with pytest.raises(B.ScatterError):
        plan.validity()
