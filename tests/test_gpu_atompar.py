"""GPU parity of the atom-parallel form of the generic sum (many atoms, few
reflections: the threads share the reflections and split the atoms) against
the FP64 oracle, through the C ABI.  Tolerance: relative L2 <= 1e-4 (FP32
path, as the S-parallel kernel)."""
import json

import numpy as np
import pytest
import torch

import __graft_entry__
import oracle
from closed_forms import rel_l2
from paper_1010_2641_gb300 import api
from paper_1010_2641_gb300 import workloads as W

pytestmark = pytest.mark.gpu
A_LAT = W.LATTICE_A


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def two_species_cloud(n, seed):
    """Random atoms in a 30^3 box, two species with a ragged split."""
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(-15.0, 15.0, (n, 3))
    species = (rng.uniform(size=n) < 0.37).astype(np.int32)
    return xyz, species, W.si_ge_species()


def run(plan, xyz, occ=None):
    x = torch.tensor(xyz, dtype=torch.float64, device="cuda:0")
    w = None if occ is None else torch.tensor(occ, dtype=torch.float32, device="cuda:0")
    A = plan.amplitude(x, w)
    plan.check()
    return A.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("K", [1, 2, 4, 8, 16])
def test_forced_list_vs_oracle(K):
    xyz, sp, coef = two_species_cloud(20011, seed=K)
    S = np.array([0.0, 0.0, 4.0]) + np.random.default_rng(100 + K).uniform(-0.3, 0.3, (300, 3))  # 2 tiles + 44
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, path="generic", atoms_per_thread=K)
    assert plan.info()["atoms_per_thread"] == K
    A = run(plan, xyz)
    ref = oracle.amplitude(xyz, S, coef, A_LAT, species=sp)
    assert rel_l2(A, ref) < 1e-4


def test_forced_grid_with_occupancy_vs_oracle():
    c = W.fcc_sphere(radius_cells=6.5, seed=2)
    occ = np.random.default_rng(3).uniform(0.1, 1.0, len(c.xyz)).astype(np.float32)
    axes = [np.linspace(-0.05, 0.05, 7), np.linspace(-0.04, 0.06, 5), np.linspace(3.9, 4.1, 9)]
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, path="generic",
                    atoms_per_thread=4)
    A = run(plan, c.xyz, occ)
    ref = oracle.amplitude(c.xyz, W.grid_points(axes), c.coef, A_LAT, species=c.species, occ=occ)
    assert rel_l2(A, ref) < 1e-4


def test_heuristic_picks_atom_parallel_for_few_reflections():
    xyz, sp, coef = two_species_cloud(200000, seed=9)
    S = np.array([1.0, 1.0, 1.0]) + np.random.default_rng(10).uniform(-0.2, 0.2, (100, 3))
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, path="generic")
    assert plan.info()["atoms_per_thread"] > 0
    A = run(plan, xyz)
    ref = oracle.amplitude(xyz, S, coef, A_LAT, species=sp)
    assert rel_l2(A, ref) < 1e-4
    # ... and the S-parallel kernel on the same problem agrees
    plan_s = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, path="generic", atoms_per_thread=-1)
    assert plan_s.info()["atoms_per_thread"] == 0
    assert rel_l2(run(plan_s, xyz), A) < 1e-5


def test_heuristic_keeps_s_parallel_for_many_reflections():
    xyz, sp, coef = two_species_cloud(5000, seed=4)
    S = np.array([0.0, 0.0, 4.0]) + np.random.default_rng(5).uniform(-0.3, 0.3, (200000, 3))
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, path="generic")
    assert plan.info()["atoms_per_thread"] == 0


def test_single_reflection_and_ragged_block():
    xyz, sp, coef = two_species_cloud(777, seed=6)  # blocks end mid-warp
    S = np.array([[0.013, -0.021, 3.987]])
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, path="generic", atoms_per_thread=2)
    A = run(plan, xyz)
    ref = oracle.amplitude(xyz, S, coef, A_LAT, species=sp)
    assert rel_l2(A, ref) < 1e-5


def test_no_atoms_gives_zero_map():
    S = np.array([0.0, 0.0, 4.0]) + np.random.default_rng(7).uniform(-0.3, 0.3, (50, 3))
    plan = api.Plan(W.unit_species(), A_LAT, 0, s_list=S, path="generic", atoms_per_thread=8)
    A = run(plan, np.zeros((0, 3)))
    assert A.shape == (50,)
    assert np.all(A == 0)


def test_autotune_considers_atom_parallel_and_caches_it(tmp_path):
    cache = tmp_path / "tune.jsonl"
    xyz, sp, coef = two_species_cloud(100000, seed=11)
    S = np.array([0.0, 0.0, 4.0]) + np.random.default_rng(12).uniform(-0.3, 0.3, (64, 3))
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, path="generic", autotune=True,
                    tune_cache=str(cache))
    k = plan.info()["atoms_per_thread"]
    entries = [json.loads(line) for line in cache.read_text().splitlines()]
    assert entries and entries[-1]["atom_k"] == k
    A = run(plan, xyz)
    ref = oracle.amplitude(xyz, S, coef, A_LAT, species=sp)
    assert rel_l2(A, ref) < 1e-4
    # a second plan of the same shape takes the cached choice
    plan2 = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, path="generic", autotune=True,
                     tune_cache=str(cache))
    assert plan2.info()["atoms_per_thread"] == k
