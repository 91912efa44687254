"""GPU parity of the batched persistent path (many crystals of uneven size,
each with its own Ewald-slice S list, one launch, CUDA-graph replay) against
the FP64 oracle, instance by instance.  Tolerance: relative L2 <= 1e-4 per
instance map."""
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


def uneven_batch(sizes, seed=40):
    xyzs, sps, Ss = [], [], []
    for b, (n, m) in enumerate(sizes):
        if n:
            c = W.fcc_sphere(radius_cells=max(0.6, (3.0 * 2 * n / (16 * np.pi)) ** (1 / 3) + 1.0), seed=seed + b)
            assert len(c.xyz) >= n
            xyz, sp = c.xyz[:n], c.species[:n]
        else:
            xyz, sp = np.zeros((0, 3)), np.zeros(0, np.int32)
        xyzs.append(xyz)
        sps.append(sp)
        Ss.append(W.ewald_slice(m, seed=seed + 100 + b) if m else np.zeros((0, 3)))
    ao = np.concatenate([[0], np.cumsum([len(x) for x in xyzs])]).astype(np.int64)
    so = np.concatenate([[0], np.cumsum([len(s) for s in Ss])]).astype(np.int64)
    return np.concatenate(xyzs), np.concatenate(sps), np.concatenate(Ss), ao, so


def run(plan, xyz, occ=None, out=None):
    x = torch.tensor(xyz, dtype=torch.float64, device="cuda:0")
    w = None if occ is None else torch.tensor(occ, dtype=torch.float32, device="cuda:0")
    A = plan.amplitude(x, w, out=out)
    plan.check()
    return A


def check_instances(A, xyz, sp, S, ao, so, coef, occ=None, tol=1e-4):
    for b in range(len(ao) - 1):
        a0, a1, s0, s1 = ao[b], ao[b + 1], so[b], so[b + 1]
        if s1 == s0:
            continue
        ref = oracle.amplitude(xyz[a0:a1], S[s0:s1], coef, A_LAT, species=sp[a0:a1],
                               occ=None if occ is None else occ[a0:a1])
        if a1 == a0:
            assert np.all(A[s0:s1] == 0)
        else:
            assert rel_l2(A[s0:s1], ref) < tol, b


SIZES = [(1, 1), (40, 300), (700, 2000), (3000, 50), (9000, 10000), (0, 100), (500, 0), (20000, 3000)]


@pytest.mark.parametrize("graph", [True, False])
def test_uneven_batch_vs_oracle(graph):
    xyz, sp, S, ao, so = uneven_batch(SIZES)
    coef = W.si_ge_species()
    occ = np.random.default_rng(1).uniform(0.5, 1.0, len(xyz)).astype(np.float32)
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, atom_off=ao, s_off=so, use_graph=graph)
    A = run(plan, xyz, occ).cpu().numpy().astype(np.complex128)
    check_instances(A, xyz, sp, S, ao, so, coef, occ)


def test_graph_replay_equals_eager_bitwise():
    xyz, sp, S, ao, so = uneven_batch(SIZES, seed=50)
    coef = W.si_ge_species()
    pg = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, atom_off=ao, s_off=so, use_graph=True)
    pe = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, atom_off=ao, s_off=so, use_graph=False)
    x = torch.tensor(xyz, dtype=torch.float64, device="cuda:0")
    out = torch.empty(len(S), dtype=torch.complex64, device="cuda:0")
    g1 = pg.amplitude(x, out=out).clone()      # capture + launch
    g2 = pg.amplitude(x, out=out).clone()      # replay
    e1 = pe.amplitude(x)
    torch.cuda.synchronize()
    assert torch.equal(g1, g2)
    assert torch.equal(g1, e1)
    # new pointers: the graph is captured again
    x2 = (x + 0.25).contiguous()
    g3 = pg.amplitude(x2)
    e3 = pe.amplitude(x2)
    assert torch.equal(g3, e3) and not torch.equal(g3, g1)


def test_fp64_batch_vs_oracle():
    xyz, sp, S, ao, so = uneven_batch(SIZES[:5], seed=60)
    coef = W.si_ge_species()
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, atom_off=ao, s_off=so, path="fp64")
    A = run(plan, xyz).cpu().numpy().astype(np.complex128)
    check_instances(A, xyz, sp, S, ao, so, coef, tol=1e-6)


def test_autotuned_batch(tmp_path):
    xyz, sp, S, ao, so = uneven_batch(SIZES, seed=70)
    coef = W.si_ge_species()
    cache = tmp_path / "tune.jsonl"
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, atom_off=ao, s_off=so, autotune=True,
                    tune_cache=str(cache))
    assert cache.exists() and "batch|" in cache.read_text()
    A = run(plan, xyz).cpu().numpy().astype(np.complex128)
    check_instances(A, xyz, sp, S, ao, so, coef)


def test_ewald_batch_full_size_sampled():
    """64 fcc crystals, 1e3-2e5 atoms and 1e4-1e6 Ewald-slice points each
    (log-uniform), one persistent launch; every 8th instance is checked on
    64 seeded points."""
    xyz, sp, coef, S, ao, so = W.ewald_batch()
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, atom_off=ao, s_off=so)
    A = run(plan, xyz).cpu().numpy().astype(np.complex128)
    assert np.all(np.isfinite(A))
    rng = np.random.default_rng(3)
    for b in range(0, 64, 8):
        a0, a1, s0, s1 = ao[b], ao[b + 1], so[b], so[b + 1]
        idx = s0 + rng.choice(s1 - s0, 64, replace=False)
        ref = oracle.amplitude(xyz[a0:a1], S[idx], coef, A_LAT, species=sp[a0:a1])
        assert rel_l2(A[idx], ref) < 1e-4, b
