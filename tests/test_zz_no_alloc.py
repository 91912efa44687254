"""The allocation-free entry point against the FP64 oracle and the plan path.

scatter_amplitude_noalloc serves callers that cannot allocate device memory:
code running while a stream is captured into a graph, processes whose
device memory belongs to another allocator, latency-critical loops.  Its
scratch is a fixed file-scope device array instead of plan workspace, so
every call reuses what the previous call left there.  These tests check its
result (f == 1) against the oracle element by element on calls in a row of
different sizes, on a crystal far from the origin, on a long chain that
takes the exact-product phases, at the largest sizes it accepts (sampled),
that a non-finite input poisons the whole output while the next call is
clean again, and a call captured into a CUDA graph and replayed on new
inputs in the same buffers.  The plan-based call is a second reference.  This file is
collected last so that a failure here, in a run that stops at the first
failure, comes after every other test.
"""
import ctypes

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
TOL = 1e-4
MAX_ATOMS, MAX_POINTS = 524288, 1048576
UNIT = W.unit_species()[None]


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _case(seed, n_atoms, n_s, offset=0.0):
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(-9, 9, (n_atoms, 3)) + offset
    occ = rng.uniform(0.3, 1.0, n_atoms).astype(np.float32)
    S = np.array([0.0, 0.0, 4.0]) + rng.uniform(-0.3, 0.3, (n_s, 3))
    return xyz, occ, S


def _noalloc(xyz, occ, S, H=(0.0, 0.0, 4.0)):
    dev = torch.device("cuda:0")
    x = torch.tensor(xyz, dtype=torch.float64, device=dev)
    w = None if occ is None else torch.tensor(occ, dtype=torch.float32, device=dev)
    s = torch.tensor(S, dtype=torch.float64, device=dev)
    out = torch.full((len(S),), float("nan"), dtype=torch.complex64, device=dev)
    h = (ctypes.c_double * 3)(*H)
    st = B.lib().scatter_amplitude_noalloc(len(xyz), x.data_ptr(), None if w is None else w.data_ptr(), len(S),
                                           s.data_ptr(), h, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    B.check(st, "scatter_amplitude_noalloc")
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)


def _with_plan(xyz, occ, S, H=(0, 0, 4)):
    plan = api.Plan(UNIT, W.LATTICE_A, len(xyz), s_list=S, center=H)
    A = plan.amplitude(torch.tensor(xyz, dtype=torch.float64, device="cuda:0"),
                       torch.tensor(occ, dtype=torch.float32, device="cuda:0"))
    return A.cpu().numpy().astype(np.complex128)


def test_noalloc_matches_oracle_two_calls():
    """Two calls in a row, the second smaller: the second must not see the
    first call's scratch.  Both against the oracle, and against the plan path."""
    for xyz, occ, S in (_case(1, 20000, 30000), _case(2, 3001, 4099)):
        got = _noalloc(xyz, occ, S)
        assert np.all(np.isfinite(got))
        assert rel_l2(got, oracle.amplitude(xyz, S, UNIT, W.LATTICE_A, occ=occ)) < TOL
        assert rel_l2(got, _with_plan(xyz, occ, S)) < TOL


def test_noalloc_crystal_far_from_the_origin():
    """Positions 60 cells from the origin: the call centres them itself (the
    translation phase comes back exactly), so the error stays at the FP32
    level."""
    xyz, occ, S = _case(3, 5000, 6000, offset=60.0)
    got = _noalloc(xyz, occ, S)
    assert rel_l2(got, oracle.amplitude(xyz, S, UNIT, W.LATTICE_A, occ=occ)) < TOL


def test_noalloc_long_chain_takes_exact_phases():
    """A displaced 20,000-atom chain starting at the origin, reflections within
    +-0.1 of (400): |s x'| reaches ~1000 cycles after centring, above the 128
    cycles from which the exact-product phases (s as a double-float) run."""
    n = 20000
    xyz = W.linear_chain(n, sigma=0.02, seed=31)
    rng = np.random.default_rng(32)
    S = np.zeros((600, 3))
    S[:, 0] = 4.0 + rng.uniform(-0.1, 0.1, len(S))
    S[:, 1:] = rng.uniform(-0.02, 0.02, (len(S), 2))
    got = _noalloc(xyz, None, S, H=(4.0, 0.0, 0.0))
    err = rel_l2(got, oracle.amplitude(xyz, S, UNIT, W.LATTICE_A))
    print(f"noalloc long chain: rel L2 {err:.1e}")
    assert err < TOL


def test_noalloc_non_finite_input_poisons_the_output():
    """No plan carries a status word here: a non-finite position makes every
    output NaN, and the next call (clean input) is correct again."""
    xyz, occ, S = _case(4, 2000, 3000)
    bad = xyz.copy()
    bad[17, 1] = np.nan
    assert np.all(np.isnan(_noalloc(bad, occ, S)))
    got = _noalloc(xyz, occ, S)
    assert rel_l2(got, oracle.amplitude(xyz, S, UNIT, W.LATTICE_A, occ=occ)) < TOL


def test_noalloc_at_the_size_limits_sampled():
    """524,288 atoms x 1,048,576 points (the stated maxima), checked on 96
    seeded points against the oracle."""
    rng = np.random.default_rng(5)
    xyz = rng.uniform(0, 80, (MAX_ATOMS, 3))
    S = np.array([0.0, 0.0, 4.0]) + rng.uniform(-0.5, 0.5, (MAX_POINTS, 3))
    got = _noalloc(xyz, None, S)
    assert np.all(np.isfinite(got))
    idx = rng.choice(MAX_POINTS, 96, replace=False)
    assert rel_l2(got[idx], oracle.amplitude(xyz, S[idx], UNIT, W.LATTICE_A)) < TOL


def test_noalloc_captured_in_a_graph_and_replayed_on_new_inputs():
    """What the entry point is for: after one call outside capture (which
    looks its scratch up), a call is captured into a CUDA graph, new inputs
    are written into the same buffers and the graph replays them."""
    dev = torch.device("cuda:0")
    xyz, occ, S = _case(61, 3000, 2500)
    x = torch.tensor(xyz, dtype=torch.float64, device=dev)
    w = torch.tensor(occ, dtype=torch.float32, device=dev)
    s = torch.tensor(S, dtype=torch.float64, device=dev)
    out = torch.full((len(S),), float("nan"), dtype=torch.complex64, device=dev)
    h = (ctypes.c_double * 3)(0.0, 0.0, 4.0)

    def call(stream):
        B.check(B.lib().scatter_amplitude_noalloc(len(xyz), x.data_ptr(), w.data_ptr(), len(S), s.data_ptr(), h,
                                                  out.data_ptr(), stream.cuda_stream), "scatter_amplitude_noalloc")

    call(torch.cuda.current_stream())
    torch.cuda.synchronize()
    ref1 = oracle.amplitude(xyz, S, UNIT, W.LATTICE_A, occ=occ)
    assert rel_l2(out.cpu().numpy().astype(np.complex128), ref1) < TOL
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        call(side)
    xyz2, occ2, S2 = _case(62, 3000, 2500, offset=3.0)
    x.copy_(torch.tensor(xyz2, dtype=torch.float64))
    w.copy_(torch.tensor(occ2, dtype=torch.float32))
    s.copy_(torch.tensor(S2, dtype=torch.float64))
    out.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    ref2 = oracle.amplitude(xyz2, S2, UNIT, W.LATTICE_A, occ=occ2)
    assert rel_l2(out.cpu().numpy().astype(np.complex128), ref2) < TOL


def test_noalloc_rejects_oversize():
    h = (ctypes.c_double * 3)(0.0, 0.0, 4.0)
    L = B.lib()
    assert L.scatter_amplitude_noalloc(MAX_ATOMS + 1, None, None, 10, None, h, None, None) == B.SCATTER_ERR_INVALID_ARG
    assert L.scatter_amplitude_noalloc(10, None, None, MAX_POINTS + 1, None, h, None, None) == B.SCATTER_ERR_INVALID_ARG
    bad = (ctypes.c_double * 3)(0.0, 0.5, 4.0)
    assert L.scatter_amplitude_noalloc(10, None, None, 10, None, bad, None, None) == B.SCATTER_ERR_INVALID_ARG
