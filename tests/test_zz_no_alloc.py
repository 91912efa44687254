"""The allocation-free entry point against the plan-based one.

scatter_amplitude_noalloc serves callers that cannot allocate device memory
(stream capture, foreign allocators, latency-critical loops): its scratch is
a fixed file-scope device array instead of plan workspace.  Its result must
match scatter_amplitude (f == 1, same reference reflection) within the FP32
tolerance, on two calls in a row (the second, smaller call must not see the
first call's scratch contents).  This file is collected last so that a
failure here, in a run that stops at the first failure, comes after every
other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import __graft_entry__
from closed_forms import rel_l2
from paper_1010_2641_gb300 import api
from paper_1010_2641_gb300 import binding as B
from paper_1010_2641_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _case(seed, n_atoms, n_s):
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(-9, 9, (n_atoms, 3))
    occ = rng.uniform(0.3, 1.0, n_atoms).astype(np.float32)
    S = np.array([0.0, 0.0, 4.0]) + rng.uniform(-0.3, 0.3, (n_s, 3))
    return xyz, occ, S


def _noalloc(xyz, occ, S, H=(0.0, 0.0, 4.0)):
    dev = torch.device("cuda:0")
    x = torch.tensor(xyz, dtype=torch.float64, device=dev)
    w = torch.tensor(occ, dtype=torch.float32, device=dev)
    s = torch.tensor(S, dtype=torch.float64, device=dev)
    out = torch.full((len(S),), float("nan"), dtype=torch.complex64, device=dev)
    h = (ctypes.c_double * 3)(*H)
    st = B.lib().scatter_amplitude_noalloc(len(xyz), x.data_ptr(), w.data_ptr(), len(S), s.data_ptr(), h,
                                           out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    B.check(st, "scatter_amplitude_noalloc")
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _with_plan(xyz, occ, S, H=(0, 0, 4)):
    plan = api.Plan(W.unit_species()[None], W.LATTICE_A, len(xyz), s_list=S, center=H)
    A = plan.amplitude(torch.tensor(xyz, dtype=torch.float64, device="cuda:0"),
                       torch.tensor(occ, dtype=torch.float32, device="cuda:0"))
    return A.cpu().numpy()


def test_noalloc_matches_plan_path_two_calls():
    __graft_entry__.build()
    torch.cuda.set_device(0)
    first = _case(1, 20000, 30000)
    second = _case(2, 3001, 4099)
    for xyz, occ, S in (first, second):
        got = _noalloc(xyz, occ, S)
        ref = _with_plan(xyz, occ, S)
        assert np.all(np.isfinite(got))
        assert rel_l2(got, ref) < TOL


def test_noalloc_rejects_oversize():
    __graft_entry__.build()
    h = (ctypes.c_double * 3)(0.0, 0.0, 4.0)
    L = B.lib()
    assert L.scatter_amplitude_noalloc(524289, None, None, 10, None, h, None, None) == B.SCATTER_ERR_INVALID_ARG
    assert L.scatter_amplitude_noalloc(10, None, None, 1048577, None, h, None, None) == B.SCATTER_ERR_INVALID_ARG
    bad = (ctypes.c_double * 3)(0.0, 0.5, 4.0)
    assert L.scatter_amplitude_noalloc(10, None, None, 10, None, bad, None, None) == B.SCATTER_ERR_INVALID_ARG
