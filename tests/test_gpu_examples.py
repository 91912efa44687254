"""The first worked example of Section 4 at its full size: a simple cubic
crystal of 100 x 100 x 100 cells (1,000,000 atoms, f = 1) on the 200 x 200
(h, l) map around (004) at k = 0.

The perfect crystal has a closed form: per axis the geometric series of
Section 2.3 over 100 cells, times the phase of the crystal's origin (-50,
-50, 0), so the whole map of every path is checked against it.  The
strained crystal of the same example (u_z = 1e-6 z (x^2 + y^2)) is checked
against the FP64 oracle on seeded sampled points.
"""
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
A_LAT = W.LATTICE_A


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _map(xyz, path):
    axes = W.example_cube_axes()
    plan = api.Plan(W.unit_species()[None], A_LAT, len(xyz), axes=axes, path=path)
    if path == "auto":
        assert plan.info()["path"] == B.SCATTER_PATH_SEPARABLE
    A = plan.amplitude(torch.tensor(xyz, dtype=torch.float64, device="cuda:0"))
    plan.check()
    return A.cpu().numpy().astype(np.complex128), W.grid_points(axes)


@pytest.mark.parametrize("path,tol", [("generic", 1e-4), ("separable", 1e-4), ("auto", 1e-4)])
def test_perfect_cube_whole_map_against_the_closed_form(path, tol):
    """AUTO takes the tensor cores: 200 columns are few, but 4e10 pairs
    make the contraction ~10x faster than the generic kernel."""
    A, S = _map(W.example_cube_100(), path)
    ref = parallelepiped_closed_form((100, 100, 100), S) * np.exp(2j * np.pi * (-50.0 * S[:, 0] - 50.0 * S[:, 1]))
    err = rel_l2(A, ref)
    print(f"perfect 100^3 cube ({path}): rel L2 {err:.1e} over all {len(S)} points")
    assert err < tol


@pytest.mark.parametrize("path,tol", [("generic", 1e-4), ("separable", 1e-4)])
def test_strained_cube_sampled_against_the_oracle(path, tol):
    xyz = W.example_cube_100(strained=True)
    A, S = _map(xyz, path)
    idx = np.sort(np.random.default_rng(91).choice(len(S), 256, replace=False))
    ref = oracle.amplitude(xyz, S[idx], W.unit_species()[None], A_LAT)
    err = rel_l2(A[idx], ref)
    print(f"strained 100^3 cube ({path}): rel L2 {err:.1e} on 256 sampled points")
    assert err < tol
