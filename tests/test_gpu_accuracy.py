"""The paper's accuracy test (Section 2.3) on the GPU: perfect linear chains of
1e3, 1e4 and 1e5 atoms at x = 0..N-1, H every 0.001 r.l.u. from 0.5 to 1.5,
against the closed form sin(pi N H) / sin(pi H).

On that grid the closed form is N at H = 1 and exactly zero at every other
point (N H is an integer), so what a single-precision sum shows there is its
noise floor.  Reading of the paper's "reliable dynamic range": the peak
intensity over the largest intensity the GPU reports at the closed form's
zeros; the paper finds > 1e8 always and ~1e10 for > 99 % of the points on
its single-precision GPU.  Chains this long make phases of thousands of
cycles, so the FP32 kernels take their exact-product route (each product's
rounding error restored), which is what keeps the floor ~1e-14 of the peak.  A second grid, offset by 0.000437 r.l.u. (no
zeros: N times the offset is not an integer), measures the relative error
where the closed form is small but non-zero; it is reported, and the FP32
error is compared with the paper's noise reference, a chain displaced by
N(0, 1e-3) per atom."""
import numpy as np
import pytest
import torch

import __graft_entry__
from closed_forms import dirichlet
from paper_1010_2641_gb300 import api
from paper_1010_2641_gb300 import workloads as W

pytestmark = pytest.mark.gpu
A_LAT = W.LATTICE_A
K = np.arange(-500, 501)
H_PAPER = 1.0 + 0.001 * K          # the paper's grid: the peak and exact zeros
H_OFFSET = 1.000437 + 0.001 * K    # no zeros of the closed form


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def chain_amplitude(N, H, path, sigma=0.0):
    xyz = W.linear_chain(N, sigma=sigma, seed=7)
    plan = api.Plan(W.unit_species()[None], A_LAT, N, axes=[H, np.array([0.0]), np.array([0.0])], path=path)
    A = plan.amplitude(torch.tensor(xyz, dtype=torch.float64, device="cuda:0"))
    plan.check()
    return A.cpu().numpy().astype(np.complex128).reshape(-1)


@pytest.mark.parametrize("N", [1000, 10000, 100000])
def test_chain_dynamic_range_as_in_the_paper(N):
    peak = int(np.argmin(np.abs(H_PAPER - 1.0)))
    for path in ("generic", "fp64"):
        I = np.abs(chain_amplitude(N, H_PAPER, path)) ** 2
        assert abs(I[peak] / N ** 2 - 1.0) < 1e-5
        floor = np.delete(I, peak)
        dr = I[peak] / floor.max()
        frac = float(np.mean(floor < I[peak] * 1e-10))
        print(f"chain N={N} {path}: dynamic range {dr:.2e}, {100 * frac:.1f} % of the zeros below 1e-10 of the peak")
        if path == "generic":  # the paper: > 1e8 always, ~1e10 for > 99 % of the points
            assert dr > 1e10
            assert frac > 0.99


@pytest.mark.parametrize("N", [1000, 10000, 100000])
def test_chain_relative_error_off_the_zeros(N):
    ref = dirichlet(N, H_OFFSET)
    I_ref = np.abs(ref) ** 2
    rel = np.abs(np.abs(chain_amplitude(N, H_OFFSET, "generic")) ** 2 - I_ref) / I_ref
    rel64 = np.abs(np.abs(chain_amplitude(N, H_OFFSET, "fp64")) ** 2 - I_ref) / I_ref
    noise = np.abs(np.abs(chain_amplitude(N, H_OFFSET, "generic", sigma=1e-3)) ** 2 - I_ref) / I_ref
    print(f"chain N={N} offset grid: FP32 median / max relative intensity error {np.median(rel):.1e} / {rel.max():.1e}, "
          f"FP64 kernel {rel64.max():.1e}, 1e-3 displacement noise median {np.median(noise):.1e}")
    assert rel64.max() < 1e-6
    assert rel.max() < 0.05  # long chains take the exact-product phases
    assert np.median(rel) < np.median(noise)


@pytest.mark.parametrize("axis", [0, 2])
def test_separable_chain_dynamic_range(axis):
    """The tensor-core path on a 1e5-atom chain along its table axis (a) and
    along its formed axis (c): exact products in the per-call table and in
    the formed operand keep the noise floor of the paper's grid."""
    N = 100000
    xyz = W.linear_chain(N)
    axes = [H_PAPER, np.array([0.0]), np.array([0.0])]
    if axis == 2:
        xyz = xyz[:, [1, 2, 0]]
        axes = [np.array([0.0]), np.array([0.0]), H_PAPER]
    plan = api.Plan(W.unit_species()[None], A_LAT, N, axes=axes, path="separable")
    A = plan.amplitude(torch.tensor(xyz, dtype=torch.float64, device="cuda:0"))
    plan.check()
    I = np.abs(A.cpu().numpy().astype(np.complex128).reshape(-1)) ** 2
    peak = int(np.argmin(np.abs(H_PAPER - 1.0)))
    assert abs(I[peak] / N ** 2 - 1.0) < 1e-4
    dr = I[peak] / np.delete(I, peak).max()
    print(f"separable chain N={N} along axis {axis}: dynamic range {dr:.2e}")
    assert dr > 1e8


@pytest.mark.parametrize("kind", ["line", "list", "separable"])
def test_long_chain_gradient(kind):
    """The adjoints on a 2e4-atom displaced chain (phases of thousands of
    cycles): the FP32 line kernel's per-tile bases and re-seeds take exact
    products, the list kernel its exact-product route, and on a SEPARABLE
    plan the tensor-core adjoint's final rotation; against the oracle."""
    import oracle
    from closed_forms import rel_l2
    N = 20000
    xyz = W.linear_chain(N, sigma=0.02, seed=11)[:, [1, 2, 0]]  # along z: the l axis
    pert = W.linear_chain(N, sigma=0.02, seed=12)[:, [1, 2, 0]]
    l = 1.0 + 0.0005 + 0.001 * np.arange(-150, 151)
    S = np.stack([np.zeros_like(l), np.zeros_like(l), l], 1)
    coef = W.unit_species()[None]
    I_obs = (np.abs(oracle.amplitude(pert, S, coef, A_LAT)) ** 2).astype(np.float32)
    if kind in ("line", "separable"):
        plan = api.Plan(coef, A_LAT, N, axes=[np.array([0.0]), np.array([0.0]), l],
                        path="generic" if kind == "line" else "separable")
    else:
        plan = api.Plan(coef, A_LAT, N, s_list=S, path="generic")
    x = torch.tensor(xyz, dtype=torch.float64, device="cuda:0")
    A = plan.amplitude(x)
    loss, grad = plan.backward(x, A, torch.tensor(I_obs, device="cuda:0"))
    plan.check()
    assert plan.info()["adjoint_form"] == {"line": 2, "list": 1, "separable": 3}[kind]
    L_ref, g_ref = oracle.loss_grad(xyz, S, I_obs, coef, A_LAT)
    err = rel_l2(grad.cpu().numpy(), g_ref)
    print(f"long chain gradient ({kind}): loss rel {abs(loss.item() - L_ref) / L_ref:.1e}, gradient rel L2 {err:.1e}")
    assert abs(loss.item() - L_ref) < 1e-3 * L_ref
    assert err < 1e-3
