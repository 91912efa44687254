"""GPU parity of the misfit L = sum (|A|^2 - I_obs)^2 and of its gradient
dL/dr_j (hand-written adjoint kernel) against the FP64 oracle's analytic
gradient and its central finite differences, through the C ABI and through
torch.autograd.

Tolerances: loss relative error <= 1e-4 (FP32 amplitudes, FP64 reduction);
gradients relative L2 <= 1e-3 against FP64 finite differences and the
oracle's analytic gradient.
"""
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
TOL_GRAD = 1e-3


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def dev(x, dtype=torch.float64, grad=False):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda:0", requires_grad=grad)


def _case(radius=3.2, shape=(9, 7, 13), step=0.02, seed=11, occ=False, offset=(0.0, 0.0, 0.0)):
    c = W.fcc_sphere(radius_cells=radius, seed=seed)
    c.xyz = c.xyz + np.asarray(offset)
    axes = [W.linspace_axis(0.0, shape[0], step=step), W.linspace_axis(0.0, shape[1], step=step),
            W.linspace_axis(4.0, shape[2], step=step)]
    S = W.grid_points(axes)
    pert = W.perturbed_copy(c, 0.03, seed=seed + 1)
    I_obs = (np.abs(oracle.amplitude(pert.xyz, S, c.coef, A_LAT, species=c.species)) ** 2).astype(np.float32)
    w = np.random.default_rng(seed).uniform(0.5, 1.0, len(c.xyz)).astype(np.float32) if occ else None
    return c, axes, S, I_obs, w


@pytest.mark.parametrize("occ,offset", [(False, (0, 0, 0)), (True, (0, 0, 0)), (True, (40.4, -7.7, 13.2))])
def test_misfit_and_gradient_vs_oracle(occ, offset):
    c, axes, S, I_obs, w = _case(occ=occ, offset=offset)
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, path="generic")
    xyz = dev(c.xyz, grad=True)
    loss = api.misfit(xyz, plan, dev(I_obs, torch.float32), None if w is None else dev(w, torch.float32))
    loss.backward()
    plan.check()
    L_ref, g_ref = oracle.loss_grad(c.xyz, S, I_obs, c.coef, A_LAT, species=c.species, occ=w)
    assert abs(loss.item() - L_ref) < 1e-4 * L_ref
    g = xyz.grad.cpu().numpy()
    assert rel_l2(g, g_ref) < TOL_GRAD
    sel = np.random.default_rng(0).choice(len(c.xyz), 12, replace=False)
    fd = oracle.fd_grad(c.xyz, S, I_obs, c.coef, A_LAT, sel, h=1e-5, species=c.species, occ=w)
    assert rel_l2(g[sel], fd) < TOL_GRAD


def test_vjp_through_autograd():
    """Any loss written in torch on A reaches the adjoint kernel through
    ScatterAmplitude.backward (scatter_vjp)."""
    c, axes, S, I_obs, _ = _case(seed=21)
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, path="generic")
    xyz = dev(c.xyz, grad=True)
    A = api.amplitude(xyz, plan)
    loss = ((A.abs() ** 2 - dev(I_obs, torch.float32)) ** 2).sum()
    loss.backward()
    L_ref, g_ref = oracle.loss_grad(c.xyz, S, I_obs, c.coef, A_LAT, species=c.species)
    assert abs(loss.item() - L_ref) < 1e-4 * L_ref
    assert rel_l2(xyz.grad.cpu().numpy(), g_ref) < TOL_GRAD


def test_list_sampling_gradient():
    rng = np.random.default_rng(5)
    c = W.fcc_sphere(radius_cells=3.0, seed=31)
    S = W.ewald_slice(3000, hkl=(1, 1, 1), seed=32)
    I_obs = rng.uniform(0, 1, len(S)).astype(np.float32) * float(len(c.xyz)) ** 2 * 1e-3
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), s_list=S, atom_species=c.species)
    xyz = dev(c.xyz, grad=True)
    loss = api.misfit(xyz, plan, dev(I_obs, torch.float32))
    loss.backward()
    L_ref, g_ref = oracle.loss_grad(c.xyz, S, I_obs, c.coef, A_LAT, species=c.species)
    assert abs(loss.item() - L_ref) < 1e-4 * L_ref
    assert rel_l2(xyz.grad.cpu().numpy(), g_ref) < TOL_GRAD


def test_strained_cube_all_atoms_subgrid():
    """All 102,400 atoms of the 40x40x16-cell strained cube, on a 16^3
    sub-grid of the 128^3 map (same 0.005 r.l.u. step)."""
    c = W.strained_cube()
    axes = [W.linspace_axis(0.0, 16, step=0.005), W.linspace_axis(0.0, 16, step=0.005),
            W.linspace_axis(4.0, 16, step=0.005)]
    S = W.grid_points(axes)
    pert = W.perturbed_copy(c)
    I_obs = (np.abs(oracle.amplitude(pert.xyz, S, c.coef, A_LAT)) ** 2).astype(np.float32)
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, path="generic")
    x = dev(c.xyz)
    A = plan.amplitude(x)
    loss, grad = plan.backward(x, A, dev(I_obs, torch.float32))
    plan.check()
    sel = np.random.default_rng(1).choice(len(c.xyz), 50, replace=False)
    L_ref, _ = oracle.loss_grad(c.xyz, S, I_obs, c.coef, A_LAT, grad=False)
    assert abs(loss.item() - L_ref) < 1e-4 * L_ref
    fd = oracle.fd_grad(c.xyz, S, I_obs, c.coef, A_LAT, sel, h=1e-5)
    assert rel_l2(grad.cpu().numpy()[sel], fd) < TOL_GRAD


def test_strained_cube_full_grid_properties():
    """Full size (102,400 atoms x 128^3 points): the gradient of a
    translation-invariant loss sums to zero over the atoms, and the loss
    equals sum (I - I_obs)^2 of the forward's own intensities."""
    c = W.strained_cube()
    axes = [W.linspace_axis(0.0, 128, step=0.005), W.linspace_axis(0.0, 128, step=0.005),
            W.linspace_axis(4.0, 128, step=0.005)]
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, path="generic")
    pert = W.perturbed_copy(c)
    I_obs = plan.intensity(dev(pert.xyz))
    x = dev(c.xyz)
    A = plan.amplitude(x)
    loss, grad = plan.backward(x, A, I_obs)
    plan.check()
    I = (A.abs().double() ** 2)
    L2 = ((I - I_obs.double()) ** 2).sum().item()
    assert abs(loss.item() - L2) < 1e-6 * L2
    g = grad.double()
    assert torch.all(torch.isfinite(g))
    assert (g.sum(0).abs().max() / g.abs().sum()).item() < 1e-4


@pytest.mark.parametrize("l_axis", ["long_uniform", "non_uniform"])
def test_gradient_line_recurrence_and_fallback(l_axis):
    """A uniform l axis longer than one 256-point tile runs the line kernel
    (phase carried along l by a complex multiply, re-seeded every 64 points,
    several tiles per line); a non-uniform l axis falls back to the table
    kernel.  Both against the oracle's analytic gradient."""
    c = W.fcc_sphere(radius_cells=2.6, seed=21)
    if l_axis == "long_uniform":
        l = W.linspace_axis(4.0, 300, step=0.004)
    else:
        t = np.linspace(-1.0, 1.0, 37)
        l = 4.0 + 0.3 * np.sign(t) * np.abs(t) ** 1.7
    axes = [W.linspace_axis(0.0, 3, step=0.02), W.linspace_axis(0.0, 2, step=0.02), l]
    S = W.grid_points(axes)
    pert = W.perturbed_copy(c, 0.03, seed=22)
    I_obs = (np.abs(oracle.amplitude(pert.xyz, S, c.coef, A_LAT, species=c.species)) ** 2).astype(np.float32)
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, path="generic")
    x = dev(c.xyz)
    A = plan.amplitude(x)
    loss, grad = plan.backward(x, A, dev(I_obs, torch.float32))
    plan.check()
    L_ref, g_ref = oracle.loss_grad(c.xyz, S, I_obs, c.coef, A_LAT, species=c.species)
    assert abs(loss.item() - L_ref) < 1e-4 * L_ref
    assert rel_l2(grad.cpu().numpy(), g_ref) < TOL_GRAD
