"""GPU parity of the tensor-core adjoint (SEPARABLE grid plans: the per-atom
sums over S contracted on k_sep with the operands' roles swapped) against the
FP64 oracle's analytic gradient and central finite differences, through the
C ABI and torch.autograd.

Tolerances: loss relative error <= 1e-3 (the split path's amplitudes, FP64
reduction); gradients relative L2 <= 1e-3.
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
TOL_LOSS = 1e-3
TC_FORM = 3


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def dev(x, dtype=torch.float64, grad=False):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda:0", requires_grad=grad)


def _case(radius, axes, seed, n_species=2, occ=False, offset=(0.0, 0.0, 0.0)):
    c = W.fcc_sphere(radius_cells=radius, seed=seed)
    if n_species == 3:
        c.species = (np.arange(len(c.xyz)) % 3).astype(np.int32)
        c.coef = np.concatenate([c.coef, c.coef[:1] * 0.7])
    c.xyz = c.xyz + np.asarray(offset)
    S = W.grid_points(axes)
    pert = W.perturbed_copy(c, 0.03, seed=seed + 1)
    I_obs = (np.abs(oracle.amplitude(pert.xyz, S, c.coef, A_LAT, species=c.species)) ** 2).astype(np.float32)
    w = np.random.default_rng(seed).uniform(0.5, 1.0, len(c.xyz)).astype(np.float32) if occ else None
    return c, S, I_obs, w


def _axes(shape, step=0.02):
    return [W.linspace_axis(0.0, shape[0], step=step), W.linspace_axis(0.0, shape[1], step=step),
            W.linspace_axis(4.0, shape[2], step=step)]


# shapes: n1 n2 not a multiple of the 16-point step; 3 n0 rows filling one
# M tile, three (an odd count: the last pair holds one tile) and four
CASES = {
    "one_tile": dict(radius=3.2, axes=_axes((9, 7, 13)), seed=11),
    "odd_tiles_occ": dict(radius=3.2, axes=_axes((50, 6, 11)), seed=12, occ=True),
    "four_tiles_offset": dict(radius=2.6, axes=_axes((70, 5, 9)), seed=13, offset=(40.4, -7.7, 13.2)),
    "three_species": dict(radius=3.0, axes=_axes((12, 9, 10)), seed=14, n_species=3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_tc_gradient_vs_oracle(name):
    kw = CASES[name]
    axes = kw["axes"]
    c, S, I_obs, w = _case(**kw)
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, path="separable")
    xyz = dev(c.xyz, grad=True)
    loss = api.misfit(xyz, plan, dev(I_obs, torch.float32), None if w is None else dev(w, torch.float32))
    loss.backward()
    plan.check()
    assert plan.info()["adjoint_form"] == TC_FORM
    L_ref, g_ref = oracle.loss_grad(c.xyz, S, I_obs, c.coef, A_LAT, species=c.species, occ=w)
    assert abs(loss.item() - L_ref) < TOL_LOSS * L_ref
    g = xyz.grad.cpu().numpy()
    assert rel_l2(g, g_ref) < TOL_GRAD
    sel = np.random.default_rng(0).choice(len(c.xyz), 8, replace=False)
    fd = oracle.fd_grad(c.xyz, S, I_obs, c.coef, A_LAT, sel, h=1e-5, species=c.species, occ=w)
    assert rel_l2(g[sel], fd) < TOL_GRAD


def test_tc_vjp_through_autograd_non_uniform_axes():
    """A torch loss on A reaches the tensor-core adjoint through scatter_vjp;
    the separable form needs no uniform axis."""
    t, u = np.linspace(-1.0, 1.0, 21), np.linspace(-1.0, 1.0, 9)
    axes = [W.linspace_axis(0.0, 5, step=0.03), 0.05 * np.sign(u) * np.abs(u) ** 1.5,
            4.0 + 0.25 * np.sign(t) * np.abs(t) ** 1.7]
    c, S, I_obs, _ = _case(2.8, axes, seed=21)
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, path="separable")
    xyz = dev(c.xyz, grad=True)
    A = api.amplitude(xyz, plan)
    loss = ((A.abs() ** 2 - dev(I_obs, torch.float32)) ** 2).sum()
    loss.backward()
    plan.check()
    assert plan.info()["adjoint_form"] == TC_FORM
    L_ref, g_ref = oracle.loss_grad(c.xyz, S, I_obs, c.coef, A_LAT, species=c.species)
    assert abs(loss.item() - L_ref) < TOL_LOSS * L_ref
    assert rel_l2(xyz.grad.cpu().numpy(), g_ref) < TOL_GRAD


def test_tc_gradient_wide_dynamic_range():
    """G spans many decades (a Bragg peak inside the window and its far
    tails): the per-row power-of-two scaling keeps the gradient within
    tolerance of the oracle's."""
    c = W.fcc_sphere(radius_cells=4.0, seed=41)
    axes = [W.linspace_axis(0.0, 17, step=0.05), W.linspace_axis(0.0, 15, step=0.05),
            W.linspace_axis(4.0, 19, step=0.05)]
    S = W.grid_points(axes)
    I_obs = np.zeros(len(S), np.float32)  # L = sum I^2: g follows I conj(A), ~1e12 between peak and tails
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, path="separable")
    xyz = dev(c.xyz, grad=True)
    loss = api.misfit(xyz, plan, dev(I_obs, torch.float32))
    loss.backward()
    plan.check()
    L_ref, g_ref = oracle.loss_grad(c.xyz, S, I_obs, c.coef, A_LAT, species=c.species)
    assert abs(loss.item() - L_ref) < TOL_LOSS * L_ref
    assert rel_l2(xyz.grad.cpu().numpy(), g_ref) < TOL_GRAD


def test_tc_strained_cube_subgrid():
    """All 102,400 atoms of the strained cube (400 atom tiles) on a 16^3
    sub-grid of the 128^3 map: loss against the oracle, 50 sampled
    gradients against FP64 central differences."""
    c = W.strained_cube()
    axes = [W.linspace_axis(0.0, 16, step=0.005), W.linspace_axis(0.0, 16, step=0.005),
            W.linspace_axis(4.0, 16, step=0.005)]
    S = W.grid_points(axes)
    pert = W.perturbed_copy(c)
    I_obs = (np.abs(oracle.amplitude(pert.xyz, S, c.coef, A_LAT)) ** 2).astype(np.float32)
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, path="separable")
    x = dev(c.xyz)
    A = plan.amplitude(x)
    loss, grad = plan.backward(x, A, dev(I_obs, torch.float32))
    plan.check()
    assert plan.info()["adjoint_form"] == TC_FORM
    L_ref, _ = oracle.loss_grad(c.xyz, S, I_obs, c.coef, A_LAT, grad=False)
    assert abs(loss.item() - L_ref) < TOL_LOSS * L_ref
    sel = np.random.default_rng(1).choice(len(c.xyz), 50, replace=False)
    fd = oracle.fd_grad(c.xyz, S, I_obs, c.coef, A_LAT, sel, h=1e-5)
    assert rel_l2(grad.cpu().numpy()[sel], fd) < TOL_GRAD


def test_tc_strained_cube_full_grid_properties():
    """Full size (102,400 atoms x 128^3 points, the bench's launch): the
    gradient of a translation-invariant loss sums to zero over the atoms,
    and the loss equals sum (I - I_obs)^2 of the forward's own intensities."""
    c = W.strained_cube()
    axes = [W.linspace_axis(0.0, 128, step=0.005), W.linspace_axis(0.0, 128, step=0.005),
            W.linspace_axis(4.0, 128, step=0.005)]
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, path="separable")
    pert = W.perturbed_copy(c)
    I_obs = plan.intensity(dev(pert.xyz))
    x = dev(c.xyz)
    A = plan.amplitude(x)
    loss, grad = plan.backward(x, A, I_obs)
    plan.check()
    assert plan.info()["adjoint_form"] == TC_FORM
    I = (A.abs().double() ** 2)
    L2 = ((I - I_obs.double()) ** 2).sum().item()
    assert abs(loss.item() - L2) < 1e-6 * L2
    g = grad.double()
    assert torch.all(torch.isfinite(g))
    assert (g.sum(0).abs().max() / g.abs().sum()).item() < 1e-4


def test_generic_plan_keeps_fp32_adjoint():
    c, S, I_obs, _ = _case(2.5, _axes((5, 4, 6)), seed=51)
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=_axes((5, 4, 6)), atom_species=c.species, path="generic")
    assert plan.info()["adjoint_form"] == 0
    x = dev(c.xyz)
    A = plan.amplitude(x)
    plan.backward(x, A, dev(I_obs, torch.float32))
    plan.check()
    assert plan.info()["adjoint_form"] == 2
