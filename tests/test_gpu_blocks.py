"""GPU parity of the block-of-atoms sum (Eq. 4: per-(type, S) structure
factors F_t(S), positions = displaced block origins) against the FP64 oracle,
through the C ABI, on every path that takes a factor table: the forward
(lists, grids, batches), and the misfit gradient with respect to the block
origins (F held fixed) on the FP32 S-tile, line and tensor-core adjoints.
Tolerances: relative L2 <= 1e-4 (FP32 paths), <= 1e-3 (split tensor-core
path, gradients), <= 1e-6 (FP64 kernel)."""
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


def block_table(model, S, coef):
    """F_t(S_m) = sum_a f_{s(a)}(|S_m|) e^{2 i pi S_m . rho_a} (FP64, oracle form factors)."""
    q = np.linalg.norm(S, axis=1) / A_LAT
    f = np.array([[oracle.form_factor(coef[s], qq) for qq in q] for s in range(coef.shape[0])])  # [species, M]
    tab = []
    for content, sp in zip(model.content, model.species):
        geo = np.exp(2j * np.pi * (S @ content.T))          # [M, atoms]
        tab.append(np.sum(f[sp].T * geo, axis=1))           # [M]
    return np.array(tab)


def run(plan, xyz, occ=None):
    x = torch.tensor(xyz, dtype=torch.float64, device="cuda:0")
    w = None if occ is None else torch.tensor(occ, dtype=torch.float32, device="cuda:0")
    A = plan.amplitude(x, w)
    plan.check()
    return A.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("path,apt,tol", [("generic", -1, 1e-4), ("generic", 4, 1e-4), ("fp64", 0, 1e-6)])
def test_block_list_vs_oracle(path, apt, tol):
    m = W.fcc_cell_blocks(n=(10, 9, 7))
    coef = W.si_ge_species()
    S = np.array([1.0, 1.0, 3.0]) + np.random.default_rng(61).uniform(-0.2, 0.2, (301, 3))
    T = block_table(m, S, coef)
    plan = api.Plan(coef, A_LAT, len(m.origins), s_list=S, atom_species=m.types, path=path, factor_table=T,
                    atoms_per_thread=apt)
    A = run(plan, m.origins)
    ref = oracle.amplitude_table(m.origins, S, T, types=m.types)
    assert rel_l2(A, ref) < tol


@pytest.mark.parametrize("path,tol", [("generic", 1e-4), ("separable", 1e-3), ("fp64", 1e-6)])
def test_block_grid_vs_oracle_and_atom_sum(path, tol):
    m = W.fcc_cell_blocks(n=(12, 12, 8))
    coef = W.si_ge_species()
    axes = [np.linspace(-0.06, 0.06, 9), np.linspace(-0.05, 0.05, 7), np.linspace(3.92, 4.08, 33)]
    S = W.grid_points(axes)
    T = block_table(m, S, coef)
    occ = np.random.default_rng(62).uniform(0.5, 1.0, len(m.origins)).astype(np.float32)
    plan = api.Plan(coef, A_LAT, len(m.origins), axes=axes, atom_species=m.types, path=path, factor_table=T)
    A = run(plan, m.origins, occ)
    ref = oracle.amplitude_table(m.origins, S, T, types=m.types, occ=occ)
    assert rel_l2(A, ref) < tol
    if path == "generic":
        # Eq. 4 with exact block factors is Eq. 2 over every atom of every block
        atoms = np.concatenate([o + m.content[t] for o, t in zip(m.origins, m.types)])
        species = np.concatenate([m.species[t] for t in m.types])
        w_atoms = np.repeat(occ, 4)
        plan_a = api.Plan(coef, A_LAT, len(atoms), axes=axes, atom_species=species, path="generic")
        assert rel_l2(run(plan_a, atoms, w_atoms), A) < 1e-4


def test_table_of_form_factors_matches_in_kernel_factors():
    c = W.fcc_sphere(radius_cells=5.5, seed=8)
    S = np.array([0.0, 0.0, 4.0]) + np.random.default_rng(63).uniform(-0.3, 0.3, (500, 3))
    q = np.linalg.norm(S, axis=1) / A_LAT
    T = np.array([[oracle.form_factor(c.coef[s], qq) for qq in q] for s in range(2)])
    with_table = api.Plan(c.coef, A_LAT, len(c.xyz), s_list=S, atom_species=c.species, factor_table=T)
    plain = api.Plan(c.coef, A_LAT, len(c.xyz), s_list=S, atom_species=c.species)
    a, b = run(with_table, c.xyz), run(plain, c.xyz)
    assert rel_l2(a, b) < 1e-5


@pytest.mark.parametrize("kind,path", [("list", "generic"), ("grid", "generic"), ("grid", "separable")])
def test_block_origin_gradient_vs_oracle(kind, path):
    """dL/d(block origin) of L = sum (|A|^2 - I_obs)^2 with the block factors
    held fixed: the S-tile adjoint (list), the line recurrence (uniform l
    axis) and the tensor-core contraction (separable plan)."""
    m = W.fcc_cell_blocks(n=(9, 8, 6))
    coef = W.si_ge_species()
    rng = np.random.default_rng(65)
    if kind == "list":
        S = np.array([1.0, 1.0, 3.0]) + rng.uniform(-0.15, 0.15, (400, 3))
        kw = dict(s_list=S)
    else:
        axes = [np.linspace(0.94, 1.06, 24), np.linspace(0.95, 1.05, 21), np.linspace(2.92, 3.08, 40)]
        S = W.grid_points(axes)
        kw = dict(axes=axes)
    T = block_table(m, S, coef)
    occ = rng.uniform(0.5, 1.0, len(m.origins)).astype(np.float32)
    pert = m.origins + rng.normal(0, 0.03, m.origins.shape)
    I_obs = (np.abs(oracle.amplitude_table(pert, S, T, types=m.types, occ=occ)) ** 2).astype(np.float32)
    plan = api.Plan(coef, A_LAT, len(m.origins), atom_species=m.types, path=path, factor_table=T, **kw)
    x = torch.tensor(m.origins, dtype=torch.float64, device="cuda:0")
    w = torch.tensor(occ, dtype=torch.float32, device="cuda:0")
    A = plan.amplitude(x, w)
    loss, grad = plan.backward(x, A, torch.tensor(I_obs, device="cuda:0"), w)
    plan.check()
    L_ref, g_ref = oracle.loss_grad_table(m.origins, S, I_obs, T, types=m.types, occ=occ)
    err = rel_l2(grad.cpu().numpy(), g_ref)
    print(f"block-origin gradient ({kind}, {path}, adjoint form {plan.info()['adjoint_form']}): rel L2 {err:.1e}")
    assert abs(loss.item() - L_ref) < 1e-3 * L_ref
    assert err < 1e-3


@pytest.mark.parametrize("path,tol", [("generic", 1e-4), ("fp64", 1e-6)])
def test_block_table_in_a_batch(path, tol):
    """Three block models of uneven size in one batched launch, each with its
    own S list; the table holds one factor per (type, point) of the batch."""
    coef = W.si_ge_species()
    rng = np.random.default_rng(66)
    models = [W.fcc_cell_blocks(n=n, seed=70 + i) for i, n in enumerate([(6, 5, 4), (11, 10, 7), (3, 3, 2)])]
    Ss = [np.array([1.0, 1.0, 3.0]) + rng.uniform(-0.2, 0.2, (k, 3)) for k in (350, 1100, 90)]
    xyz = np.concatenate([mm.origins for mm in models])
    types = np.concatenate([mm.types for mm in models])
    S = np.concatenate(Ss)
    T = np.concatenate([block_table(mm, s_b, coef) for mm, s_b in zip(models, Ss)], axis=1)
    ao = np.concatenate([[0], np.cumsum([len(mm.origins) for mm in models])]).astype(np.int64)
    so = np.concatenate([[0], np.cumsum([len(s_b) for s_b in Ss])]).astype(np.int64)
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=types, atom_off=ao, s_off=so, path=path,
                    factor_table=T)
    A = run(plan, xyz)
    for b, mm in enumerate(models):
        ref = oracle.amplitude_table(mm.origins, Ss[b], T[:, so[b]:so[b + 1]], types=mm.types)
        assert rel_l2(A[so[b]:so[b + 1]], ref) < tol, b


def test_table_rejected_on_grazing_incidence():
    m = W.fcc_cell_blocks(n=(4, 4, 4))
    coef = W.si_ge_species()
    gid = dict(wavelength=W.WAVELENGTH_10KEV, alpha_i=W.GID_ALPHA_I, delta=W.GID_DELTA, beta=W.GID_BETA)
    axes = [np.linspace(3.9, 4.0, 4), np.linspace(-0.02, 0.02, 5), np.deg2rad(np.linspace(0.1, 0.9, 1))]
    with pytest.raises(B.ScatterError):
        api.Plan(coef, A_LAT, len(m.origins), axes=axes, atom_species=m.types, gid=gid,
                 factor_table=np.ones((2, 20), complex))
