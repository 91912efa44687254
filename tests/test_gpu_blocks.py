"""GPU parity of the block-of-atoms sum (Eq. 4: per-(type, S) structure
factors F_t(S), positions = displaced block origins) against the FP64 oracle,
through the C ABI, on every forward path that takes a factor table.
Tolerances: relative L2 <= 1e-4 (FP32 paths), <= 1e-3 (split tensor-core
path), <= 1e-6 (FP64 kernel)."""
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


def test_table_rejected_where_unsupported():
    m = W.fcc_cell_blocks(n=(4, 4, 4))
    coef = W.si_ge_species()
    S = np.array([1.0, 1.0, 3.0]) + np.random.default_rng(64).uniform(-0.2, 0.2, (20, 3))
    T = block_table(m, S, coef)
    plan = api.Plan(coef, A_LAT, len(m.origins), s_list=S, atom_species=m.types, factor_table=T)
    x = torch.tensor(m.origins, dtype=torch.float64, device="cuda:0")
    A = plan.amplitude(x)
    with pytest.raises(B.ScatterError):
        plan.backward(x, A, torch.ones(len(S), dtype=torch.float32, device="cuda:0"))
    gid = dict(wavelength=W.WAVELENGTH_10KEV, alpha_i=W.GID_ALPHA_I, delta=W.GID_DELTA, beta=W.GID_BETA)
    axes = [np.linspace(3.9, 4.0, 4), np.linspace(-0.02, 0.02, 5), np.deg2rad(np.linspace(0.1, 0.9, 1))]
    with pytest.raises(B.ScatterError):
        api.Plan(coef, A_LAT, len(m.origins), axes=axes, atom_species=m.types, gid=gid,
                 factor_table=np.ones((2, 20), complex))
    with pytest.raises(B.ScatterError):
        api.Plan(coef, A_LAT, len(m.origins), s_list=S, atom_species=m.types, factor_table=T,
                 atom_off=[0, 30, len(m.origins)], s_off=[0, 10, 20])
