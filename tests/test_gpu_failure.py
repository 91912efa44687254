"""Failure detection on the GPU without a fault: a bounded wait on a flag that
nothing sets gives up, records TIMEOUT in the plan's status word, the host
reads it through scatter_check (which clears it), and the context stays
usable for the next call."""
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


def test_timed_out_wait_is_reported_and_cleared():
    c = W.fcc_sphere(radius_cells=2.5, seed=95)
    S = np.array([0.0, 0.0, 4.0]) + np.random.default_rng(96).uniform(-0.2, 0.2, (300, 3))
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), s_list=S, atom_species=c.species)
    plan.check()
    plan.selftest_wait()
    with pytest.raises(B.ScatterError) as e:
        plan.check()
    assert e.value.status == B.SCATTER_ERR_TIMEOUT
    plan.check()  # the word was cleared
    # the context is intact: the next call is correct
    A = plan.amplitude(torch.tensor(c.xyz, dtype=torch.float64, device="cuda:0"))
    plan.check()
    ref = oracle.amplitude(c.xyz, S, c.coef, A_LAT, species=c.species)
    assert rel_l2(A.cpu().numpy().astype(np.complex128), ref) < 1e-4


def test_timeout_and_numeric_bits_are_distinct():
    c = W.fcc_sphere(radius_cells=2.0, seed=97)
    S = np.array([0.0, 0.0, 4.0]) + np.random.default_rng(98).uniform(-0.2, 0.2, (64, 3))
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), s_list=S, atom_species=c.species)
    xyz = c.xyz.copy()
    xyz[3, 1] = np.nan
    plan.amplitude(torch.tensor(xyz, dtype=torch.float64, device="cuda:0"))
    with pytest.raises(B.ScatterError) as e:
        plan.check()
    assert e.value.status == B.SCATTER_ERR_NUMERIC
    plan.selftest_wait()
    with pytest.raises(B.ScatterError) as e:
        plan.check()
    assert e.value.status == B.SCATTER_ERR_TIMEOUT


def _small_plan():
    c = W.fcc_sphere(radius_cells=2.5, seed=99)
    axes = [W.linspace_axis(0.0, 9, step=0.01), W.linspace_axis(0.0, 7, step=0.01), W.linspace_axis(4.0, 5, step=0.01)]
    return c, axes, lambda: api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species,
                                     path="generic")


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_injected_allocation_failure_is_reported_and_leaks_nothing(monkeypatch, n):
    """SCATTER_FAULT=alloc:N fails the N-th device allocation of plan
    building (host side): scatter_plan returns OOM, frees what it had
    allocated, and a plan built afterwards works."""
    c, axes, make = _small_plan()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("SCATTER_FAULT", f"alloc:{n}")
    with pytest.raises(B.ScatterError) as e:
        make()
    assert e.value.status == B.SCATTER_ERR_OOM
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 4 << 20
    monkeypatch.delenv("SCATTER_FAULT")
    plan = make()
    A = plan.amplitude(torch.tensor(c.xyz, dtype=torch.float64, device="cuda:0"))
    plan.check()
    ref = oracle.amplitude(c.xyz, W.grid_points(axes), c.coef, A_LAT, species=c.species)
    assert rel_l2(A.cpu().numpy().astype(np.complex128).reshape(-1), ref) < 1e-4
