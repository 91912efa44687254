"""The sharded plans of the library on one GPU, without a process group.

Two AtomShardedPlans (ranks 0 and 1 of two) each sum their half of the atoms
through the library; the sum of their partial maps is the map of all atoms,
and the gradients they return from that full map are the full plan's
gradient rows.  Two PointShardedPlans cover a list in two blocks.  All against
the FP64 oracle.  (The exchanges themselves, all-reduce and gathers, run in
the world-size-2 gloo tests.)
"""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle
from closed_forms import rel_l2
from paper_1010_2641_gb300 import api, sharding
from paper_1010_2641_gb300 import workloads as W

pytestmark = pytest.mark.gpu
A_LAT = W.LATTICE_A


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


@pytest.mark.parametrize("kind", ["list", "grid"])
def test_atom_sharded_halves_sum_to_the_full_map_and_gradient(kind):
    c = W.fcc_sphere(radius_cells=4.2, seed=51)
    if kind == "list":
        S = W.ewald_slice(900, seed=52)
        kw = dict(s_list=S)
    else:
        axes = [W.linspace_axis(0.0, 12, step=0.01), W.linspace_axis(0.0, 10, step=0.01),
                W.linspace_axis(4.0, 9, step=0.01)]
        S = W.grid_points(axes)
        kw = dict(axes=axes, path="generic")
    pert = W.perturbed_copy(c, 0.03, seed=53)
    I_obs = (np.abs(oracle.amplitude(pert.xyz, S, c.coef, A_LAT, species=c.species)) ** 2).astype(np.float32)
    n = len(c.xyz)
    parts = [sharding.AtomShardedPlan(c.coef, A_LAT, n, world=2, rank=r, atom_species=c.species, **kw)
             for r in range(2)]
    T = [p.partial_amplitude(_dev(p.local_slice(c.xyz))) for p in parts]
    A = T[0] + T[1]  # what the all-reduce returns on every rank
    ref = oracle.amplitude(c.xyz, S, c.coef, A_LAT, species=c.species)
    assert rel_l2(A.cpu().numpy().astype(np.complex128), ref) < 1e-4
    losses, grads = [], []
    for p in parts:
        loss, g = p.backward(_dev(p.local_slice(c.xyz)), A, _dev(I_obs, torch.float32))
        losses.append(loss.item())
        grads.append(g.cpu().numpy().astype(np.float64))
    assert abs(losses[0] - losses[1]) <= 1e-12 * abs(losses[0])
    L_ref, g_ref = oracle.loss_grad(c.xyz, S, I_obs, c.coef, A_LAT, species=c.species)
    assert abs(losses[0] - L_ref) < 1e-3 * L_ref
    assert rel_l2(np.concatenate(grads), g_ref) < 1e-3


def test_point_sharded_blocks_cover_the_list():
    c = W.fcc_sphere(radius_cells=3.5, seed=54)
    S = W.ewald_slice(1001, seed=55)
    x = _dev(c.xyz)
    blocks = [sharding.PointShardedPlan(c.coef, A_LAT, len(c.xyz), S, world=2, rank=r, atom_species=c.species)
              for r in range(2)]
    got = np.concatenate([b.amplitude(x).cpu().numpy() for b in blocks]).astype(np.complex128)
    assert got.shape == (len(S),)
    assert rel_l2(got, oracle.amplitude(c.xyz, S, c.coef, A_LAT, species=c.species)) < 1e-4
