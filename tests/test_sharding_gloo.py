"""Multi-rank logic on CPU: world-size-2 gloo process groups.

S-point sharding: each rank evaluates Eq. 2 (FP64 oracle, CPU) for its
shard of the S points; the gathered map must equal the single-process map
exactly, and the timing reduction must return the maximum over ranks.

Atom sharding: the per-rank partial maps (Eq. 2 over each rank's atoms) and
the per-rank gradient rows are the values each rank's GPU plan would hand
the exchange; here they are computed once by the oracle in the parent, and
the ranks run the library's own exchange code on them (the all-reduce of the
partial maps, the gather of the gradient rows).  The result must equal the
oracle's single-process map and gradient.  No GPU involved.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1010_2641_gb300 import sharding
from paper_1010_2641_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = W.fcc_sphere(radius_cells=2.5, seed=3)
        S = W.ewald_slice(101, seed=4)
        mine = sharding.shard_points(S, world, rank)
        A = oracle.amplitude(c.xyz, mine, c.coef, W.LATTICE_A, species=c.species)
        local = torch.tensor(np.stack([A.real, A.imag], 1))
        full = sharding.gather_map(local, len(S))
        t = sharding.max_over_ranks([1.0 + rank, 5.0 - rank])
        q.put((rank, full.numpy(), t))
    finally:
        dist.destroy_process_group()


def _atom_worker(rank, world, port, partials, grads, n_atoms, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A = sharding.allreduce_amplitude(torch.tensor(partials[rank]))
        g = sharding.gather_atom_rows(torch.tensor(grads[rank]), n_atoms)
        q.put((rank, A.numpy(), g.numpy()))
    finally:
        dist.destroy_process_group()


def _run_atom_sharding(c, S, I_obs, world=2):
    import oracle
    n = len(c.xyz)
    A_full = oracle.amplitude(c.xyz, S, c.coef, W.LATTICE_A, species=c.species)
    partials, grads = [], []
    for r in range(world):
        lo, hi = sharding.shard_range(n, world, r)
        partials.append(oracle.amplitude(c.xyz[lo:hi], S, c.coef, W.LATTICE_A, species=c.species[lo:hi]))
        # what rank r's plan.backward returns: its atoms' rows, from the full map
        grads.append(oracle.loss_grad_atoms(c.xyz, S, A_full, I_obs, c.coef, W.LATTICE_A, np.arange(lo, hi),
                                            species=c.species)[1])
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_atom_worker, args=(r, world, port, partials, grads, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return A_full, results


def test_two_rank_atom_sharding_sums_the_partial_maps():
    """Eq. 2 is linear in the atoms: the all-reduce of the two ranks' partial
    maps is the map of all atoms on both ranks, and the gathered gradient rows
    (each rank's atoms, from that full map) are the full misfit gradient."""
    import oracle
    oracle.build()
    c = W.fcc_sphere(radius_cells=2.7, seed=13)
    S = W.ewald_slice(120, seed=14)
    pert = W.perturbed_copy(c, 0.03, seed=15)
    I_obs = np.abs(oracle.amplitude(pert.xyz, S, c.coef, W.LATTICE_A, species=c.species)) ** 2
    A_full, results = _run_atom_sharding(c, S, I_obs)
    L_ref, g_ref = oracle.loss_grad(c.xyz, S, I_obs, c.coef, W.LATTICE_A, species=c.species)
    for rank, A, g in results:
        assert np.max(np.abs(A - A_full)) <= 1e-12 * np.max(np.abs(A_full))
        assert abs(np.sum((np.abs(A) ** 2 - I_obs) ** 2) - L_ref) <= 1e-10 * L_ref
        assert g.shape == g_ref.shape
        assert np.max(np.abs(g - g_ref)) <= 1e-10 * np.max(np.abs(g_ref))


def test_atom_sharding_with_an_empty_rank():
    """One atom on two ranks: rank 1 owns none and contributes a zero map."""
    import oracle
    c = W.Crystal(xyz=np.array([[0.3, -1.2, 2.1]]), species=np.zeros(1, np.int32), coef=W.si_ge_species()[:1])
    assert sharding.shard_range(1, 2, 1) == (1, 1)
    S = W.ewald_slice(17, seed=16)
    A_full, results = _run_atom_sharding(c, S, np.ones(len(S)))
    for rank, A, g in results:
        assert np.max(np.abs(A - A_full)) <= 1e-12 * np.max(np.abs(A_full))
        assert g.shape == (1, 3)


def test_shard_range_partitions():
    for n in (0, 1, 7, 100, 101):
        for world in (1, 2, 3, 8):
            parts = [sharding.shard_range(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1


def test_shard_instances_balances():
    costs = [100, 1, 50, 50, 3, 99]
    owned = [sharding.shard_instances(costs, 2, r) for r in range(2)]
    assert sorted(owned[0] + owned[1]) == list(range(6))
    loads = [sum(costs[i] for i in o) for o in owned]
    assert abs(loads[0] - loads[1]) <= 5


def test_two_rank_gather_equals_single_process():
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    c = W.fcc_sphere(radius_cells=2.5, seed=3)
    S = W.ewald_slice(101, seed=4)
    A = oracle.amplitude(c.xyz, S, c.coef, W.LATTICE_A, species=c.species)
    ref = np.stack([A.real, A.imag], 1)
    for rank, full, t in results:
        assert np.array_equal(full, ref)
        assert t == [2.0, 5.0]
