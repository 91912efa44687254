"""Multi-rank logic on CPU: world-size-2 gloo process groups.

Each rank evaluates Eq. 2 (FP64 oracle, CPU) for its shard of the S points;
the gathered map must equal the single-process map exactly, and the timing
reduction must return the maximum over ranks.  No GPU involved.
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
