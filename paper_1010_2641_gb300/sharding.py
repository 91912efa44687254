"""Work distribution over several GPUs (one process per GPU).

The direct sum shards over reciprocal-space points with no exchange: each
rank evaluates Eq. 2 for its own block of S points (or whole instances of a
batch), which is how the paper spreads a computation over the GPUs of a
card (Section 3).  Only assembling the full map on one rank needs a
collective (a gather); the timing of a benchmark needs a max over ranks.

Works with any torch.distributed backend (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def shard_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous block of [0, n) owned by `rank`; block sizes differ by at most one."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def shard_points(S: np.ndarray, world: int, rank: int) -> np.ndarray:
    """This rank's rows of an [M, 3] list of S points."""
    a, b = shard_range(len(S), world, rank)
    return S[a:b]


def shard_instances(costs, world: int, rank: int) -> list[int]:
    """Instances of a batch owned by `rank`: longest-processing-time-first
    assignment of the per-instance costs (e.g. atoms x points) to ranks."""
    order = np.argsort(-np.asarray(costs, dtype=np.float64), kind="stable")
    load = np.zeros(world)
    owner = np.empty(len(order), dtype=np.int64)
    for i in order:
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += costs[i]
    return [int(i) for i in range(len(owner)) if owner[i] == rank]


def gather_map(local: torch.Tensor, n_total: int, group=None) -> torch.Tensor:
    """Concatenate every rank's block (in rank order) into the full map on all
    ranks.  Blocks follow shard_range(n_total, world, rank)."""
    world = dist.get_world_size(group)
    blocks = []
    for r in range(world):
        a, b = shard_range(n_total, world, r)
        blocks.append(torch.empty((b - a,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device))
    # pad to equal length for all_gather
    width = max(bl.shape[0] for bl in blocks)
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    out = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(out, pad, group=group)
    return torch.cat([out[r][: blocks[r].shape[0]] for r in range(world)])


def max_over_ranks(values, device=None, group=None) -> list[float]:
    """Element-wise maximum of a few floats over all ranks (step times)."""
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return t.tolist()
