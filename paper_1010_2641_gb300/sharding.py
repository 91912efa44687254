"""Work distribution over several GPUs (one process per GPU).

The direct sum shards over reciprocal-space points with no exchange: each
rank evaluates Eq. 2 for its own block of S points (or whole instances of a
batch), which is how the paper spreads a computation over the GPUs of a
card (Section 3).  Only assembling the full map on one rank needs a
collective (a gather); the timing of a benchmark needs a max over ranks.

For one huge crystal and a map that one GPU holds, the sum shards over the
atoms instead: every rank sums its block of atoms into a partial map, and
one all-reduce (sum) of the n_s complex values gives A on every rank
(Eq. 2 is linear in the atoms).  The misfit gradient then needs no further
exchange: with the full A, each rank's dL/dr_j of its own atoms is
independent (g(S) depends on A only); a gather assembles them if one rank
wants all.  AtomShardedPlan and PointShardedPlan wrap a per-rank plan of the
library with these exchanges.

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


def allreduce_amplitude(partial: torch.Tensor, group=None) -> torch.Tensor:
    """The sum over ranks of every rank's partial map (complex64 [M], or
    float [M, 2] as (Re, Im)), returned on every rank in the input's form.
    One all-reduce of 2 M floats; without a process group (or with one rank)
    the partial is the map."""
    buf = torch.view_as_real(partial).clone() if partial.is_complex() else partial.clone()
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return torch.view_as_complex(buf) if partial.is_complex() else buf


def gather_atom_rows(local: torch.Tensor, n_atoms: int, group=None) -> torch.Tensor:
    """Every rank's rows of a per-atom array (gradients [n_local, 3]) in atom
    order, on every rank; rank blocks follow shard_range(n_atoms, ...)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return local
    return gather_map(local, n_atoms, group)


class AtomShardedPlan:
    """This rank's share of a plan sharded over atoms.

    The rank owns atoms [lo, hi) = shard_range(n_atoms, world, rank) and plans
    them with the library (every other argument as for api.Plan: the same S
    sampling on every rank, so every rank picks the same reference
    reflection; each rank centres its own atoms).  amplitude() returns the
    full A on every rank (one all-reduce); backward() returns the misfit L
    (the same on every rank) and dL/dr of this rank's atoms, computed from
    the full A with no further exchange."""

    def __init__(self, coef, lattice_a: float, n_atoms: int, *, world: int, rank: int, atom_species=None,
                 group=None, **plan_kw):
        from . import api  # the GPU library (only constructed on a GPU rank)
        self.lo, self.hi = shard_range(int(n_atoms), world, rank)
        self.n_atoms = int(n_atoms)
        self.group = group
        sp = None if atom_species is None else np.asarray(atom_species)[self.lo:self.hi]
        self.plan = api.Plan(coef, lattice_a, self.hi - self.lo, atom_species=sp, **plan_kw)

    def local_slice(self, a):
        """This rank's rows of a per-atom array of all atoms."""
        return a[self.lo:self.hi]

    def partial_amplitude(self, xyz_local: torch.Tensor, occ_local=None) -> torch.Tensor:
        """Eq. 2 summed over this rank's atoms only (complex64 [n_s])."""
        return self.plan.amplitude(xyz_local, occ_local)

    def amplitude(self, xyz_local: torch.Tensor, occ_local=None) -> torch.Tensor:
        return allreduce_amplitude(self.partial_amplitude(xyz_local, occ_local), self.group)

    def backward(self, xyz_local: torch.Tensor, A: torch.Tensor, I_obs: torch.Tensor, occ_local=None):
        """(L, dL/dr of this rank's atoms) for L = sum (|A|^2 - I_obs)^2, A the
        full map from amplitude()."""
        return self.plan.backward(xyz_local, A, I_obs, occ_local)


class PointShardedPlan:
    """This rank's share of an S-point list, planned with the library: every
    rank sums all atoms for its block of points; gather() assembles the map."""

    def __init__(self, coef, lattice_a: float, n_atoms: int, S, *, world: int, rank: int, group=None,
                 **plan_kw):
        from . import api
        self.n_s = len(S)
        self.group = group
        self.lo, self.hi = shard_range(self.n_s, world, rank)
        self.plan = api.Plan(coef, lattice_a, n_atoms, s_list=np.asarray(S)[self.lo:self.hi], **plan_kw)

    def amplitude(self, xyz: torch.Tensor, occ=None) -> torch.Tensor:
        """This rank's block of the map (complex64 [hi - lo])."""
        return self.plan.amplitude(xyz, occ)

    def gather(self, local: torch.Tensor) -> torch.Tensor:
        full = gather_map(torch.view_as_real(local).contiguous(), self.n_s, self.group)
        return torch.view_as_complex(full.contiguous())


def max_over_ranks(values, device=None, group=None) -> list[float]:
    """Element-wise maximum of a few floats over all ranks (step times)."""
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return t.tolist()
