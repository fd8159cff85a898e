"""Sharding of the likelihood over ranks (one process per GPU).

The work splits into independent units -- parameter points, and systems --
so each rank evaluates a contiguous range of the points with no exchange
during the evaluation; the only collective is a host gather of the FP64
log-likelihood vector (8 bytes per point) when the caller wants all of it,
and a max-reduction of the step time for the benchmark.  Works with any
torch.distributed backend (NCCL between GPUs, gloo on the host).
"""
from __future__ import annotations

import numpy as np


def shard_range(n, rank, world):
    """Contiguous [start, end) of n units for this rank; sizes differ by at
    most one, lower ranks take the extra units."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"bad shard request n={n} rank={rank} world={world}")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def reduce_max(value, device="cpu"):
    """Max of a float over all ranks (the value itself without a process
    group).  device: where the reduction tensor lives ("cuda" for NCCL)."""
    dist = _dist()
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def loglike_sharded(evaluate, points, rank=None, world=None, gather=True):
    """Evaluate points [P, ...] split over ranks: this rank calls
    evaluate(points[start:end]) -> [end - start] log-likelihoods; with
    gather=True every rank receives the whole [P] vector in point order
    (one host all-gather), else only its own slice."""
    dist = _dist()
    if rank is None or world is None:
        rank, world = (dist.get_rank(), dist.get_world_size()) if dist else (0, 1)
    start, end = shard_range(len(points), rank, world)
    local = np.asarray(evaluate(points[start:end]), dtype=np.float64).reshape(-1)
    if len(local) != end - start:
        raise ValueError("evaluate returned the wrong number of values")
    if not gather or world == 1:
        return local
    parts = [None] * world
    dist.all_gather_object(parts, (rank, local))
    parts.sort(key=lambda x: x[0])
    return np.concatenate([p[1] for p in parts])
