"""Data-parallel sharding of a multi-pose batch over ranks.

Poses are independent in the forward, so a batch splits across GPUs with no
exchange; the backward has one exchange step when the ranks render poses of
one shared volume: the sum of their volume gradients (pose gradients stay
local to the rank that owns the pose).  One process drives one GPU; the
helpers below take a torch.distributed process group (NCCL on GPUs, gloo on
CPU).
"""
from __future__ import annotations

import numpy as np


def shard_ranges(work, world: int):
    """Contiguous split of poses 0..P-1 over `world` ranks, balanced by work
    (ray-samples per pose): rank r owns [start_r, end_r), the cut placed where
    the running work sum is closest to r/world of the total.  Contiguous
    ranges keep each pose's global index as its speckle counter (a rank's
    batch is built with pose counter start_r), so every rank renders exactly
    the images of the unsharded batch.  Returns a list of (start, end)."""
    work = np.asarray(work, dtype=np.int64)
    P = work.size
    if world < 1:
        raise ValueError("world must be >= 1")
    csum = np.concatenate([[0], np.cumsum(work)])
    total = int(csum[-1])
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        i = int(np.searchsorted(csum, target))
        # the boundary nearest the target, never before the previous cut
        if i > 0 and (i > P or abs(csum[i - 1] - target) <= abs(csum[i] - target)):
            i -= 1
        cuts.append(min(max(i, cuts[-1]), P))
    cuts.append(P)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def allreduce_volume_grad(grad_vol, group=None):
    """Sum the per-rank volume gradients in place (the only exchange step of
    a data-parallel forward+backward over one shared volume)."""
    import torch.distributed as dist
    dist.all_reduce(grad_vol, op=dist.ReduceOp.SUM, group=group)
    return grad_vol


def job_rate(units_local: int, ms_local: float, group=None):
    """Whole-job throughput of one timed region: all ranks' units over the
    slowest rank's time."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], dtype=torch.float64)
    u = torch.tensor([float(units_local)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(u.item()) / (float(t.item()) * 1e-3), float(t.item())
