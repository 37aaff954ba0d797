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


def shard_poses(work, world: int):
    """Deterministic split of poses over `world` ranks, balanced by work
    (ray-samples per pose): longest-processing-time-first greedy, ties by
    pose index.  Returns one sorted index list per rank."""
    work = np.asarray(work, dtype=np.int64)
    order = np.lexsort((np.arange(work.size), -work))
    load = np.zeros(world, dtype=np.int64)
    owned = [[] for _ in range(world)]
    for p in order:
        r = int(np.lexsort((np.arange(world), load))[0])   # least loaded, lowest rank on ties
        owned[r].append(int(p))
        load[r] += work[p]
    return [sorted(o) for o in owned]


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
