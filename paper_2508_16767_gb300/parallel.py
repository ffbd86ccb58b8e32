"""Walk-range sharding across ranks and the merge of raw moments.

The estimator partitions by walks: rank r of R runs the walks
[walk_begin + r W / R, walk_begin + (r+1) W / R) of every point (ranges aligned
to the schedule group) with `woi_estimate_range`, and the raw moments
(sum of f, sum of squared schedule-group means) of disjoint ranges add up.
The merge is the only exchange step; it is one all-reduce (SUM) of
[P, 2, dim+1] doubles, or a host-side sum for replicas that never talk.
"""
from __future__ import annotations

import numpy as np


def shard_walk_range(rank: int, world: int, n_walks: int, sched_group: int = 1, walk_begin: int = 0):
    """(begin, count) of this rank's share; shares differ by at most one group."""
    if n_walks % sched_group:
        raise ValueError("n_walks must be a multiple of sched_group")
    groups = n_walks // sched_group
    lo = groups * rank // world
    hi = groups * (rank + 1) // world
    return walk_begin + lo * sched_group, (hi - lo) * sched_group


def merge_moments(moments_list):
    """Sum of raw moment arrays of disjoint walk ranges (host)."""
    out = np.zeros_like(np.asarray(moments_list[0], dtype=np.float64))
    for m in moments_list:
        out += np.asarray(m, dtype=np.float64)
    return out


def allreduce_moments(moments, group=None):
    """All-reduce (SUM) of a [P, 2, dim+1] moment array over a torch.distributed
    group (gloo on CPU tensors, NCCL on CUDA tensors); returns the merged array
    in the input's type."""
    import torch
    import torch.distributed as dist
    t = moments if isinstance(moments, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(moments))
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t if isinstance(moments, torch.Tensor) else t.numpy()


def finalize(moments, n_walks, sched_group=1, stream=None):
    """Mean and SE of merged moments [P, 2, dim+1] (host or device) by the library's
    finalize kernel (woi_finalize_moments)."""
    from . import woi
    return woi.woi_finalize_moments(moments, n_walks, sched_group, stream=stream)
