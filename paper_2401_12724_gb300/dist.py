"""Sharding of hit records over ranks (one process per GPU).

Records are independent, so the forward pass shards with no collective: each
rank evaluates a contiguous range of the record set.  The only exchange is in
the backward pass: the per-material parameter gradients ([n_mat, 8] floats)
of the ranks are summed with one all-reduce.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous, balanced record range [begin, end) of `rank`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def shard_segments(seg_offsets: np.ndarray, begin: int, end: int) -> np.ndarray:
    """Material segment offsets of the records [begin, end) of a
    material-sorted set, rebased to the shard (materials keep their ids)."""
    seg = np.asarray(seg_offsets, np.int64)
    return (np.clip(seg, begin, end) - begin).astype(np.int64)


def allreduce_param_grads(grad, group=None):
    """Sum the [n_mat, 8] gradient tensor over ranks (in place)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    return grad
