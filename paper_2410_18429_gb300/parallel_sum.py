"""Sum of the per-rank gradients and objectives when sources are sharded across ranks.

The systems of different (source, frequency) pairs are independent; the one
exchange step of a sharded gradient evaluation is the sum of g and f over ranks.
"""
from __future__ import annotations


def allreduce_gradient(grads, f, group=None):
    """In-place all-reduce (sum) of the gradient tensors and the objective."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return grads, f
    for g in grads:
        dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(f, op=dist.ReduceOp.SUM, group=group)
    return grads, f


def shard(n_items: int, rank: int, world: int):
    """Contiguous [begin, end) share of n_items for this rank (sizes differ by at most one)."""
    q, r = divmod(n_items, world)
    b = rank * q + min(rank, r)
    return b, b + q + (1 if rank < r else 0)
