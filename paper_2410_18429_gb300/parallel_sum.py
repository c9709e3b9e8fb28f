"""Sum of the per-rank gradients and objectives when sources are sharded across ranks.

The systems of different (source, frequency) pairs are independent; the one
exchange step of a sharded gradient evaluation is the sum of g and f over ranks.
"""
from __future__ import annotations


def allreduce_gradient(grads, f, group=None):
    """In-place all-reduce (sum) of the gradient tensors and the objective.

    All of them (float64, one device) travel in one flat buffer, so the exchange is a single
    collective however many frequency groups there are."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return grads, f
    parts = list(grads) + [f]
    flat = torch.cat([t.reshape(-1) for t in parts])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for t in parts:
        k = t.numel()
        t.copy_(flat[off:off + k].view_as(t))
        off += k
    return grads, f


def shard(n_items: int, rank: int, world: int):
    """Contiguous [begin, end) share of n_items for this rank (sizes differ by at most one)."""
    q, r = divmod(n_items, world)
    b = rank * q + min(rank, r)
    return b, b + q + (1 if rank < r else 0)
