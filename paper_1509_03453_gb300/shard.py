"""Search sharded by data rows across ranks of a torch.distributed group.

Each rank indexes a contiguous block of rows [lo, hi) of the dataset.  A
cone key depends only on its row, so every shard holds exactly its rows of
every cone, and a query (whose probe list depends only on the query) visits
the same cones on every shard: the shards' candidate sets partition the
unsharded one.  One exchange step -- an all-gather of each rank's Q x k
(distance, id) lists -- and a k-way merge by (distance, id) then give the
unsharded answer, bit for bit.  On one GPU per process the merge is the
library's CUDA kernel (osann_merge_topk).
"""
from __future__ import annotations


def shard_rows(N: int, rank: int, world: int):
    """Contiguous block of rows [lo, hi) of rank `rank` out of `world`."""
    if world < 1 or not 0 <= rank < world or N < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(N, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def to_global(ids, lo: int):
    """Local shard ids -> global row ids (padding -1 kept)."""
    import torch
    return torch.where(ids >= 0, ids + lo, ids)


def gather_lists(ids, d2, group=None):
    """All-gather every rank's [Q, k] lists into [world, Q, k] tensors."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    gi = [torch.empty_like(ids) for _ in range(world)]
    gd = [torch.empty_like(d2) for _ in range(world)]
    dist.all_gather(gi, ids.contiguous(), group=group)
    dist.all_gather(gd, d2.contiguous(), group=group)
    return torch.stack(gi), torch.stack(gd)


class ShardedIndex:
    """One rank's shard.  ``X_local`` holds rows [lo, lo + len) of the whole
    dataset.  ``index_factory(X, L)`` builds the local index (default: the
    library's Index on the tensor's device) and must offer
    ``search(Y, P, k) -> (ids, sqdists)``; ``merge(ids[G,Q,k], d2[G,Q,k])``
    combines the gathered lists (default: the library's CUDA merge)."""

    def __init__(self, X_local, L: int, lo: int, group=None, index_factory=None, merge=None):
        if index_factory is None:
            from . import Index
            index_factory = Index
        if merge is None:
            from . import merge_topk
            merge = merge_topk
        self.lo = int(lo)
        self.group = group
        self.index = index_factory(X_local, L)
        self.merge = merge

    def search(self, Y, P: int, k: int):
        ids, d2 = self.index.search(Y, P, k)
        gi, gd = gather_lists(to_global(ids, self.lo), d2, self.group)
        return self.merge(gi, gd)
