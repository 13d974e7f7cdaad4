"""Sharding a batch of protocols over ranks (one process per GPU).

Definition 1 makes protocols independent of each other, so a batch shards
with no exchange on the data path: each rank checks a contiguous slice of
the protocols and the per-protocol results are gathered back in order.  The
only collective is that final gather of small result records.
"""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int):
    """[lo, hi) of the n items that `rank` of `world` checks: contiguous,
    sizes differing by at most one, lower ranks take the larger ones."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def check_sharded(items, rank: int, world: int, check_slice, group=None):
    """Runs check_slice(items[lo:hi]) on this rank's slice and returns every
    rank's results concatenated in item order (an all-gather of objects)."""
    import torch.distributed as dist

    lo, hi = shard_range(len(items), rank, world)
    mine = list(check_slice(items[lo:hi]))
    if len(mine) != hi - lo:
        raise RuntimeError("check_slice returned the wrong number of results")
    if world == 1:
        return mine
    parts = [None] * world
    dist.all_gather_object(parts, (rank, mine), group=group)
    out = []
    for r, res in sorted(parts, key=lambda p: p[0]):
        out.extend(res)
    return out
