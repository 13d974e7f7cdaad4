"""Sharding checks over ranks (one process per GPU).

Two forms, both with no exchange on the data path:

* A batch of protocols: Definition 1 makes protocols independent of each
  other; each rank checks a contiguous slice of the protocols and the
  per-protocol results are gathered back in order.
* One protocol: Definition 1 decides each (phase, array, index) cell on its
  own, so the cells shard -- each rank checks the window of cell positions
  the library assigns it (drf_shard_range / drf_check_shard) -- and the
  ranks' result records (a few dozen bytes each) are gathered and merged by
  a lexicographic minimum over the racy cells, after checking that every
  rank saw the same facts of the whole protocol (drf_merge_shards).

The only collective in either form is that final gather of small records.
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


def check_protocol_sharded(rank: int, world: int, check_shard, group=None):
    """One protocol split by cells over `world` ranks: check_shard(rank,
    world) returns this rank's shard result (a drf_result); the ranks'
    records are all-gathered and merged into the protocol's result."""
    from . import drf

    mine = bytes(check_shard(rank, world))
    if world == 1:
        parts = [mine]
    else:
        import torch.distributed as dist
        got = [None] * world
        dist.all_gather_object(got, (rank, mine), group=group)
        parts = [b for _, b in sorted(got, key=lambda x: x[0])]
    return drf.drf_merge_shards([drf.drf_result.from_buffer_copy(b) for b in parts])


def gpu_shard_checker(ctx, bytecode: bytes, nthreads: int, cells, params, stream=None):
    """check_shard for check_protocol_sharded on this rank's GPU."""
    from . import drf

    def check_shard(rank, world):
        return drf.drf_check_shard(ctx, bytecode, nthreads, cells, params, rank, world, stream)
    return check_shard
