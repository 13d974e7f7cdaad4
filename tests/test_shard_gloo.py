"""Sharded checking over two CPU ranks (gloo), no GPU needed.

Batches: each rank checks its slice of a batch, the gathered results equal
the unsharded ones in order (the checker is the oracle; on GPUs each rank
would call drf_check_batch on its slice).

One protocol split by cells: the library's shard windows (drf_shard_range)
and merge (drf_merge_shards) with the all-gather of shard.py, the device
part of each shard stood in for by the oracle's accesses restricted to the
rank's window; the merged result equals the oracle's for the whole
protocol, on every field."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2203_12878_b300.shard import shard_range


def test_shard_range_covers_everything_once():
    for n in (0, 1, 5, 96, 4097):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = shard_range(n, r, world)
                seen.extend(range(lo, hi))
                assert 0 <= hi - lo <= n // world + 1
            assert seen == list(range(n))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, count, out_path):
    import torch.distributed as dist
    from oracle import oracle
    from paper_2203_12878_b300 import protogen
    from paper_2203_12878_b300.shard import check_sharded

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ps = protogen.config4(master_seed=4, count=count)

    def check_slice(items):
        return [oracle.check(p.text, p.nthreads, p.cells, p.params, 1) for p in items]

    res = check_sharded(ps, rank, world, check_slice)
    if rank == 0:
        import json
        with open(out_path, "w") as f:
            json.dump(res, f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_gloo_sharded_batch_equals_unsharded(tmp_path, oracle, world):
    import json
    from paper_2203_12878_b300 import protogen

    count = 37
    out = str(tmp_path / "res.json")
    mp.start_processes(_worker, args=(world, _free_port(), count, out), nprocs=world, start_method="spawn")
    got = json.load(open(out))
    ps = protogen.config4(master_seed=4, count=count)
    want = [oracle.check(p.text, p.nthreads, p.cells, p.params, 1) for p in ps]
    assert got == want


_STATUS_CODE = {"OK": 0, "INDEX_OOB": -9, "DIV_ZERO": -10}
_VERDICT_CODE = {"DRF": 0, "RACY": 1, "BARRIER_DIVERGENCE": 2}


def fake_shard_result(p, rank, world):
    """What a GPU's drf_check_shard reports for shard `rank` of `world`,
    from the oracle: the whole protocol's facts, and the first racy cell
    among the accesses whose cell position falls in the shard's window
    (positions and window from the library)."""
    from oracle import oracle
    from paper_2203_12878_b300 import drf

    bc = drf.drf_protocol_compile(p.text)
    lo, hi, _ = drf.drf_shard_range(bc, p.nthreads, p.cells, p.params, rank, world)
    whole = oracle.check(p.text, p.nthreads, p.cells, p.params, 1)
    r = drf.drf_result()
    r.status = _STATUS_CODE[whole["status"]]
    r.tuples = whole.get("tuples", 0)
    if r.status:
        r.verdict = -1
        r.err_tid, r.err_ordinal = whole["err_tid"], whole["err_ordinal"]
        return r
    r.phases = whole["phases"]
    r.verdict = _VERDICT_CODE[whole["verdict"]]
    if whole["verdict"] == "BARRIER_DIVERGENCE":
        r.div_tid, r.sync_count_0, r.sync_count_div = whole["div_tid"], whole["sync_count_0"], whole["sync_count_div"]
        return r
    r.sync_count_0 = whole["phases"] - 1
    base = [sum(p.cells[:l]) for l in range(len(p.cells))]
    row = sum(p.cells)
    acc = {}
    for ph, loc, idx, tid, w in oracle.tuples(p.text, p.nthreads, p.cells, p.params).tolist():
        pos = ph * row + base[loc] + idx
        if lo <= pos < hi:
            a = acc.setdefault((ph, loc, idx), [set(), set()])
            a[0].add(tid)
            if w:
                a[1].add(tid)
    r.verdict = 0
    for cell in sorted(acc):
        ts, ws = acc[cell]
        if ws and len(ts) >= 2:
            t = sorted(ts)
            i = t[0]
            j = t[1] if i in ws else min(ws)
            r.verdict = 1
            r.phase, r.loc, r.index = cell
            r.tid_i, r.tid_j = i, j
            r.i_writes, r.j_writes = int(i in ws), int(j in ws)
            break
    return r


def _cell_worker(rank, world, port, out_path):
    import json

    import torch.distributed as dist
    from paper_2203_12878_b300 import drf, protogen
    from paper_2203_12878_b300.shard import check_protocol_sharded

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = []
    for p in _cell_cases():
        merged = check_protocol_sharded(rank, world, lambda k, n, p=p: fake_shard_result(p, k, n))
        res.append(drf.result_dict(merged))
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump(res, f)
    dist.barrier()
    dist.destroy_process_group()


def _cell_cases():
    from paper_2203_12878_b300 import protogen
    ps = [protogen.shifted_small(s) for s in range(6)]
    ps += [protogen.config4_one(__import__("random").Random(s), s % 2 == 0) for s in range(6)]
    ps += [q for q in (protogen.random_small(s) for s in range(40)) if q.nthreads >= 2][:16]
    ps.append(protogen.config1("nosync"))
    ps.append(protogen.config1("drf"))
    return ps


def test_gloo_one_protocol_split_by_cells(tmp_path, oracle):
    import json

    out = str(tmp_path / "cells.json")
    mp.start_processes(_cell_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    got = json.load(open(out))
    ps = _cell_cases()
    want = []
    for p in ps:
        d = oracle.check(p.text, p.nthreads, p.cells, p.params, 1)
        d.pop("message", None)
        want.append(d)
    assert len(got) == len(want)
    for p, g, w in zip(ps, got, want):
        if w["status"] == "OVERFLOW":
            continue
        assert g == w, p.text


def test_shard_windows_partition_the_cells():
    from paper_2203_12878_b300 import drf, protogen
    p = protogen.config3(0)
    bc = drf.drf_protocol_compile(p.text)
    for n in (1, 2, 3, 8):
        spans = [drf.drf_shard_range(bc, p.nthreads, p.cells, p.params, k, n) for k in range(n)]
        assert spans[0][0] == 0 and spans[-1][1] == spans[0][2] == 8 * 4 * (1 << 24)
        assert all(spans[k][1] == spans[k + 1][0] for k in range(n - 1))
