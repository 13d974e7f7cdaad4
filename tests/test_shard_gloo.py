"""Sharded batch checking over two CPU ranks (gloo): each rank checks its
slice of a batch, the gathered results equal the unsharded ones in order.
The checker here is the oracle, so no GPU is needed; on GPUs each rank would
call drf_check_batch on its slice."""
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
