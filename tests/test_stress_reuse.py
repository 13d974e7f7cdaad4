"""One context's device buffers, owner table and look-back words reused
across hundreds of launches of different shapes -- single checks, batches
of varied size, plans launched and re-launched in alternation, and a server
fed in bursts -- on each back end, every result against the oracle.

The owner-table back end keeps its table all zero between launches (each
launch clears exactly the records it touched), and interpreted launches of
batches whose protocols all have static phases leave the count and scan
passes out; a record, sync total or phase left over from an earlier launch
would show here as a wrong verdict, witness or count."""
import random

import pytest

from paper_2203_12878_b300 import drf, protogen

pytestmark = pytest.mark.gpu

_EXPECTED = {}


def _pool():
    ps = protogen.config4(master_seed=21, count=48)
    ps += [protogen.random_small(s) for s in range(500, 540)]
    ps += [protogen.config1(v) for v in ("drf", "rdwr", "nosync")]
    ps += [protogen.config2(s, "constructed", target=1e5, plant=s % 2 == 0) for s in range(3)]
    ps.append(protogen.config2(4, "literal", target=1e5))
    return ps


POOL = _pool()


def expected(oracle, i):
    if i not in _EXPECTED:
        p = POOL[i]
        d = oracle.check(p.text, p.nthreads, p.cells, p.params, oracle.METHOD_CELLS)
        d.pop("message", None)
        _EXPECTED[i] = d
    return _EXPECTED[i]


def usable(oracle, i):
    return expected(oracle, i)["status"] != "OVERFLOW"


def compiled(i, cache={}):
    if i not in cache:
        cache[i] = drf.drf_protocol_compile(POOL[i].text)
    return cache[i]


def bounds(i):
    p = POOL[i]
    return (p.nthreads, p.cells, p.params)


def check_one(oracle, i, r, what):
    got = drf.result_dict(r)
    exp = expected(oracle, i)
    assert got == exp, (what, POOL[i].text, got, exp)


@pytest.mark.parametrize("flags", [drf.OPT_PATH_SORT, drf.OPT_PATH_TABLE, 0, drf.OPT_SPECIALIZE])
def test_interleaved_checks_batches_and_plans(oracle, flags):
    rng = random.Random(1000 + flags)
    ids = [i for i in range(len(POOL)) if usable(oracle, i)]
    ctx = drf.drf_ctx_create(0, flags=flags)
    plans = []                       # (plan, protocol ids), launched again later
    launches = 0
    try:
        for step in range(160):
            k = rng.random()
            if k < 0.3:
                i = rng.choice(ids)
                check_one(oracle, i, drf.drf_check(ctx, compiled(i), *bounds(i)), ("check", step))
                launches += 1
            elif k < 0.65:
                sel = [rng.choice(ids) for _ in range(rng.randint(1, 48))]
                res = drf.drf_check_batch(ctx, [compiled(i) for i in sel], [bounds(i) for i in sel])
                for i, r in zip(sel, res):
                    check_one(oracle, i, r, ("batch", step, len(sel)))
                launches += 1
            else:
                if plans and (len(plans) >= 3 or rng.random() < 0.5):
                    plan, sel = plans[rng.randrange(len(plans))]        # an older plan again
                else:
                    n = 1 if (flags & drf.OPT_SPECIALIZE and rng.random() < 0.3) else rng.randint(1, 24)
                    sel = [rng.choice(ids) for _ in range(n)]
                    # a plan takes only protocols that evaluate without error
                    sel = [i for i in sel if expected(oracle, i)["status"] == "OK"] or [ids[0]]
                    plan = drf.drf_plan_create(ctx, [compiled(i) for i in sel], [bounds(i) for i in sel])
                    plans.append((plan, sel))
                    if len(plans) > 3:
                        drf.drf_plan_destroy(plans.pop(0)[0])
                for _ in range(rng.randint(1, 3)):
                    drf.drf_plan_launch(plan)
                    launches += 1
                    for i, r in zip(sel, drf.drf_plan_results(plan)):
                        check_one(oracle, i, r, ("plan", step, len(sel)))
    finally:
        for plan, _ in plans:
            drf.drf_plan_destroy(plan)
        drf.drf_ctx_destroy(ctx)
    assert launches >= 200


@pytest.mark.parametrize("flags", [drf.OPT_PATH_SORT, drf.OPT_PATH_TABLE, 0])
def test_server_bursts_on_reused_buffers(oracle, flags):
    rng = random.Random(77 + flags)
    ids = [i for i in range(len(POOL)) if usable(oracle, i)]
    ctx = drf.drf_ctx_create(0, flags=flags)
    try:
        drf.drf_server_start(ctx, max_round_tuples=1 << 21, poll_us=200)
        done = 0
        for burst in range(12):
            sel = [rng.choice(ids) for _ in range(rng.randint(1, 60))]
            tickets = [drf.drf_server_submit(ctx, compiled(i), *bounds(i)) for i in sel]
            for i, t in zip(sel, tickets):
                out = drf.drf_server_poll(ctx, t, timeout_us=60_000_000)
                assert out is not None
                check_one(oracle, i, out[0], ("server", burst))
                done += 1
        stats = drf.drf_server_stats(ctx)
        drf.drf_server_stop(ctx)
    finally:
        drf.drf_ctx_destroy(ctx)
    assert stats["completed"] == done and stats["rounds"] >= 12


def test_grown_table_starts_clear(oracle):
    """A context's owner table grows (free, then a larger allocation) right
    after another context freed buffers full of non-zero sort keys, which the
    allocator may hand back at the table's old address: the grown table is
    cleared all the same (it once was not when the address came back
    unchanged, and a stale word showed up as a race with a single accessor).
    Race-free protocols of growing table size, every result against the
    oracle."""
    t = drf.drf_ctx_create(0, flags=drf.OPT_PATH_TABLE)
    try:
        for step, cells in enumerate((1 << 12, 1 << 16, 1 << 19, 1 << 21, 1 << 23)):
            s = drf.drf_ctx_create(0, flags=drf.OPT_PATH_SORT)
            try:
                k = protogen.Protocol("array A;\nforU x in 0 .. 64 { rd A[(tid + 977 * x) % 65536]; }\n",
                                      65536, [65536], [])
                drf.drf_check(s, drf.drf_protocol_compile(k.text), k.nthreads, k.cells, k.params)
            finally:
                drf.drf_ctx_destroy(s)
            p = protogen.Protocol("array A, B;\nwr A[tid];\nsync;\nrd A[(tid + 1) %% %d];\nwr B[tid];\n" % cells,
                                  cells, [cells, cells], [])
            got = drf.result_dict(drf.drf_check(t, drf.drf_protocol_compile(p.text), p.nthreads, p.cells, p.params))
            exp = oracle.check(p.text, p.nthreads, p.cells, p.params, oracle.METHOD_CELLS)
            exp.pop("message", None)
            assert got == exp, (step, cells, got)
    finally:
        drf.drf_ctx_destroy(t)
