"""GPU parity: the CUDA pipeline, called through the C ABI, against the
oracle.  Everything here is integer work, so the bar is bit-exact equality of
status, verdict, witness (phase, array, index, i, j, i_writes, j_writes),
divergence fields, error tid and ordinal, tuple and phase counts."""
import json
import os
import random

import numpy as np
import pytest

from paper_2203_12878_b300 import drf, protogen

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
CELLS = 1


PATH_FLAGS = {"sort": drf.OPT_PATH_SORT, "table": drf.OPT_PATH_TABLE,
              "table+range": drf.OPT_PATH_TABLE | drf.OPT_RANGE_ANY,   # range pass at any size
              "sort+range": drf.OPT_PATH_SORT | drf.OPT_RANGE_ANY}     # range accesses' keys from the pieces
TABLE_LIMIT = 64 << 30           # bytes: the largest owner table the library sets up


@pytest.fixture(scope="module", params=["sort", "table", "table+range", "sort+range"])
def ctx(request):
    """A context forced onto one back end; every test using it runs on both
    (each with and without the range pieces)."""
    c = drf.drf_ctx_create(0, flags=PATH_FLAGS[request.param])
    c.path = request.param
    yield c
    drf.drf_ctx_destroy(c)


@pytest.fixture(scope="module")
def sort_ctx():
    c = drf.drf_ctx_create(0, flags=drf.OPT_PATH_SORT)
    yield c
    drf.drf_ctx_destroy(c)


def run(ctx, p):
    bc = drf.drf_protocol_compile(p.text)
    try:
        return drf.result_dict(drf.drf_check(ctx, bc, p.nthreads, p.cells, p.params))
    except drf.DrfError as e:
        return {"status": e.name}


def table_fits(p):
    """Whether the owner table of p is within the library's limit: one
    record (4 bytes, 8 above 15-bit thread ids) per cell and phase row."""
    st, a = drf.drf_protocol_analyze(drf.drf_protocol_compile(p.text), p.nthreads, p.cells, p.params)
    if st != "OK":
        return True
    rec = 8 if max(p.nthreads - 1, 0).bit_length() > 15 else 4
    return (a["sync_bound"] + 1) * sum(p.cells) * rec <= TABLE_LIMIT


def want(oracle, p, ctx=None):
    exp = oracle.check(p.text, p.nthreads, p.cells, p.params, CELLS)
    if ctx is not None and getattr(ctx, "path", "").startswith("table") and exp["status"] == "OK" and not table_fits(p):
        return {"status": "LIMIT"}
    return exp


def same(got, exp):
    exp = {k: v for k, v in exp.items() if k != "message"}
    return got == exp


def test_paper_examples(ctx):
    with open(os.path.join(HERE, "golden", "paper_examples.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        p = protogen.Protocol(c["text"], c["nthreads"], c["cells"], c["params"])
        try:
            got = run(ctx, p)
        except drf.DrfError as e:
            got = {"status": e.name}
        for k, v in c["expect"].items():
            assert got[k] == v, (c["name"], k, got)


@pytest.mark.parametrize("chunk", range(6))
def test_random_small_sweep(ctx, oracle, chunk):
    """600 tiny protocols per chunk over the whole syntax: conditionals,
    thread-dependent bounds, min/max, floor division, Euclidean remainder,
    parameters, syncs, evaluation errors, barrier divergence."""
    mism = []
    for seed in range(chunk * 600, (chunk + 1) * 600):
        p = protogen.random_small(seed)
        exp = want(oracle, p, ctx)
        if exp["status"] == "OVERFLOW":
            continue
        got = run(ctx, p)
        if not same(got, exp):
            mism.append((seed, got, exp))
    assert not mism, mism[:3]


def _decode(keys, lay):
    tb, ib, lb, pb = lay["tid_bits"], lay["idx_bits"], lay["loc_bits"], lay["phase_bits"]
    k = keys.astype(np.uint64)
    mode = k & np.uint64(1)
    k = k >> np.uint64(1)
    tid = k & np.uint64((1 << tb) - 1)
    k = k >> np.uint64(tb)
    idx = k & np.uint64((1 << ib) - 1)
    k = k >> np.uint64(ib)
    loc = k & np.uint64((1 << lb) - 1)
    k = k >> np.uint64(lb)
    phase = k & np.uint64((1 << pb) - 1)
    return np.stack([phase, loc, idx, tid, mode], axis=1)


def _rows_sorted(rows):
    order = np.lexsort(rows.T[::-1])
    return rows[order]


@pytest.mark.parametrize("maker", [
    lambda: protogen.config1("drf"), lambda: protogen.config1("nosync"),
    lambda: protogen.config2(2, target=3e5), lambda: protogen.config2(4, "constructed", target=3e5),
    lambda: protogen.config4_one(random.Random(11), True),
])
def test_emitted_keys_are_the_access_multiset_and_sorted(sort_ctx, oracle, maker):
    """Stage check: the keys the emit kernel wrote are exactly the oracle's
    dynamic accesses (as a multiset), and after the radix passes they are
    ordered by (phase, array, index)."""
    p = maker()
    got = run(sort_ctx, p)
    assert got["status"] == "OK"
    keys, lay = drf.drf_debug_sorted_keys(sort_ctx)
    rows = _decode(keys, lay)
    seg = keys >> np.uint64(lay["tid_bits"] + 1)
    assert np.all(seg[1:] >= seg[:-1])
    ref = oracle.tuples(p.text, p.nthreads, p.cells, p.params)
    assert len(ref) == len(rows) == got["tuples"]
    assert np.array_equal(_rows_sorted(rows), _rows_sorted(ref.astype(np.uint64)))


def test_random_small_keys(sort_ctx, oracle):
    for seed in range(200):
        p = protogen.random_small(seed)
        exp = want(oracle, p)
        if exp["status"] != "OK" or exp["verdict"] == "BARRIER_DIVERGENCE":
            continue
        run(sort_ctx, p)
        keys, lay = drf.drf_debug_sorted_keys(sort_ctx)
        ref = oracle.tuples(p.text, p.nthreads, p.cells, p.params)
        rows = _decode(keys, lay) if len(keys) else np.zeros((0, 5), np.uint64)
        assert np.array_equal(_rows_sorted(rows), _rows_sorted(ref.astype(np.uint64))), p.text


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("mode", ["literal", "constructed"])
def test_config2_shapes_small(ctx, oracle, seed, mode):
    """The one-protocol workload's shape (1024 threads, two arrays of 2^20
    cells, depth-3 nests, 1..6 syncs) at ~2x10^5 accesses: several sort tiles
    and ragged tails."""
    p = protogen.config2(seed, mode, target=2e5)
    assert same(run(ctx, p), want(oracle, p, ctx))


@pytest.mark.parametrize("seed,mode,plant", [(0, "literal", None), (3, "constructed", True),
                                             (3, "constructed", False)])
def test_config2_full_size(ctx, oracle, seed, mode, plant):
    """The benchmarked workload at full size (~10^7 accesses), same launch
    path as the benchmark: whole result against the oracle."""
    p = protogen.config2(seed, mode, plant=plant)
    assert same(run(ctx, p), want(oracle, p, ctx))


def test_config2_full_size_plan_equals_check(ctx, oracle):
    """The captured-graph path the benchmark times gives the same result as
    the direct path and the oracle, launch after launch."""
    p = protogen.config2(0)
    bc = drf.drf_protocol_compile(p.text)
    plan = drf.drf_plan_create(ctx, [bc], [(p.nthreads, p.cells, p.params)])
    try:
        exp = want(oracle, p, ctx)
        for _ in range(3):
            drf.drf_plan_launch(plan)
            got = drf.result_dict(drf.drf_plan_results(plan)[0])
            assert same(got, exp)
        info = drf.drf_plan_info(plan)
        assert info["tuples"] == exp["tuples"]
    finally:
        drf.drf_plan_destroy(plan)


def test_batch_equals_alone_and_oracle(ctx, oracle):
    ps = protogen.config4(master_seed=7, count=96)
    ps += [protogen.random_small(s) for s in range(40)]
    ps.append(protogen.config1("nosync"))
    bcs = [drf.drf_protocol_compile(p.text) for p in ps]
    res = drf.drf_check_batch(ctx, bcs, [(p.nthreads, p.cells, p.params) for p in ps])
    for p, r in zip(ps, res):
        exp = want(oracle, p, ctx)
        if exp["status"] == "OVERFLOW":
            continue
        assert same(drf.result_dict(r), exp), p.text
    for p, r in list(zip(ps, res))[::9]:
        assert drf.result_dict(r) == run(ctx, p)


@pytest.mark.parametrize("case", [
    ("array A;\nwr A[tid];\n", 0, [4], []),                        # no threads
    ("array A;\nwr A[0];\n", 1, [1], []),                          # one thread
    ("", 5, [], []),                                               # empty protocol
    ("array A;\nforS x in 0 .. 3 { sync; }\n", 64, [1], []),       # syncs only
    ("array A;\nrd A[0];\n", 3, [0], []),                          # zero-size array
    ("array A;\nwr A[tid % 7];\n", 1 << 20, [7], []),              # a million threads
    ("array A;\nrd A[tid];\nwr A[tid * 2 % 1000003];\n", 200000, [1000003], []),
    ("array A, B;\nwr B[tid];\nsync;\nwr A[tid % 2];\n", 33, [1, 64], []),
    ("array A;\nforU x in 0 .. 70000 { wr A[x]; }\n", 2, [70000], []),      # one long item loop
    ("array A;\nwr A[4294967295 + tid];\n", 2, [1 << 40], []),      # 40-bit index field
])
def test_edge_cases(ctx, oracle, case):
    text, T, cells, params = case
    p = protogen.Protocol(text, T, cells, params)
    assert same(run(ctx, p), want(oracle, p, ctx))


def test_key_too_wide_is_reported(ctx):
    p = protogen.Protocol("array A;\nwr A[tid];\n", 1 << 27, [1 << 40], [])
    got = run(ctx, p)
    assert got["status"] == "KEY_TOO_WIDE"


@pytest.mark.parametrize("poll_us", [0, 500])
def test_server_results_equal_alone(ctx, oracle, poll_us):
    ps = protogen.config4(master_seed=3, count=60) + [protogen.config2(1, target=3e5)]
    s = drf.drf_ctx_create(0, flags=PATH_FLAGS[ctx.path])
    try:
        drf.drf_server_start(s, max_round_tuples=1 << 20, poll_us=poll_us)
        tickets = [drf.drf_server_submit(s, drf.drf_protocol_compile(p.text), p.nthreads, p.cells, p.params)
                   for p in ps]
        out = [drf.drf_server_poll(s, t, timeout_us=60_000_000) for t in tickets]
        stats = drf.drf_server_stats(s)
        drf.drf_server_stop(s)
    finally:
        drf.drf_ctx_destroy(s)
    assert stats["completed"] == len(ps) and stats["rounds"] >= 2
    for i, (p, o) in enumerate(zip(ps, out)):
        assert o is not None
        got = drf.result_dict(o[0])
        if not same(got, want(oracle, p, ctx)):
            print(json.dumps({"i": i, "got": got, "stats": stats}))
        assert same(got, want(oracle, p, ctx))


def test_server_rejects_bad_options():
    s = drf.drf_ctx_create(0)
    try:
        with pytest.raises(drf.DrfError) as e:
            drf.drf_server_start(s, poll_us=2_000_000)     # polls of more than a second
        assert e.value.name == "INVALID_ARG"
    finally:
        drf.drf_ctx_destroy(s)


def test_param_sweep_equals_per_value(ctx, oracle):
    """Fig. 1's MAP with M swept over 0..9 in one batched pass: DRF for M = 0,
    racy on cell 0 for every M >= 1; each entry equals the oracle at that M."""
    text = "array A;\nparam M;\nforU x in 0 .. M { rd A[x]; wr A[x]; }\n"
    bc = drf.drf_protocol_compile(text)
    res = drf.drf_check_param_sweep(ctx, bc, 4, [16], [0], 0, 0, 10)
    for m, r in enumerate(res):
        assert same(drf.result_dict(r), oracle.check(text, 4, [16], [m], CELLS))
    assert drf.result_dict(res[0])["verdict"] == "DRF"
    assert all(drf.result_dict(r)["verdict"] == "RACY" for r in res[1:])
    # a parameter that moves an index out of range in part of the sweep
    text2 = "array A;\nparam K;\nwr A[tid + K];\n"
    res2 = drf.drf_check_param_sweep(ctx, drf.drf_protocol_compile(text2), 4, [6], [0], 0, -1, 4)
    for k, r in zip(range(-1, 4), res2):
        assert same(drf.result_dict(r), oracle.check(text2, 4, [6], [k], CELLS))


@pytest.mark.parametrize("racy", [False, True])
def test_config3_full_size(ctx, grid_expected, racy):
    """Grid-scale protocol (65,536 threads, 4 arrays of 2^24 cells, 8 phases,
    ~2.2x10^8 accesses) at full size on both back ends: every result field
    against the oracle's method B over the whole protocol (all threads, all
    accesses).  Thread ids there need 17 bits of the sort key and 64-bit
    owner records."""
    p = protogen.config3(0, racy=racy)
    exp = grid_expected(0, racy)
    assert exp["status"] == "OK" and exp["verdict"] == ("RACY" if racy else "DRF")
    assert same(run(ctx, p), exp)


def test_autotuned_batched_plan(oracle):
    """The batched workload's shape through an autotuned plan (every
    candidate launch configuration is run while tuning): the chosen
    configuration is a candidate and every result equals the oracle."""
    c = drf.drf_ctx_create(0, flags=drf.OPT_AUTOTUNE)
    try:
        ps = protogen.config4(master_seed=11, count=64)
        plan = drf.drf_plan_create(c, [drf.drf_protocol_compile(p.text) for p in ps],
                                   [(p.nthreads, p.cells, p.params) for p in ps])
        cfg = drf.drf_plan_config(plan)
        assert cfg["granularity"] in (32, 128, 512) and cfg["radix_items"] in (12, 16, 24)
        assert drf.drf_plan_path(plan) in ("sort", "table")
        for _ in range(2):
            drf.drf_plan_launch(plan)
            for p, r in zip(ps, drf.drf_plan_results(plan)):
                assert same(drf.result_dict(r), want(oracle, p))
        drf.drf_plan_destroy(plan)
    finally:
        drf.drf_ctx_destroy(c)


# ------------------------------------------------------------ owner table

@pytest.mark.parametrize("T", [2, 32767, 32768, 32769, 65536])
def test_owner_record_width_boundary(ctx, oracle, T):
    """Thread ids up to 15 bits take 32-bit owner records, wider ones 64-bit
    records: the first and the last thread collide on one cell, and only
    they do."""
    text = "array A;\nwr A[tid % (NT - 1)];\n".replace("NT", str(T))
    p = protogen.Protocol(text, T, [T], [])
    got = run(ctx, p)
    assert same(got, want(oracle, p, ctx))
    assert (got["verdict"], got["index"], got["tid_i"], got["tid_j"]) == ("RACY", 0, 0, T - 1)


def test_table_is_clean_between_checks(ctx, oracle):
    """A racy check followed by race-free checks of the same shape on one
    context: records of the first must not leak into the next (the table
    scan clears what it reads)."""
    racy = protogen.config2(3, "constructed", target=3e5, plant=True)
    clean = protogen.config2(3, "constructed", target=3e5, plant=False)
    for p in (racy, clean, racy, clean, clean):
        assert same(run(ctx, p), want(oracle, p, ctx))


def test_table_reuse_across_many_batches(oracle):
    """Ninety protocols in small batches, one after another on one owner-table
    context, three times in different groupings: every record a
    launch creates must be cleared before the next (a record left behind
    would surface as a false race wherever a later batch's rows land)."""
    ps = protogen.config4(master_seed=11, count=90)
    exp = [want(oracle, p) for p in ps]            # small tables: no size limit applies
    bcs = [drf.drf_protocol_compile(p.text) for p in ps]
    c = drf.drf_ctx_create(0, flags=drf.OPT_PATH_TABLE)
    try:
        for size, shift in ((3, 0), (2, 1), (5, 2)):
            idx = list(range(shift, len(ps))) + list(range(shift))
            for g in range(0, len(idx), size):
                grp = idx[g:g + size]
                res = drf.drf_check_batch(c, [bcs[i] for i in grp], [(ps[i].nthreads, ps[i].cells, ps[i].params) for i in grp])
                for i, r in zip(grp, res):
                    assert same(drf.result_dict(r), exp[i]), (size, shift, i, ps[i].text)
    finally:
        drf.drf_ctx_destroy(c)


def test_table_plan_replays(oracle):
    """Graph replays of an owner-table plan: the witness is found launch after
    launch (each launch leaves the table zero for the next)."""
    c = drf.drf_ctx_create(0, flags=drf.OPT_PATH_TABLE)
    try:
        ps = [protogen.config2(3, "constructed", target=3e5, plant=True), protogen.config1("nosync"),
              protogen.config1("drf"), protogen.random_small(5)]
        plan = drf.drf_plan_create(c, [drf.drf_protocol_compile(p.text) for p in ps],
                                   [(p.nthreads, p.cells, p.params) for p in ps])
        assert drf.drf_plan_path(plan) == "table"
        info = drf.drf_plan_info(plan)
        assert info["sort_passes"] == 0
        for _ in range(4):
            drf.drf_plan_launch(plan)
            for p, r in zip(ps, drf.drf_plan_results(plan)):
                assert same(drf.result_dict(r), want(oracle, p))
        drf.drf_plan_destroy(plan)
    finally:
        drf.drf_ctx_destroy(c)


def test_automatic_path_choice(oracle):
    """Without a forced back end the library picks one per batch; results are
    the same either way."""
    c = drf.drf_ctx_create(0)
    try:
        for p in (protogen.config1("nosync"), protogen.config2(0, target=3e5),
                  protogen.Protocol("array A;\nwr A[4294967295 + tid];\n", 2, [1 << 40], [])):
            assert same(run(c, p), want(oracle, p))
    finally:
        drf.drf_ctx_destroy(c)


def test_lookback_wait_runs_out_and_context_recovers(oracle):
    """The radix look-back's bounded wait, made to run out: with the test
    hook, tile 0 of every radix pass publishes nothing and the tiles after
    it give up after 64 waits.  The check returns DRF_E_TIMEOUT (nothing
    faults: the waits end and every store stays in the key buffers), and
    the next checks on the same context equal the oracle."""
    c = drf.drf_ctx_create(0, flags=drf.OPT_PATH_SORT)
    try:
        p = protogen.config2(2, target=2e5)           # ~50 radix tiles per pass
        bc = drf.drf_protocol_compile(p.text)
        exp = want(oracle, p)
        assert same(run(c, p), exp)
        drf.drf_debug_stall_lookback(c, 1)
        with pytest.raises(drf.DrfError) as e:
            drf.drf_check(c, bc, p.nthreads, p.cells, p.params)
        assert e.value.name == "TIMEOUT"
        for _ in range(2):
            assert same(run(c, p), exp)
        q = protogen.config1("nosync")
        assert same(run(c, q), want(oracle, q))
    finally:
        drf.drf_ctx_destroy(c)


@pytest.mark.parametrize("nshards", [1, 2, 3, 5])
def test_one_protocol_split_by_cells(oracle, nshards):
    """drf_check_shard over every shard of a protocol, merged by
    drf_merge_shards, equals the oracle on the whole protocol -- every
    field, races in one shard or several, errors and divergence (facts of
    the whole protocol that every shard reports alike)."""
    c = drf.drf_ctx_create(0)
    try:
        ps = [protogen.shifted_small(s) for s in range(8)]
        ps += protogen.config4(master_seed=13, count=10)
        ps += [protogen.random_small(s) for s in range(60, 100)]
        ps += [protogen.config1(v) for v in ("drf", "nosync")]
        for p in ps:
            exp = want(oracle, p)
            if exp["status"] == "OVERFLOW":
                continue
            bc = drf.drf_protocol_compile(p.text)
            parts = [drf.drf_check_shard(c, bc, p.nthreads, p.cells, p.params, k, nshards) for k in range(nshards)]
            assert same(drf.result_dict(drf.drf_merge_shards(parts)), exp), p.text
    finally:
        drf.drf_ctx_destroy(c)


def test_grid_scale_split_by_cells(grid_expected):
    """The grid-scale protocol (65,536 threads, 2.2e8 accesses) in four
    shards: each shard records only its quarter of the cells; the merged
    result equals the oracle over the whole protocol."""
    c = drf.drf_ctx_create(0)
    try:
        p = protogen.config3(0, racy=True)
        bc = drf.drf_protocol_compile(p.text)
        parts = [drf.drf_check_shard(c, bc, p.nthreads, p.cells, p.params, k, 4) for k in range(4)]
        assert sum(drf.result_dict(x)["verdict"] == "RACY" for x in parts) == 1
        assert drf.result_dict(drf.drf_merge_shards(parts)) == grid_expected(0, True)
    finally:
        drf.drf_ctx_destroy(c)


@pytest.mark.parametrize("bits", [4, 5, 6, 7, 8])
def test_radix_digit_width(oracle, bits):
    """The sort path with every radix digit width the context may fix: the
    pass count follows the width (widened when the key would need more than
    eight passes) and every result equals the oracle."""
    c = drf.drf_ctx_create(0, radix_bits=bits, flags=drf.OPT_PATH_SORT)
    try:
        ps = [protogen.config2(1, target=2e5), protogen.config2(3, "constructed", target=2e5, plant=True)]
        ps += [protogen.random_small(s) for s in range(200, 230)]
        for p in ps:
            assert same(run(c, p), want(oracle, p)), p.text
        batch = protogen.config4(master_seed=17, count=24)
        plan = drf.drf_plan_create(c, [drf.drf_protocol_compile(p.text) for p in batch],
                                   [(p.nthreads, p.cells, p.params) for p in batch])
        try:
            info, cfg = drf.drf_plan_info(plan), drf.drf_plan_config(plan)
            width = max(bits, -(-info["sort_bits"] // 8))
            assert cfg["radix_bits"] == width and info["sort_passes"] == -(-info["sort_bits"] // width)
            drf.drf_plan_launch(plan)
            for p, r in zip(batch, drf.drf_plan_results(plan)):
                assert same(drf.result_dict(r), want(oracle, p))
        finally:
            drf.drf_plan_destroy(plan)
    finally:
        drf.drf_ctx_destroy(c)


def test_autotuned_radix_width(oracle):
    """The tuner picks the digit width of a sort-path plan among 6, 7 and 8
    bits; the plan it keeps gives the oracle's results."""
    c = drf.drf_ctx_create(0, flags=drf.OPT_AUTOTUNE | drf.OPT_PATH_SORT)
    try:
        ps = protogen.config4(master_seed=19, count=48)
        plan = drf.drf_plan_create(c, [drf.drf_protocol_compile(p.text) for p in ps],
                                   [(p.nthreads, p.cells, p.params) for p in ps])
        try:
            assert drf.drf_plan_config(plan)["radix_bits"] in (6, 7, 8)
            drf.drf_plan_launch(plan)
            for p, r in zip(ps, drf.drf_plan_results(plan)):
                assert same(drf.result_dict(r), want(oracle, p))
        finally:
            drf.drf_plan_destroy(plan)
    finally:
        drf.drf_ctx_destroy(c)


def test_server_splits_a_round_that_does_not_fit(oracle):
    """Requests whose owner tables fit the context's device-memory cap one at
    a time, but not two in one round: the server runs such a round again in
    halves, so every request gets the result it gets alone."""
    n = 1 << 23                                   # a 32 MiB table per request
    texts = [f"array A;\nwr A[(tid + {k}) % {n}];\n" for k in range(5)] + ["array A;\nwr A[tid % 3];\n"]
    c = drf.drf_ctx_create(0, flags=drf.OPT_PATH_TABLE, max_device_bytes=48 << 20)
    try:
        drf.drf_server_start(c)
        tickets = [drf.drf_server_submit(c, drf.drf_protocol_compile(t), 1024, [n], []) for t in texts]
        got = [drf.result_dict(drf.drf_server_poll(c, tk, timeout_us=60_000_000)[0]) for tk in tickets]
        drf.drf_server_stop(c)
    finally:
        drf.drf_ctx_destroy(c)
    for t, g in zip(texts, got):
        assert same(g, oracle.check(t, 1024, [n], [], CELLS)), t
    assert got[-1]["verdict"] == "RACY"


def test_sort_path_batch_emits_range_keys(oracle):
    """A forced sort path over a batch: the range accesses' keys come from
    the pieces (one per distinct thread and offset), the others from the
    interpreter; fewer keys than tuples, every result equal to the oracle,
    launch after launch."""
    c = drf.drf_ctx_create(0, flags=drf.OPT_PATH_SORT | drf.OPT_RANGE_ANY)
    try:
        ps = protogen.config4(master_seed=29, count=40) + [protogen.shifted_small(s) for s in range(40, 60)]
        ps += [protogen.strided_small(s) for s in range(200, 220)] + [protogen.random_small(s) for s in range(330, 340)]
        ps = [p for p in ps if want(oracle, p)["status"] == "OK"]
        plan = drf.drf_plan_create(c, [drf.drf_protocol_compile(p.text) for p in ps],
                                   [(p.nthreads, p.cells, p.params) for p in ps])
        try:
            assert drf.drf_plan_path(plan) == "sort"
            for _ in range(3):
                drf.drf_plan_launch(plan)
                for p, r in zip(ps, drf.drf_plan_results(plan)):
                    assert same(drf.result_dict(r), want(oracle, p)), p.text
            info = drf.drf_plan_info(plan)
            assert 0 < drf.drf_plan_keys(plan) < info["tuples"]
        finally:
            drf.drf_plan_destroy(plan)
    finally:
        drf.drf_ctx_destroy(c)


def test_interpreted_batch_runs_the_range_pass(oracle):
    """An interpreted owner-table plan over a batch: the protocols whose
    accesses at +-tid plus loop terms make most of their tuples go to the
    range pass (tasks spanning several protocols' rows), the others to the
    table pass alone; every result equals the oracle, launch after launch."""
    c = drf.drf_ctx_create(0, flags=drf.OPT_PATH_TABLE | drf.OPT_RANGE_ANY)
    try:
        ps = protogen.config4(master_seed=23, count=40) + [protogen.shifted_small(s) for s in range(20)]
        ps += [protogen.strided_small(s) for s in range(100, 120)]
        ps += [protogen.random_small(s) for s in range(300, 320)]
        ps = [p for p in ps if want(oracle, p)["status"] == "OK"]
        plan = drf.drf_plan_create(c, [drf.drf_protocol_compile(p.text) for p in ps],
                                   [(p.nthreads, p.cells, p.params) for p in ps])
        try:
            for _ in range(3):
                drf.drf_plan_launch(plan)
                for p, r in zip(ps, drf.drf_plan_results(plan)):
                    assert same(drf.result_dict(r), want(oracle, p)), p.text
            tuples, updates = drf.drf_plan_range_tuples(plan)
            assert tuples > 0 and updates > 0
        finally:
            drf.drf_plan_destroy(plan)
    finally:
        drf.drf_ctx_destroy(c)
