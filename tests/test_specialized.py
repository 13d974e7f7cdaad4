"""GPU parity of plans that run kernels specialized to their protocol
(count, owner-table and witness passes compiled at run time) against the
oracle: bit-exact status, verdict, witness, divergence and counts."""
import json
import os
import random

import pytest

from paper_2203_12878_b300 import drf, protogen

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def sctx():
    c = drf.drf_ctx_create(0, flags=drf.OPT_SPECIALIZE)
    yield c
    drf.drf_ctx_destroy(c)


@pytest.fixture(scope="module")
def rctx():
    """Specialized plans that take the range pass at any size."""
    c = drf.drf_ctx_create(0, flags=drf.OPT_SPECIALIZE | drf.OPT_RANGE_ANY)
    yield c
    drf.drf_ctx_destroy(c)


def want(oracle, p):
    return oracle.check(p.text, p.nthreads, p.cells, p.params, 1)


def plan_result(ctx, p, launches=2):
    """Result of a one-protocol plan (checked equal over `launches`
    launches), whether it runs specialized kernels, or the creation error."""
    bc = drf.drf_protocol_compile(p.text)
    try:
        plan = drf.drf_plan_create(ctx, [bc], [(p.nthreads, p.cells, p.params)])
    except drf.DrfError as e:
        return {"status": e.name}, False
    try:
        spec, _ = drf.drf_plan_specialized(plan)
        out = None
        for _ in range(launches):
            drf.drf_plan_launch(plan)
            r = drf.result_dict(drf.drf_plan_results(plan)[0])
            assert out is None or r == out
            out = r
        return out, spec
    finally:
        drf.drf_plan_destroy(plan)


def check(ctx, oracle, p, need_spec=True):
    """Compares the plan's result with the oracle's; returns how the plan
    ran (0 interpreted, 1 specialized, 2 specialized with static phases, 3
    the same with the range pass)."""
    exp = {k: v for k, v in want(oracle, p).items() if k != "message"}
    got, spec = plan_result(ctx, p)
    if exp["status"] != "OK":
        assert got["status"] == exp["status"], (p.text, got, exp)
        return spec
    assert got == exp, (p.text, got, exp)
    if need_spec:
        assert spec, p.text
    return spec


def test_paper_examples(sctx, oracle):
    with open(os.path.join(HERE, "golden", "paper_examples.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        p = protogen.Protocol(c["text"], c["nthreads"], c["cells"], c["params"])
        exp = want(oracle, p)
        if exp["status"] in ("OK", "INDEX_OOB", "DIV_ZERO"):
            check(sctx, oracle, p, need_spec=False)


@pytest.mark.parametrize("chunk", range(4))
def test_random_small(sctx, oracle, chunk):
    """Conditionals, thread-dependent bounds, min/max, floor division,
    Euclidean remainder, parameters, syncs, barrier divergence."""
    kinds = []
    for seed in range(chunk * 40, (chunk + 1) * 40):
        p = protogen.random_small(seed)
        if want(oracle, p)["status"] == "OVERFLOW":
            continue
        kinds.append(check(sctx, oracle, p, need_spec=False))
    # both forms of the specialized kernels are exercised
    assert kinds.count(2) >= 5 and kinds.count(1) >= 1, kinds


def late_phase_race(T, rows, racy_row, writer):
    """Row x is written in phase x and read (shifted by one thread) in phase
    x + 1; after the sync of iteration racy_row - 1 (phase racy_row, the
    phase that row racy_row is written in) thread `writer` also writes cell 1
    of row racy_row: a race unless the writer is that cell's own thread 1."""
    text = (f"array A;\nforS x in 0 .. {rows} {{\n  wr A[tid + {T} * x];\n  sync;\n"
            f"  rd A[(tid + 1) % {T} + {T} * x];\n"
            f"  if (tid == {writer} && x == {racy_row - 1}) {{ wr A[{T} * {racy_row} + 1]; }}\n}}\n")
    return protogen.Protocol(text, T, [T * (rows + 1)], [])


@pytest.mark.parametrize("T,rows,racy_row,writer", [(8, 6, 3, 5), (64, 9, 8, 0), (96, 4, 1, 1), (40, 7, 6, 39)])
def test_static_phases_late_race(sctx, oracle, T, rows, racy_row, writer):
    """Phases compiled into the kernels: a race planted in a late phase is
    reported with the oracle's phase and threads (writer 1 owns the cell
    itself in one case: then the protocol is race-free)."""
    p = late_phase_race(T, rows, racy_row, writer)
    assert check(sctx, oracle, p) == 2


@pytest.mark.parametrize("maker", [
    lambda: protogen.config1("drf"), lambda: protogen.config1("rdwr"), lambda: protogen.config1("nosync"),
    lambda: protogen.config2(1, target=3e5), lambda: protogen.config2(2, "constructed", target=3e5, plant=True),
    lambda: protogen.config2(2, "constructed", target=3e5, plant=False),
    lambda: protogen.config4_one(random.Random(3), True), lambda: protogen.config4_one(random.Random(4), False),
])
def test_workload_shapes(sctx, oracle, maker):
    check(sctx, oracle, maker())


def test_record_width_boundary(sctx, oracle):
    for T in (32768, 32769):
        p = protogen.Protocol(f"array A;\nwr A[tid % {T - 1}];\n", T, [T], [])
        check(sctx, oracle, p)


def test_config2_full_size(sctx, oracle):
    """The 1,024-thread protocol at full size, launch after launch; its sync
    structure is the same for every thread, so the plan runs with static
    phases, and its accesses at a * tid plus a loop function (|a| <= 8) make
    most of its tuples, so it takes the range pass."""
    assert check(sctx, oracle, protogen.config2(0)) == 3


@pytest.mark.parametrize("seed,racy", [(0, True), (0, False), (1, True), (1, False)])
def test_config3_full_size(sctx, grid_expected, seed, racy):
    """Grid scale (65,536 threads, ~2.2x10^8 accesses) through specialized
    kernels with static phases and the range pass, launch after launch:
    every result field against the oracle's method B over the whole
    protocol."""
    p = protogen.config3(seed, racy=racy)
    got, spec = plan_result(sctx, p, launches=3)
    assert got == grid_expected(seed, racy)
    assert spec == 3


def test_config3_benchmark_launch_configuration(grid_expected):
    """The benchmark's launch configuration on its workload: an autotuned
    plan with specialization allowed, launched repeatedly, equals the
    oracle over the whole protocol."""
    c = drf.drf_ctx_create(0, flags=drf.OPT_SPECIALIZE | drf.OPT_AUTOTUNE)
    try:
        got, _ = plan_result(c, protogen.config3(0, racy=True), launches=4)
        assert got == grid_expected(0, True)
    finally:
        drf.drf_ctx_destroy(c)


def test_autotuned_specialized_plan(oracle):
    """With the tuner, specialized kernels are candidates beside the
    interpreted back ends; whichever wins gives the oracle's result."""
    c = drf.drf_ctx_create(0, flags=drf.OPT_SPECIALIZE | drf.OPT_AUTOTUNE)
    try:
        p = protogen.config2(5, target=1e6)
        got, _ = plan_result(c, p)
        assert got == {k: v for k, v in want(oracle, p).items() if k != "message"}
    finally:
        drf.drf_ctx_destroy(c)


def test_drf_check_with_specialized_kernels(oracle):
    """drf_check on a context with DRF_OPT_SPECIALIZE: a protocol that may
    make 2^21 accesses or more gets kernels compiled for it on its first
    check, reused by later checks; smaller ones are interpreted.  Results
    equal the oracle's either way, with static and thread-dependent phases,
    checks of different protocols interleaved on the context's buffers."""
    c = drf.drf_ctx_create(0, flags=drf.OPT_SPECIALIZE)
    try:
        # the last one's index is never negative, but the analysis cannot
        # prove it: its phases are thread-dependent (count and scan run)
        big = [protogen.config2(0), protogen.config2(4), protogen.config2(2, "constructed", plant=True),
               protogen.config2(6, "constructed", plant=False), late_phase_race(4096, 600, 500, 7),
               protogen.Protocol("array A;\nforS x in 0 .. 300 {\n  wr A[tid - (tid % 2) + 4096 * x];\n  sync;\n"
                                 "  rd A[(tid + 1) % 4096 + 4096 * x];\n}\n", 4096, [4096 * 300], []),
               # more items than the generator compiles a schedule for: its
               # kernels read the batch's warp-item array
               protogen.Protocol("array A;\nforU x in 0 .. 4000 {\n  forU y in 0 .. 20 {\n"
                                 "    wr A[tid + 64 * ((20 * x + y) % 1000)];\n  }\n}\nsync;\nrd A[(tid + 1) % 64];\n"
                                 "wr A[tid];\n", 64, [64000], [])]
        small = [protogen.config1("nosync"), protogen.random_small(3), protogen.random_small(11)]
        for p in big:
            assert drf.drf_protocol_analyze(drf.drf_protocol_compile(p.text), p.nthreads, p.cells,
                                            p.params)[1]["tuple_bound"] >= 1 << 21
        assert drf.drf_protocol_analyze(drf.drf_protocol_compile(big[-1].text), 64, [64000], [])[1]["items"] > 1024
        for rnd in range(2):
            for p in big + small:
                exp = {k: v for k, v in want(oracle, p).items() if k != "message"}
                if exp["status"] == "OVERFLOW":
                    continue
                got = drf.result_dict(drf.drf_check(c, drf.drf_protocol_compile(p.text), p.nthreads, p.cells, p.params))
                if exp["status"] != "OK":
                    assert got["status"] == exp["status"], (rnd, p.text, got, exp)
                else:
                    assert got == exp, (rnd, p.text, got, exp)
    finally:
        drf.drf_ctx_destroy(c)


def affine_case(seed):
    """A fast loop whose index takes each post-operation (none, mask,
    Euclidean remainder with positive or negative modulus, floor division by
    a positive or negative divisor), some with 64-bit intermediates, some
    with a sync in the body; most are racy."""
    r = random.Random(0xAFF1 ^ (seed * 7919))
    T = r.choice([8, 32, 40, 64])
    post = seed % 4
    a, b = r.randint(-3, 3), r.randint(-5, 5)
    lo = r.randint(0, 4)
    hi = lo + r.randint(1, 13)
    syncs = seed % 3 == 2
    wide = seed % 7 == 3
    big = 4000000000 if wide else 0
    if post == 0:
        c = abs(a) * T + abs(b) * hi + r.randint(0, 9)
        N = 2 * c + 1
        idx = f"{a} * tid + {b} * x + {c}"
    elif post == 1:
        N = r.choice([16, 64, 256])
        idx = f"({a} * tid + {b} * x + {r.randint(0, 50) + big}) % {N}"
    elif post == 2:
        N = r.choice([12, 48, 100, -36])
        idx = f"({a} * tid + {b} * x + {r.randint(0, 50) + big}) % {N}"
        N = abs(N)
    else:
        d = r.choice([2, 3, 5, -2, -3])
        c = abs(a) * T + abs(b) * hi + r.randint(0, 9)
        idx = f"({a} * tid + {b} * x + {c}) / {d}" if d > 0 else f"({a} * tid + {b} * x - {c}) / {d}"
        N = 2 * c + 2
    mode = r.choice(["wr", "rd"])
    body = f"  {mode} A[{idx}];\n  wr A[{idx}];\n" if r.random() < 0.5 else f"  wr A[{idx}];\n"
    if syncs:
        text = f"array A;\nforS x in {lo} .. {hi} {{\n{body}  sync;\n  rd A[({a} * tid + {b} * x + 7) % {N}];\n}}\n"
    else:
        text = f"array A;\nforU x in {lo} .. {hi} {{\n{body}}}\n"
    return text, T, [N]


@pytest.mark.parametrize("chunk", range(3))
def test_witness_hits_solved_per_loop(sctx, oracle, chunk):
    """The witness pass decides whether a thread's fast loop hits the witness
    cell by solving the index equation (a linear congruence whose constants
    the code generator computes) rather than iterating:
    the witness threads (the two smallest accessors of the first racy cell)
    must be the oracle's."""
    wide = 0
    for seed in range(chunk * 16, (chunk + 1) * 16):
        text, T, cells = affine_case(seed)
        p = protogen.Protocol(text, T, cells, [])
        wide += drf.drf_protocol_analyze(drf.drf_protocol_compile(text), T, cells, [])[1]["wide_arithmetic"]
        assert check(sctx, oracle, p) in (2, 3)
    assert wide >= 1


@pytest.mark.parametrize("chunk", range(4))
def test_range_pass_against_oracle(rctx, oracle, chunk):
    """Accesses at +-tid plus a function of the loop variables (with and
    without a remainder, arrays of odd sizes across several 16384-record
    tasks, conditions on loop variables) go through the range pass, mixed
    with accesses of other tid coefficients that the table pass applies and
    the range pass merges: every result field equals the oracle's, launch
    after launch."""
    kinds = []
    for seed in range(chunk * 20, (chunk + 1) * 20):
        kinds.append(check(rctx, oracle, protogen.shifted_small(seed)))
    assert kinds.count(3) >= 10, kinds


@pytest.mark.parametrize("chunk", range(4))
def test_strided_range_pass_against_oracle(rctx, oracle, chunk):
    """Accesses at a * tid plus a function of the loop variables, |a| in
    2..8 (pieces whose records lie a apart, interleaving without meeting
    when their offsets differ mod a), with and without a remainder, mixed
    with +-tid, tid-free and conditional accesses: every result field equals
    the oracle's, launch after launch."""
    kinds = []
    for seed in range(chunk * 20, (chunk + 1) * 20):
        kinds.append(check(rctx, oracle, protogen.strided_small(seed)))
    assert kinds.count(3) >= 15, kinds


@pytest.mark.parametrize("text,T,cells", [
    ("array A;\nforU x in 0 .. 4 { rd A[x]; }\nsync;\nwr A[3];\n", 64, [8]),            # all threads write one cell
    ("array A;\nforU x in 0 .. 9 { rd A[(x * 7) % 5]; }\n", 300, [5]),                  # shared reads only
    ("array A, B;\nforU x in 0 .. 6 { rd A[x]; wr B[tid + 64 * x]; }\nwr A[5];\n", 64, [8, 512]),
    ("array A;\nforU x in 0 .. 3 { wr A[2 * tid + x]; }\nsync;\nrd A[7];\n", 1, [8]),    # one thread
])
def test_range_pass_tid_free_accesses(rctx, oracle, text, T, cells):
    """Accesses whose index does not depend on tid go to the range pass as
    one record per offset, saturated when two or more threads reach it; the
    witness comes from the two smallest threads of such a piece."""
    assert check(rctx, oracle, protogen.Protocol(text, T, cells, [])) == 3


@pytest.mark.parametrize("text,T,cells", [
    ("array A;\nforU x in 0 .. 5 { rd A[(6 * tid + x) % 4096]; }\nwr A[(7 * tid + 3) % 4096];\n", 853, [4096]),
    ("array A;\nforU x in 0 .. 4 { rd A[(-5 * tid + 2 * x) % 1000]; }\nsync;\nwr A[(-3 * tid + 1) % 1000];\n",
     700, [1000]),
    ("array A;\nwr A[(4 * tid) % 1000];\n", 600, [1000]),                            # t and t + 250 collide
    ("array A, B;\nforU x in 0 .. 3 { wr B[(9 * tid + 1000 * x) % 3001]; rd A[(2 * tid) % 999]; }\n", 2000, [999, 3001]),
])
def test_range_pass_multi_wrap(rctx, oracle, text, T, cells):
    """Indices that wrap around their modulus several times over the
    threads: one run of tids per wrap, the runs of one offset meeting (or
    not) in the task's records."""
    assert check(rctx, oracle, protogen.Protocol(text, T, cells, [])) == 3


def test_small_protocols_skip_the_range_pass_by_default(sctx, oracle):
    """Under 2^22 range tuples a check keeps the table pass alone (same
    results)."""
    for seed in range(6):
        assert check(sctx, oracle, protogen.shifted_small(seed)) in (1, 2)


def test_config3_runs_the_range_pass(sctx):
    p = protogen.config3(0, racy=True)
    plan = drf.drf_plan_create(sctx, [drf.drf_protocol_compile(p.text)], [(p.nthreads, p.cells, p.params)])
    try:
        assert drf.drf_plan_specialized(plan)[0] == 3
        # init, table, range, touch listing, table scan, witness, result
        assert drf.drf_plan_info(plan)["kernels_per_launch"] == 7
        drf.drf_plan_launch(plan)
        tuples, updates = drf.drf_plan_range_tuples(plan)
        assert tuples == 221642754 - 2 and 0 < updates < tuples
    finally:
        drf.drf_plan_destroy(plan)
