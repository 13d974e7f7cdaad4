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
    exp = {k: v for k, v in want(oracle, p).items() if k != "message"}
    got, spec = plan_result(ctx, p)
    if exp["status"] != "OK":
        assert got["status"] == exp["status"], (p.text, got, exp)
        return
    assert got == exp, (p.text, got, exp)
    if need_spec:
        assert spec, p.text


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
    for seed in range(chunk * 40, (chunk + 1) * 40):
        p = protogen.random_small(seed)
        if want(oracle, p)["status"] == "OVERFLOW":
            continue
        check(sctx, oracle, p, need_spec=False)


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
    """The benchmarked protocol at full size, launch after launch."""
    check(sctx, oracle, protogen.config2(0))


def test_config3_full_size_racy(sctx, oracle):
    """Grid scale (65,536 threads: 64-bit owner records), one planted race;
    the witness threads come from the oracle's one-cell recomputation."""
    p = protogen.config3(0, racy=True)
    got, spec = plan_result(sctx, p, launches=1)
    m = p.meta
    assert spec and got["status"] == "OK" and got["tuples"] == m["accesses"] + 2
    assert (got["verdict"], got["phase"], got["loc"], got["index"]) == ("RACY", m["phase"], m["loc"], m["index"])
    cell = oracle.cell(p.text, p.nthreads, p.cells, p.params, m["phase"], m["loc"], m["index"])
    assert {k: got[k] for k in ("tid_i", "tid_j", "i_writes", "j_writes")} == \
           {k: cell[k] for k in ("tid_i", "tid_j", "i_writes", "j_writes")}


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
