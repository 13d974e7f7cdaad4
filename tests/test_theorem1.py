"""Theorem 1 (Sec. 4) as a differential property, and the typing examples.

For a well-typed BabyCUDA program b with inferred MAP u (rules of Fig. 4,
implemented by the library's drf_babycuda_infer), the access values of b's
history (Fig. 3 semantics with array contents, executed by oracle/babycuda.py)
equal u's access values (evaluated by the oracle's MAP interpreter), phase
by phase; hence the history is DRF iff the MAP is (Definition 1)."""
import pytest

from oracle import babycuda
from paper_2203_12878_b300 import drf, protogen


def test_typing_examples_of_the_paper():
    # Fig. 1 (middle -> right) and Fig. 2 (middle -> right), Sec. 4 "Examples"
    fig1 = "array A;\nparam M;\nfor x in 0 .. M {\n  let y = A[x];\n  A[x] := y + 1;\n}\n"
    fig1_map = "array A;\nparam M;\nforU x in 0 .. M {\n  rd A[x];\n  wr A[x];\n}\n"
    assert drf.drf_babycuda_infer(fig1) == drf.drf_protocol_compile(fig1_map)
    fig2 = "array A;\nif (tid = 0) {\n  A[0] := tid;\n} else {\n  skip;\n}\n"
    fig2_map = "array A;\nif (tid = 0) { wr A[0]; } else { skip; }\n"
    assert drf.drf_babycuda_infer(fig2) == drf.drf_protocol_compile(fig2_map)


def test_illtyped_program_is_rejected():
    # eqn. illtyped: A[tid] := tid; let x = A[tid] in A[x] := 9
    with pytest.raises(drf.DrfError) as e:
        drf.drf_babycuda_infer("array A;\nA[tid] := tid;\nlet x = A[tid];\nA[x] := 9;\n")
    assert e.value.name == "UNBOUND_VAR"


@pytest.mark.parametrize("text", [
    "array A;\nlet x = A[0];\nif (x > 1) { A[tid] := 1; }\n",       # data-dependent control (t-if)
    "array A;\nlet x = A[0];\nfor i in 0 .. x { A[i] := 1; }\n",     # data-dependent bound (t-for)
    "array A;\nlet x = A[0];\nlet y = A[x];\n",                       # data-dependent read index (t-read)
])
def test_data_dependence_is_not_typable(text):
    with pytest.raises(drf.DrfError) as e:
        drf.drf_babycuda_infer(text)
    assert e.value.name == "UNBOUND_VAR"


def test_payloads_may_use_data():
    bc = drf.drf_babycuda_infer("array A;\nlet x = A[tid];\nlet y = A[0];\nA[tid] := x * y + min(x, 3);\n")
    assert "rd A0[tid]" in drf.drf_protocol_text(bc)


def test_map_text_round_trips():
    for seed in range(300):
        p = protogen.random_small(seed)
        bc = drf.drf_protocol_compile(p.text)
        assert drf.drf_protocol_compile(drf.drf_protocol_text(bc)) == bc


def _oracle_access_set(oracle, map_text, p):
    rows = oracle.tuples(map_text, p.nthreads, p.cells, p.params)
    return {tuple(int(v) for v in row) for row in rows}


def test_theorem1_on_random_programs(oracle):
    """Access values of the history == access values of the inferred MAP,
    and DRF(history) == DRF(MAP), over 600 random well-typed programs."""
    checked = racy = 0
    for seed in range(600):
        p = protogen.random_babycuda(seed)
        bc = drf.drf_babycuda_infer(p.text)                    # typable by construction
        map_text = drf.drf_protocol_text(bc)
        hist = babycuda.run(p.text, p.nthreads, p.cells, p.params)
        got = oracle.check(map_text, p.nthreads, p.cells, p.params, 1)
        if hist["error"] is not None:
            assert got["status"] == hist["error"][0] and got["err_tid"] == hist["error"][1]
            continue
        if len(set(hist["syncs"].values())) > 1:
            assert got["verdict"] == "BARRIER_DIVERGENCE"
            continue
        assert babycuda.access_set(hist) == _oracle_access_set(oracle, map_text, p), p.text
        drf_hist = babycuda.history_drf(hist)
        assert drf_hist == (got["verdict"] == "DRF"), p.text
        checked += 1
        racy += not drf_hist
    assert checked > 300 and racy > 50


def test_ill_typed_random_programs_are_rejected():
    for seed in range(200):
        p = protogen.random_babycuda(seed, ill_typed=True)
        with pytest.raises(drf.DrfError) as e:
            drf.drf_babycuda_infer(p.text)
        assert e.value.name == "UNBOUND_VAR"


@pytest.mark.gpu
def test_theorem1_verdicts_on_the_gpu():
    """The GPU checker's verdict on the inferred MAP equals Definition 1 on
    the BabyCUDA history."""
    ctx = drf.drf_ctx_create(0)
    try:
        n = 0
        for seed in range(300):
            p = protogen.random_babycuda(seed)
            hist = babycuda.run(p.text, p.nthreads, p.cells, p.params)
            if hist["error"] is not None or len(set(hist["syncs"].values())) > 1:
                continue
            bc = drf.drf_babycuda_infer(p.text)
            r = drf.result_dict(drf.drf_check(ctx, bc, p.nthreads, p.cells, p.params))
            assert (r["verdict"] == "DRF") == babycuda.history_drf(hist), p.text
            n += 1
        assert n > 150
    finally:
        drf.drf_ctx_destroy(ctx)
