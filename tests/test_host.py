"""Host-side tests of the C-ABI library (no GPU needed): it loads and exports
every entry point the header declares, its front-end accepts and rejects the
same protocols as the oracle's independent parser, its bytecode decoder
survives malformed input, and its interval analysis is sound against the
oracle's exact counts."""
import os
import random
import re

import pytest

from paper_2203_12878_b300 import drf, protogen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "drf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(drf_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    lib = drf.lib()
    declared = _header_functions()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(drf.EXPORTED)
    assert drf.drf_version() == 1
    assert drf.drf_status_string(-9) == "DRF_E_INDEX_OOB"


def test_context_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(drf.DrfError) as e:
        drf.drf_ctx_create(0)
    assert e.value.name == "CUDA"


def _compile_status(text):
    try:
        drf.drf_protocol_compile(text)
        return "OK"
    except drf.DrfError as e:
        return e.name


INVALID = [
    "array A;\nforU x in 0 .. 4 { sync; }\n",
    "array A;\nif (tid = 0) { sync; }\n",
    "array A;\nforU x in 0 .. 4 { forS y in 0 .. 2 { rd A[0]; } }\n",
    "array A;\nforU x in 0 .. 4 { forU x in 0 .. 2 { rd A[x]; } }\n",
    "array A;\nparam M;\nforU M in 0 .. 4 { rd A[0]; }\n",
    "array A, A;\nrd A[0];\n",
    "array A;\nrd B[0];\n",
    "array A;\nrd A[y];\n",
    "array A;\nforU x in 0 .. x { rd A[0]; }\n",
    "array A;\nforU x in 0 .. 3 { rd A[x]; }\nrd A[x];\n",
    "array A;\nrd A[0]\n",
    "array A;\nrd A[99999999999999999999];\n",
    "array A;\nforU x in 0 : 3 { rd A[0]; }\n",
    "array A;\nif (tid) { rd A[0]; }\n",
    "array A;\nrd A[tid < 3];\n",
    "array A;\nif (1 < 2 < 3) { rd A[0]; }\n",
    "array A;\nrd A[tid & 1];\n",
    "array A;\nwr A[tid];\nrd A[tid];\nwr A[x];\n",
    "array A;\nif ((tid < 3) + 1 > 2) { rd A[0]; }\n",
    "array A;\nrd A[min(tid)];\n",
    "array A; sync; array B;\n",
    "array tid;\n",
    "forU x in 0 .. 2 { skip; }\nrd A[0];\n",
]
VALID = [
    "array A;\nforS x in 0 .. 2 { sync; rd A[x]; }\nforS y in 0 .. 2 { forS z in 0 .. y { sync; } }\n",
    "array A;\nif (!tid < 3 && tid != 1 || tid = 7) { rd A[0]; } else { wr A[1]; }\n",
    "array A;\nif ((tid < 3)) { rd A[-(-2)]; }\n",
    "array A;\nrd A[((tid))];\n",
    "# comment\narray A; // another\nparam M, N;\nforU x in M .. N { rd A[x % 4]; }\n",
    "array A;\nif (!(tid < 3)) { skip; }\n",
    "",
]


@pytest.mark.parametrize("text", INVALID + VALID)
def test_front_end_agrees_with_oracle(oracle, text):
    assert _compile_status(text) == oracle.validate(text)[0]


def test_front_end_agrees_on_random_protocols(oracle):
    for seed in range(1500):
        p = protogen.random_small(seed)
        assert _compile_status(p.text) == oracle.validate(p.text)[0] == "OK"
        bc = drf.drf_protocol_compile(p.text)
        assert drf.drf_protocol_info(bc) == (len(p.cells), len(p.params))


def test_bytecode_decoder_survives_corruption():
    p = protogen.config1()
    bc = bytearray(drf.drf_protocol_compile(p.text))
    r = random.Random(5)
    seen = set()
    for trial in range(3000):
        b = bytearray(bc)
        kind = trial % 3
        if kind == 0:
            b = b[:r.randrange(len(b))]
        elif kind == 1:
            for _ in range(r.randint(1, 4)):
                b[r.randrange(len(b))] = r.randrange(256)
        else:
            b += bytes(r.randrange(256) for _ in range(r.randint(1, 8)))
        try:
            drf.drf_protocol_info(bytes(b))
            st = "OK"
        except drf.DrfError as e:
            st = e.name
        seen.add(st)
        st2, _ = drf.drf_protocol_analyze(bytes(b), 4, [64])
        assert st2 in ("OK", "INVALID_BYTECODE", "UNBOUND_VAR", "UNKNOWN_ARRAY", "REBIND", "SYNC_IN_UNSYNC",
                       "LIMIT", "INVALID_ARG", "OVERFLOW_RISK")
    assert "INVALID_BYTECODE" in seen


def test_bounds_validation():
    bc = drf.drf_protocol_compile("array A, B;\nparam M;\nrd A[M];\n")
    assert drf.drf_protocol_analyze(bc, 4, [8, 8], [1])[0] == "OK"
    assert drf.drf_protocol_analyze(bc, 4, [8], [1])[0] == "INVALID_ARG"
    assert drf.drf_protocol_analyze(bc, 4, [8, 8], [])[0] == "INVALID_ARG"


@pytest.mark.parametrize("text,status", [
    ("array A;\nrd A[(9223372036854775807 + tid) % 8];\n", "OVERFLOW_RISK"),
    ("array A;\nrd A[(tid * 4611686018427387904 * 4) % 8];\n", "OVERFLOW_RISK"),
    ("array A;\nforU x in 0 .. 4 { rd A[(x - 9223372036854775807 - 2) % 8]; }\n", "OVERFLOW_RISK"),
    ("array A;\nrd A[(-9223372036854775807 - 1) / (tid - 1) % 8];\n", "OVERFLOW_RISK"),
    ("array A;\nrd A[(9223372036854775806 + tid) % 8];\n", "OK"),
    ("array A;\nforU x in 0 .. 0 { rd A[x * 9223372036854775807 * 9]; }\n", "OK"),     # never runs
    ("array A;\nforU x in 0 .. 100000000000 { forU y in 0 .. 100000000000 { rd A[0]; } }\n", "LIMIT"),
])
def test_interval_analysis_rejections(text, status):
    bc = drf.drf_protocol_compile(text)
    assert drf.drf_protocol_analyze(bc, 2, [8])[0] == status


def test_arithmetic_width_choice():
    small = drf.drf_protocol_compile("array A;\nforU x in 0 .. 100 { rd A[(tid * 1000 + x) % 64]; }\n")
    assert drf.drf_protocol_analyze(small, 1024, [64])[1]["wide_arithmetic"] == 0
    big = drf.drf_protocol_compile("array A;\nforU x in 0 .. 100 { rd A[(tid * 100000000 + x) % 64]; }\n")
    assert drf.drf_protocol_analyze(big, 1024, [64])[1]["wide_arithmetic"] == 1


def test_static_bounds_cover_the_oracle(oracle):
    """The analysis' tuple and sync bounds are upper bounds of what the
    protocol really does (interval analysis is sound)."""
    n = 0
    for seed in range(800):
        p = protogen.random_small(seed)
        got = oracle.check(p.text, p.nthreads, p.cells, p.params, 2)
        st, a = drf.drf_protocol_analyze(drf.drf_protocol_compile(p.text), p.nthreads, p.cells, p.params)
        if st != "OK" or got["status"] != "OK":
            continue
        n += 1
        assert a["tuple_bound"] >= got["tuples"], p.text
        if got.get("phases"):
            assert a["sync_bound"] >= got["phases"] - 1
        assert a["items"] >= 1
    assert n > 500


def test_key_layout_for_workloads():
    p = protogen.config1()
    st, a = drf.drf_protocol_analyze(drf.drf_protocol_compile(p.text), 256, p.cells)
    # 9 phases -> 4 bits, one array -> 0, 2048 cells -> 11 bits; tid 8 bits + mode
    assert (st, a["sort_bits"], a["key_bits"], a["tuple_bound"], a["sync_bound"]) == ("OK", 15, 24, 4096, 8)
    p = protogen.config3(0)
    st, a = drf.drf_protocol_analyze(drf.drf_protocol_compile(p.text), p.nthreads, p.cells)
    assert st == "OK" and a["key_bits"] <= 64 and a["tuple_bound"] == p.meta["accesses"]


def test_work_items_follow_protocol_size():
    """A lone check cuts a small protocol into short items, so that its
    threads' chains of dependent steps spread over about a wave of warps
    (config 1: one item per iteration of its forS loop), and a large one into
    items of at least 64 interpreter steps (config 2: 354 items)."""
    def items(p):
        st, a = drf.drf_protocol_analyze(drf.drf_protocol_compile(p.text), p.nthreads, p.cells, p.params)
        assert st == "OK"
        return a["items"]
    assert items(protogen.config1("drf")) == 8
    assert items(protogen.config2(0)) == 354
    # a protocol of a handful of steps per thread is not cut below 4 steps per item
    assert items(protogen.Protocol("array A;\nwr A[tid];\nrd A[tid];\n", 32, [32], [])) == 1
