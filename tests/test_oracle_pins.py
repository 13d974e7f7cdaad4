"""Pins for the oracle: it is checked against things other than itself --
the paper's worked examples, closed forms from elementary number theory,
the semantics readings spelled out on literal cases, invariants that any
correct race checker satisfies, and agreement between its two independent
checkers (every thread pair vs. per-cell records) on thousands of tiny
random protocols."""
import json
import math
import os
import random
import re

import pytest

from paper_2203_12878_b300 import protogen

HERE = os.path.dirname(os.path.abspath(__file__))
PAIRS, CELLS, EVAL = 0, 1, 2


def _golden():
    with open(os.path.join(HERE, "golden", "paper_examples.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
@pytest.mark.parametrize("method", [PAIRS, CELLS])
def test_paper_examples(oracle, case, method):
    got = oracle.check(case["text"], case["nthreads"], case["cells"], case["params"], method)
    for k, v in case["expect"].items():
        assert got[k] == v, (case["name"], k, got)


# ---------------------------------------------------------- closed forms --

@pytest.mark.parametrize("T", [1, 2, 6, 8, 12, 16, 30])
@pytest.mark.parametrize("a", [-4, -1, 0, 1, 2, 3, 5, 6])
@pytest.mark.parametrize("b", [-7, 0, 5])
def test_affine_map_closed_form(oracle, T, a, b):
    """wr A[(a*tid + b) mod T]: injective (DRF) iff gcd(a, T) = 1.  Otherwise
    every image cell has g = gcd(a, T) preimages spaced T/g apart; the
    smallest image cell is b mod g and its two smallest preimages race."""
    text = f"array A;\nwr A[(({a}) * tid + ({b})) % {T}];\n"
    got = oracle.check(text, T, [T], [], PAIRS)
    g = math.gcd(a, T)
    if T == 1 or g == 1:
        assert got["verdict"] == "DRF"
        return
    c0 = b % g                     # smallest cell of the image
    m = T // g
    # a*t = c0 - b (mod T)  <=>  (a/g)*t = (c0-b)/g (mod T/g)
    t0 = ((c0 - b) // g) * pow((a // g) % m, -1, m) % m if m > 1 else 0
    assert got["verdict"] == "RACY"
    assert (got["phase"], got["loc"], got["index"]) == (0, 0, c0)
    assert (got["tid_i"], got["tid_j"]) == (t0, t0 + m)
    assert got["i_writes"] and got["j_writes"]
    assert oracle.check(text, T, [T], [], CELLS) == got


@pytest.mark.parametrize("lo,hi", [(0, 0), (0, 5), (3, 7), (7, 3), (-2, 2), (5, 6)])
@pytest.mark.parametrize("T", [1, 3, 8])
def test_loop_range_counts(oracle, lo, hi, T):
    """Rules for-1 / for-2: lo..hi runs x = lo, ..., hi-1 (none if lo >= hi)."""
    text = f"array A;\nforU x in {lo} .. {hi} {{ rd A[0]; }}\n"
    got = oracle.check(text, T, [1], [], CELLS)
    assert got["tuples"] == T * max(0, hi - lo)
    assert got["verdict"] == "DRF"       # reads only


def test_loop_variable_values(oracle):
    """x takes exactly the values lo..hi-1: one write per value by thread 0 and
    a read of a single cell v by thread 1 races iff v is in the range."""
    for v in range(-1, 9):
        text = ("array A;\n"
                "if (tid = 0) { forU x in 2 .. 6 { wr A[x]; } } else { rd A[" + str(v) + "]; }\n")
        got = oracle.check(text, 2, [16], [], PAIRS) if v >= 0 else None
        if v < 0:
            continue
        if 2 <= v < 6:
            assert got["verdict"] == "RACY" and got["index"] == v
        else:
            assert got["verdict"] == "DRF"


def _euclid_mod(a, b):
    r = abs(a) % abs(b)
    return r if a >= 0 or r == 0 else abs(b) - r


@pytest.mark.parametrize("a", [-9, -7, -1, 0, 1, 7, 9])
@pytest.mark.parametrize("b", [-4, -3, 3, 4])
def test_division_and_remainder(oracle, a, b):
    """'/' is floor division and '%' the Euclidean remainder (in [0, |b|)).
    Two threads write the same cell, so the witness index reveals the value."""
    n = 64
    q = math.floor(a / b)
    r = _euclid_mod(a, b)
    for expr, want in ((f"({a}) / ({b}) + 32", q + 32), (f"({a}) % ({b})", r)):
        got = oracle.check(f"array A;\nwr A[{expr}];\n", 2, [n], [], CELLS)
        assert got["verdict"] == "RACY" and got["index"] == want, (expr, got)


def test_min_max_and_conditions(oracle):
    cases = [("min(7, 3)", 3), ("max(7, 3)", 7), ("min(-2, 5) + 4", 2), ("max(2 * 3, 5 - 1)", 6),
             ("2 + 3 * 4", 14), ("(2 + 3) * 4", 20), ("10 - 3 - 2", 5), ("-3 + 10", 7),
             ("20 / 3 / 2", 3), ("- (2 - 9)", 7)]
    for expr, want in cases:
        got = oracle.check(f"array A;\nwr A[{expr}];\n", 2, [64], [], CELLS)
        assert got["index"] == want, expr
    # conditions: thread t writes iff the condition holds for t
    conds = {"tid < 2": {0, 1}, "tid >= 2 && tid != 3": {2}, "!(tid = 1) && tid <= 2": {0, 2},
             "tid = 0 || tid = 3": {0, 3}, "(tid + 1) * 2 > 6": {3}, "true": {0, 1, 2, 3},
             "false": set(), "((tid < 1)) || (tid > 2)": {0, 3}}
    for c, writers in conds.items():
        got = oracle.check(f"array A;\nif ({c}) {{ wr A[0]; }}\n", 4, [1], [], PAIRS)
        assert got["tuples"] == len(writers), c
        if len(writers) >= 2:
            w = sorted(writers)
            assert got["verdict"] == "RACY" and (got["tid_i"], got["tid_j"]) == (w[0], w[1]), c
        else:
            assert got["verdict"] == "DRF", c


def test_phases_and_barrier_divergence(oracle):
    for k in range(0, 5):
        got = oracle.check(f"array A;\nforS x in 0 .. {k} {{ sync; }}\n", 3, [1], [], CELLS)
        assert got["verdict"] == "DRF" and got["phases"] == k + 1
    # a loop whose trip count depends on tid: thread t syncs t times
    got = oracle.check("array A;\nforS x in 0 .. tid { sync; }\n", 4, [1], [], CELLS)
    assert got["verdict"] == "BARRIER_DIVERGENCE"
    assert (got["div_tid"], got["sync_count_0"], got["sync_count_div"]) == (1, 0, 1)
    got = oracle.check("array A;\nforS x in 0 .. min(tid, 2) + 5 * (tid / 3) { sync; }\n", 8, [1], [], CELLS)
    assert (got["div_tid"], got["sync_count_0"], got["sync_count_div"]) == (1, 0, 1)
    got = oracle.check("array A;\nforS x in 0 .. 2 - tid / 5 { sync; }\n", 8, [1], [], CELLS)
    assert (got["div_tid"], got["sync_count_0"], got["sync_count_div"]) == (5, 2, 1)
    # divergence wins over a race; a race in phase 0 does not hide it
    got = oracle.check("array A;\nwr A[0];\nforS x in 0 .. tid { sync; }\n", 2, [1], [], PAIRS)
    assert got["verdict"] == "BARRIER_DIVERGENCE"
    # a sync splits write-write on one cell into two phases
    assert oracle.check("array A;\nif (tid = 0) { wr A[0]; }\nsync;\nif (tid = 1) { wr A[0]; }\n",
                        2, [1], [], PAIRS)["verdict"] == "DRF"
    assert oracle.check("array A;\nif (tid = 0) { wr A[0]; }\nif (tid = 1) { wr A[0]; }\n",
                        2, [1], [], PAIRS)["verdict"] == "RACY"


def test_synchronized_loop_phase_carry(oracle):
    """Accesses after the last sync of iteration x share a phase with the
    accesses before the first sync of iteration x+1 (a per-thread phase
    counter).  Thread 0 writes cell x after the sync of iteration x (phase
    x+1), thread 1 reads cell x-1 before the sync of iteration x (phase x):
    they first meet in phase 1 on cell 0; phase 0 only has thread 1 reading
    cell 15."""
    text = ("array A;\n"
            "forS x in 0 .. 4 {\n"
            "  if (tid = 1) { rd A[(x + 15) % 16]; }\n"
            "  sync;\n"
            "  if (tid = 0) { wr A[x]; }\n"
            "}\n")
    got = oracle.check(text, 2, [16], [], PAIRS)
    assert got["verdict"] == "RACY"
    assert (got["phase"], got["index"], got["tid_i"], got["tid_j"]) == (1, 0, 0, 1)
    assert got["i_writes"] and not got["j_writes"]


def test_evaluation_errors(oracle):
    got = oracle.check("array A;\nrd A[tid];\n", 3, [2], [], CELLS)
    assert (got["status"], got["err_tid"], got["err_ordinal"]) == ("INDEX_OOB", 2, 0)
    got = oracle.check("array A;\nrd A[0];\nrd A[tid - 1];\n", 3, [4], [], CELLS)
    assert (got["status"], got["err_tid"], got["err_ordinal"]) == ("INDEX_OOB", 0, 1)
    got = oracle.check("array A;\nforU x in 0 .. 3 { rd A[0]; }\nrd A[(7 / (tid - 2)) % 8];\n", 4, [8], [], CELLS)
    assert (got["status"], got["err_tid"], got["err_ordinal"]) == ("DIV_ZERO", 2, 3)
    got = oracle.check("array A;\nrd A[0];\nif (tid % (tid - 1) = 0) { rd A[0]; }\n", 4, [8], [], CELLS)
    assert (got["status"], got["err_tid"], got["err_ordinal"]) == ("DIV_ZERO", 1, 1)
    got = oracle.check("array A;\nforU x in 0 .. (9223372036854775807 + tid) * 0 { rd A[0]; }\n", 2, [8], [], EVAL)
    assert (got["status"], got["err_tid"], got["err_ordinal"]) == ("OVERFLOW", 1, 0)
    got = oracle.check("array A;\nrd A[(0 - 4611686018427387904 * (1 + tid)) % 8];\n", 2, [8], [], EVAL)
    assert (got["status"], got["err_tid"]) == ("OVERFLOW", 1)
    # an error wins over a race and over divergence; the smallest tid reports
    got = oracle.check("array A;\nwr A[0];\nforS x in 0 .. tid { sync; }\nrd A[3 - tid];\n", 5, [3], [], PAIRS)
    assert (got["status"], got["err_tid"], got["err_ordinal"]) == ("INDEX_OOB", 0, 1)


@pytest.mark.parametrize("text,status", [
    ("array A;\nforU x in 0 .. 4 { sync; }\n", "SYNC_IN_UNSYNC"),
    ("array A;\nif (tid = 0) { sync; }\n", "SYNC_IN_UNSYNC"),
    ("array A;\nforU x in 0 .. 4 { forS y in 0 .. 2 { rd A[0]; } }\n", "SYNC_IN_UNSYNC"),
    ("array A;\nforS x in 0 .. 4 { forU y in 0 .. 2 { sync; } }\n", "SYNC_IN_UNSYNC"),
    ("array A;\nforU x in 0 .. 4 { forU x in 0 .. 2 { rd A[x]; } }\n", "REBIND"),
    ("array A;\nparam M;\nforU M in 0 .. 4 { rd A[0]; }\n", "REBIND"),
    ("array A, A;\nrd A[0];\n", "REBIND"),
    ("array A;\nrd B[0];\n", "UNKNOWN_ARRAY"),
    ("array A;\nrd A[y];\n", "UNBOUND_VAR"),
    ("array A;\nforU x in 0 .. x { rd A[0]; }\n", "UNBOUND_VAR"),
    ("array A;\nforU x in 0 .. 3 { rd A[x]; }\nrd A[x];\n", "UNBOUND_VAR"),
    ("array A;\nrd A[0]\n", "PARSE"),
    ("array A;\nrd A[99999999999999999999];\n", "PARSE"),
    ("array A;\nforU x in 0 : 3 { rd A[0]; }\n", "PARSE"),
    ("array A;\nif (tid) { rd A[0]; }\n", "PARSE"),
    ("array A;\nforS x in 0 .. 2 { sync; rd A[x]; }\nforS y in 0 .. 2 { forS z in 0 .. y { sync; } }\n", "OK"),
])
def test_validation(oracle, text, status):
    assert oracle.validate(text)[0] == status


# ------------------------------------------------------------ invariants --

def _ok(d):
    return d["status"] == "OK"


def test_read_only_single_thread_and_duplication(oracle):
    for seed in range(400):
        p = protogen.random_small(seed)
        base = oracle.check(p.text, p.nthreads, p.cells, p.params, CELLS)
        if not _ok(base):
            continue
        ro = oracle.check(p.text.replace("wr ", "rd "), p.nthreads, p.cells, p.params, CELLS)
        if ro["verdict"] != "BARRIER_DIVERGENCE":
            assert ro["verdict"] == "DRF", p.text
        one = oracle.check(p.text, 1, p.cells, p.params, CELLS)
        if _ok(one):
            assert one["verdict"] == "DRF"
        # every access statement run twice: same sets, so same verdict and witness
        dup = oracle.check(_duplicate_accesses(p.text), p.nthreads, p.cells, p.params, CELLS)
        assert dup["tuples"] == 2 * base["tuples"]
        strip = lambda d: {k: v for k, v in d.items() if k != "tuples"}
        assert strip(dup) == strip(base), p.text


def _duplicate_accesses(text):
    """Every access statement written twice in a row (index expressions
    contain no brackets, so one regular expression finds them)."""
    return re.sub(r"\b(rd|wr) ([A-Z])\[([^\]]*)\];", lambda m: m.group(0) + " " + m.group(0), text)


def test_sync_prefix_shifts_phases(oracle):
    for seed in range(300):
        p = protogen.random_small(seed)
        base = oracle.check(p.text, p.nthreads, p.cells, p.params, CELLS)
        if not _ok(base):
            continue
        head, _, body = p.text.partition(";\n")
        lines = p.text.split("\n")
        decl = [l for l in lines if l.startswith(("array", "param"))]
        rest = [l for l in lines if not l.startswith(("array", "param"))]
        shifted = "\n".join(decl + ["sync;", "sync;"] + rest)
        got = oracle.check(shifted, p.nthreads, p.cells, p.params, CELLS)
        assert got["verdict"] == base["verdict"]
        if base["verdict"] == "RACY":
            assert got["phase"] == base["phase"] + 2
            assert {k: got[k] for k in ("loc", "index", "tid_i", "tid_j")} == \
                   {k: base[k] for k in ("loc", "index", "tid_i", "tid_j")}
        if p.nthreads:
            assert got["phases"] == base["phases"] + 2


def test_tid_permutation(oracle):
    """Renaming threads by a bijection t -> (a t + b) mod T keeps the verdict
    and the racing cell (Definition 1 only asks for two distinct ids)."""
    rng = random.Random(7)
    n = 0
    for seed in range(600):
        p = protogen.random_small(seed)
        T = p.nthreads
        base = oracle.check(p.text, T, p.cells, p.params, CELLS)
        if not _ok(base) or T < 2:
            continue
        a = rng.choice([x for x in range(1, 2 * T) if math.gcd(x, T) == 1])
        b = rng.randrange(T)
        perm = p.text.replace("tid", f"((({a}) * TID_ + {b}) % {T})").replace("TID_", "tid")
        got = oracle.check(perm, T, p.cells, p.params, CELLS)
        if not _ok(got):
            continue
        n += 1
        assert got["verdict"] == base["verdict"], (p.text, perm)
        if base["verdict"] == "RACY":
            assert (got["phase"], got["loc"], got["index"]) == (base["phase"], base["loc"], base["index"])
    assert n > 100


def test_range_split_and_constructed_race_free(oracle):
    text = "array A;\nforU x in 0 .. 10 { wr A[(3 * tid + 16 * x) % 64]; rd A[x % 4]; }\n"
    split = ("array A;\nforU x in 0 .. 4 { wr A[(3 * tid + 16 * x) % 64]; rd A[x % 4]; }\n"
             "forU x in 4 .. 10 { wr A[(3 * tid + 16 * x) % 64]; rd A[x % 4]; }\n")
    for T in (1, 2, 5, 16):
        assert oracle.check(text, T, [64], [], PAIRS) == oracle.check(split, T, [64], [], PAIRS)


@pytest.mark.parametrize("seed", range(6))
def test_planted_race_caught_exactly(oracle, seed):
    """A race-free-by-construction base (every cell owned by one thread) with
    one write planted by two threads: the witness is exactly the planted cell."""
    r = random.Random(seed)
    p = protogen.config4_one(r, racy=False)
    assert oracle.check(p.text, p.nthreads, p.cells, p.params, CELLS)["verdict"] == "DRF"
    q = protogen.config4_one(random.Random(1000 + seed), racy=True)
    got = oracle.check(q.text, q.nthreads, q.cells, q.params, CELLS)
    m = q.meta
    assert got["verdict"] == "RACY"
    assert (got["phase"], got["loc"], got["index"]) == (m["phase"], m["loc"], m["index"])
    assert got["tid_i"] <= m["threads"][0]


def test_config2_constructed_small(oracle):
    p = protogen.config2(5, mode="constructed", target=2e5, plant=False)
    assert oracle.check(p.text, p.nthreads, p.cells, p.params, CELLS)["verdict"] == "DRF"
    q = protogen.config2(5, mode="constructed", target=2e5, plant=True)
    got = oracle.check(q.text, q.nthreads, q.cells, q.params, CELLS)
    m = q.meta
    assert (got["verdict"], got["phase"], got["loc"], got["index"]) == ("RACY", m["phase"], m["loc"], m["index"])


# ----------------------------------------------- the two checkers agree --

def test_pairs_equal_cells_on_random_small(oracle):
    """Definition 1 over every thread pair and the per-cell records agree on
    every field (status, verdict, witness, flags, counts) for 3000 protocols."""
    kinds = {}
    for seed in range(3000):
        p = protogen.random_small(seed)
        a = oracle.check(p.text, p.nthreads, p.cells, p.params, PAIRS)
        b = oracle.check(p.text, p.nthreads, p.cells, p.params, CELLS)
        assert a == b, p.text
        kinds[a.get("verdict") or a["status"]] = kinds.get(a.get("verdict") or a["status"], 0) + 1
    # the sweep covers every outcome
    assert kinds.get("RACY", 0) > 300 and kinds.get("DRF", 0) > 300
    assert kinds.get("BARRIER_DIVERGENCE", 0) > 20 and kinds.get("INDEX_OOB", 0) > 20


def test_pairs_equal_cells_config1(oracle):
    for v in ("drf", "rdwr", "nosync"):
        p = protogen.config1(v)
        assert oracle.check(p.text, 256, p.cells, [], PAIRS) == oracle.check(p.text, 256, p.cells, [], CELLS)


def test_single_cell_helper_agrees_with_whole_check(oracle):
    """oracle.cell (accessors of one cell, one thread at a time) gives the
    same witness as the whole-protocol checkers on the witness cell."""
    n = 0
    for seed in range(400):
        p = protogen.random_small(seed)
        got = oracle.check(p.text, p.nthreads, p.cells, p.params, PAIRS)
        if got["status"] != "OK" or got["verdict"] != "RACY":
            continue
        c = oracle.cell(p.text, p.nthreads, p.cells, p.params, got["phase"], got["loc"], got["index"])
        assert c["racy"] and c["total"] == got["tuples"]
        assert {k: c[k] for k in ("tid_i", "tid_j", "i_writes", "j_writes")} == \
               {k: got[k] for k in ("tid_i", "tid_j", "i_writes", "j_writes")}
        n += 1
    assert n > 50


def test_strided_quiet_seeds_race_free(oracle):
    """Quiet strided_small seeds write only cells a * (tid + T * j), j < 6
    (distinct per thread and j), and read only other arrays: race-free by
    construction, as the oracle finds."""
    n = 0
    for s in range(40):
        p = protogen.strided_small(s)
        if not p.meta["quiet"]:
            continue
        n += 1
        assert oracle.check(p.text, p.nthreads, p.cells, p.params, CELLS)["verdict"] == "DRF", p.text
    assert n >= 10
