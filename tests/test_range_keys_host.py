"""The sort path's range keys as planned on the host, against the oracle.

A range access (index sigma * tid + c, c a function of the loop variables)
is planned as pieces, and on the sort path each piece's keys are written as
k0 + o * d for its threads o.  Definition 1 decides a cell from the set of
(thread, mode) pairs that reach it, so a key stream is correct when the set
of (phase, array, index, tid, mode) its keys decode to is the protocol's set
of accesses (repeats of one access collapse to one key).  Expanding the
templates the packer writes must therefore give exactly the oracle's access
set when every access of the protocol is a range access, and a subset of it
otherwise.  Host only: a helper compiled against the library packs the
protocol; no GPU is involved.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2203_12878_b300 import drf, protogen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2203_12878_b300")
HELPER_SRC = os.path.join(ROOT, "tests", "helpers", "range_keys_dump.cpp")


@pytest.fixture(scope="module")
def helper(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    lib = os.path.join(PKG, "libdrfcheck.so")
    if not os.path.exists(lib):
        from paper_2203_12878_b300 import build
        build.build()
    exe = str(tmp_path_factory.mktemp("rkd") / "range_keys_dump")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    subprocess.run(["g++", "-std=c++17", "-O2", "-I", os.path.join(PKG, "csrc"), "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(cuda, "include"), HELPER_SRC, "-L", PKG, "-ldrfcheck",
                    f"-Wl,-rpath,{PKG}", "-L", os.path.join(cuda, "lib64"), "-lcudart", "-o", exe], check=True)
    return exe


def planned_keys(helper, tmp_path, p):
    """(layout, access instructions, range instructions, decoded keys as an
    (n, 5) array of phase, array, index, tid, mode)."""
    bc = drf.drf_protocol_compile(p.text)
    out = tmp_path / "keys.bin"
    subprocess.run([helper, str(out), str(p.nthreads), bytes(bc).hex(), *map(str, p.cells)], check=True)
    raw = np.fromfile(out, dtype=np.uint64)
    pb, phb, lb, ib, tb, acc, racc, rtuples, n = (int(x) for x in raw[:9])
    keys = raw[9:]
    assert len(keys) == n
    planned_keys.range_tuples = rtuples
    one = np.uint64(1)
    field = keys >> np.uint64(tb + 1)
    rows = np.stack([
        (field >> np.uint64(ib + lb)) & np.uint64((1 << phb) - 1) if phb else np.zeros_like(keys),
        (field >> np.uint64(ib)) & np.uint64((1 << lb) - 1) if lb else np.zeros_like(keys),
        field & np.uint64((1 << ib) - 1),
        (keys >> one) & np.uint64((1 << tb) - 1) if tb else np.zeros_like(keys),
        keys & one,
    ], axis=1)
    assert pb == 0 or not np.any(field >> np.uint64(ib + lb + phb)), "one protocol: the protocol field is 0"
    return acc, racc, rows


def as_set(rows):
    return set(map(tuple, np.unique(rows, axis=0).tolist()))


def config3_small(nthreads, racy):
    p = protogen.config3(0, racy=racy)
    return protogen.Protocol(p.text, nthreads, p.cells, p.params)


@pytest.mark.parametrize("nthreads", [256, 300])
def test_grid_protocol_range_keys_are_its_accesses(helper, tmp_path, oracle, nthreads):
    """Every access of the race-free grid-scale protocol (restricted to its
    first threads) is a range access, so the planned keys decode to exactly
    its access set, with fewer keys than tuples (repeated offsets)."""
    p = config3_small(nthreads, racy=False)
    acc, racc, rows = planned_keys(helper, tmp_path, p)
    assert acc == racc > 0
    want = oracle.tuples(p.text, p.nthreads, p.cells, p.params)
    assert as_set(rows) == as_set(want)
    assert len(rows) < len(want)
    # the host's count of the range accesses' tuples is every tuple here
    assert planned_keys.range_tuples == len(want)


def test_grid_protocol_planted_write_stays_with_the_interpreter(helper, tmp_path, oracle):
    """The racy variant adds one conditional write (two threads): the range
    keys are every other access, and the two writes are left out."""
    p = config3_small(256, racy=True)
    acc, racc, rows = planned_keys(helper, tmp_path, p)
    assert racc == acc - 1
    want = as_set(oracle.tuples(p.text, p.nthreads, p.cells, p.params))
    got = as_set(rows)
    missing = want - got
    assert got <= want and len(missing) <= 2
    assert all(m[4] == 1 for m in missing)


@pytest.mark.parametrize("text,T,cells", [
    # indices that wrap around their modulus several times over the threads
    ("array A;\nforU x in 0 .. 5 { rd A[(6 * tid + x) % 4096]; }\nwr A[(7 * tid + 3) % 4096];\n", 853, [4096]),
    ("array A;\nforU x in 0 .. 4 { rd A[(-5 * tid + 2 * x) % 1000]; }\nsync;\nwr A[(-3 * tid + 1) % 1000];\n",
     700, [1000]),
    ("array A;\nwr A[(4 * tid) % 1000];\n", 600, [1000]),
    ("array A, B;\nforU x in 0 .. 3 { wr B[(9 * tid + 1000 * x) % 3001]; rd A[(2 * tid) % 999]; }\n", 2000,
     [999, 3001]),
    # tid-free accesses: one key per thread at one record
    ("array A;\nforU x in 0 .. 9 { rd A[(x * 7) % 5]; }\n", 300, [5]),
    # negative steps and a loop over the offsets
    ("array A, B;\nforU x in 0 .. 6 { rd A[x]; wr B[tid + 64 * x]; }\nwr A[5];\n", 64, [8, 512]),
])
def test_wrapping_and_tid_free_range_keys(helper, tmp_path, oracle, text, T, cells):
    p = protogen.Protocol(text, T, cells, [])
    acc, racc, rows = planned_keys(helper, tmp_path, p)
    assert racc > 0
    ref = oracle.tuples(p.text, p.nthreads, p.cells, p.params)
    want = as_set(ref)
    got = as_set(rows)
    if acc == racc:
        assert got == want
        assert planned_keys.range_tuples == len(ref)
    else:
        assert got <= want and got


@pytest.mark.parametrize("seed", range(12))
def test_strided_range_keys_are_accesses(helper, tmp_path, oracle, seed):
    """Strides 2..8 (both signs), mixed with accesses the range pass leaves
    to the interpreter: every planned key is one of the protocol's
    accesses, and all of them when every access is a range access."""
    p = protogen.strided_small(seed)
    acc, racc, rows = planned_keys(helper, tmp_path, p)
    ref = oracle.tuples(p.text, p.nthreads, p.cells, p.params)
    want = as_set(ref)
    got = as_set(rows)
    if racc == 0:
        assert not got
    elif acc == racc:
        assert got == want
        assert planned_keys.range_tuples == len(ref)
    else:
        assert got <= want and got


# ---------------------------------------------------------------------------
# The range pass's merged pieces, applied on the host with the owner-record
# rule, against Definition 1 on the oracle's accesses.

K_SAT, K_WRITE, K_LEN = 1 << 31, 1 << 30, (1 << 30) - 1


def planned_pieces(helper, tmp_path, p):
    bc = drf.drf_protocol_compile(p.text)
    out = tmp_path / "pieces.bin"
    subprocess.run([helper, "--pieces", str(out), str(p.nthreads), bytes(bc).hex(), *map(str, p.cells)], check=True)
    raw = np.fromfile(out, dtype=np.uint8)
    hdr = raw[:72].view(np.uint64)
    recs, tab_off, cells_sum, tab_phases, nlocs, ntask, npiece, acc, racc = (int(x) for x in hdr)
    off = 72
    cbase = raw[off:off + 8 * nlocs].view(np.uint64).astype(np.int64)
    off += 8 * nlocs
    tasks = raw[off:off + 16 * ntask].view(np.uint32).reshape(ntask, 4).astype(np.int64)
    off += 16 * ntask
    pw = raw[off:off + 16 * npiece].view(np.uint32).reshape(npiece, 4)
    pieces = np.stack([pw[:, 0].astype(np.int64), pw[:, 1].astype(np.int64),
                       pw[:, 2].view(np.int32).astype(np.int64), pw[:, 3].view(np.int32).astype(np.int64)], axis=1)
    layout = dict(recs=recs, tab_off=tab_off, cells_sum=cells_sum, tab_phases=tab_phases, cbase=cbase)
    return layout, tasks, pieces, acc, racc


def apply_pieces(layout, tasks, pieces, nthreads):
    """Every record update the parts make: (record, tid or -1 for a
    saturating piece, writes).  Also checks that each task's parts cover its
    256-record blocks once."""
    recs = layout["recs"]
    total = layout["tab_off"] + layout["tab_phases"] * layout["cells_sum"]
    cover = {}
    rec_l, tid_l, w_l = [], [], []
    for task, p0, p1, win in tasks:
        blo, bhi = win & 0xFFFF, win >> 16
        cover.setdefault(task, []).append((blo, bhi))
        lo, hi = blo * 256, bhi * 256
        for t0, lenf, l0, step in pieces[p0:p1]:
            n = lenf & K_LEN
            o = np.arange(n, dtype=np.int64)
            r = l0 + step * o
            keep = (r >= lo) & (r < hi)
            assert np.all((r >= 0) & (r < recs)), "a piece leaves its task"
            rec_l.append(task * recs + r[keep])
            if lenf & K_SAT:
                tid_l.append(np.full(int(keep.sum()), -1, dtype=np.int64))
            else:
                assert step != 0, "merged pieces never step by 0"
                tid = t0 + o[keep]
                assert np.all(tid < nthreads)
                tid_l.append(tid)
            w_l.append(np.full(int(keep.sum()), 1 if lenf & K_WRITE else 0, dtype=np.int64))
    for task, parts in cover.items():
        nblk = -(-min(recs, total - task * recs) // 256)
        blocks = sorted(b for lo, hi in parts for b in range(lo, hi))
        assert blocks == list(range(nblk)), f"task {task}: parts {parts} do not cover its {nblk} blocks once"
    return np.concatenate(rec_l), np.concatenate(tid_l), np.concatenate(w_l)


def racy_records(rec, tid, w):
    """Owner records after the updates: "second thread" when a saturating
    piece reaches the record or two distinct tids do, "written" when any
    update writes; racy when both."""
    recs = np.unique(rec)
    idx = np.searchsorted(recs, rec)
    sat = np.zeros(len(recs), dtype=bool)
    np.logical_or.at(sat, idx, tid < 0)
    written = np.zeros(len(recs), dtype=bool)
    np.logical_or.at(written, idx, w > 0)
    pairs = np.unique(np.stack([rec[tid >= 0], tid[tid >= 0]], axis=1), axis=0)
    ntid = np.zeros(len(recs), dtype=np.int64)
    np.add.at(ntid, np.searchsorted(recs, pairs[:, 0]), 1)
    return recs, recs[(sat | (ntid >= 2)) & written]


def cells_of(layout, records):
    rel = records - layout["tab_off"]
    phase = rel // layout["cells_sum"]
    c = rel - phase * layout["cells_sum"]
    loc = np.searchsorted(layout["cbase"], c, side="right") - 1
    return set(zip(phase.tolist(), loc.tolist(), (c - layout["cbase"][loc]).tolist()))


def oracle_cells(oracle, p):
    """(accessed cells, racy cells by Definition 1: a write and two distinct
    threads)."""
    t = oracle.tuples(p.text, p.nthreads, p.cells, p.params).astype(np.int64)
    cell = t[:, 0] * (1 << 42) + t[:, 1] * (1 << 40) + t[:, 2]
    cells, inv = np.unique(cell, return_inverse=True)
    written = np.zeros(len(cells), dtype=bool)
    np.logical_or.at(written, inv, t[:, 4] == 1)
    ct = np.unique(np.stack([inv, t[:, 3]], axis=1), axis=0)
    ntid = np.bincount(ct[:, 0], minlength=len(cells))
    dec = lambda v: set(zip((v >> 42).tolist(), ((v >> 40) & 3).tolist(), (v & ((1 << 40) - 1)).tolist()))
    return dec(cells), dec(cells[written & (ntid >= 2)])


RANGE_ONLY = [
    ("array A;\nforU x in 0 .. 5 { rd A[(6 * tid + x) % 4096]; }\nwr A[(7 * tid + 3) % 4096];\n", 853, [4096]),
    ("array A;\nforU x in 0 .. 4 { rd A[(-5 * tid + 2 * x) % 1000]; }\nsync;\nwr A[(-3 * tid + 1) % 1000];\n",
     700, [1000]),
    ("array A;\nwr A[(4 * tid) % 1000];\n", 600, [1000]),
    ("array A, B;\nforU x in 0 .. 3 { wr B[(9 * tid + 1000 * x) % 3001]; rd A[(2 * tid) % 999]; }\n", 2000,
     [999, 3001]),
    # tid-free: every thread reads five cells, then writes one (saturated pieces)
    ("array A;\nforU x in 0 .. 9 { rd A[(x * 7) % 5]; }\nsync;\nwr A[2];\n", 300, [5]),
]


@pytest.mark.parametrize("case", range(len(RANGE_ONLY) + 2))
def test_merged_pieces_mark_the_racy_cells(helper, tmp_path, oracle, case):
    """The merged pieces reach exactly the protocol's cells, and the owner
    records they leave are racy exactly at Definition 1's racy cells
    (saturated pieces standing for two or more threads included)."""
    if case < len(RANGE_ONLY):
        text, T, cells = RANGE_ONLY[case]
        p = protogen.Protocol(text, T, cells, [])
    else:
        p = config3_small(256 if case == len(RANGE_ONLY) else 300, racy=False)
    layout, tasks, pieces, acc, racc = planned_pieces(helper, tmp_path, p)
    assert acc == racc > 0 and len(tasks) and len(pieces)
    rec, tid, w = apply_pieces(layout, tasks, pieces, p.nthreads)
    touched, racy = racy_records(rec, tid, w)
    want_cells, want_racy = oracle_cells(oracle, p)
    assert cells_of(layout, touched) == want_cells
    assert cells_of(layout, racy) == want_racy


@pytest.mark.parametrize("seed", range(12))
def test_strided_merged_pieces_mark_the_racy_cells(helper, tmp_path, oracle, seed):
    """The same on strided protocols (steps 2..8 of both signs, pieces that
    interleave in one task's records)."""
    p = protogen.strided_small(seed)
    layout, tasks, pieces, acc, racc = planned_pieces(helper, tmp_path, p)
    assert acc == racc > 0
    rec, tid, w = apply_pieces(layout, tasks, pieces, p.nthreads)
    touched, racy = racy_records(rec, tid, w)
    want_cells, want_racy = oracle_cells(oracle, p)
    assert cells_of(layout, touched) == want_cells
    assert cells_of(layout, racy) == want_racy


def test_split_task_parts_cover_it_once(helper, tmp_path, oracle):
    """Steps 1, 2, 3 and 4 (pieces that never merge) give the first task more
    than 2^15 record updates, so it is split into parts over disjoint windows
    of its records; together the parts apply every piece once."""
    text = "array A;\nrd A[tid];\nrd A[2 * tid];\nrd A[3 * tid];\nwr A[4 * tid];\nrd A[65535 - tid];\n"
    p = protogen.Protocol(text, 16384, [65536], [])
    layout, tasks, pieces, acc, racc = planned_pieces(helper, tmp_path, p)
    assert acc == racc == 5
    assert len(tasks) > len(set(tasks[:, 0].tolist())), "no task was split"
    rec, tid, w = apply_pieces(layout, tasks, pieces, p.nthreads)
    touched, racy = racy_records(rec, tid, w)
    want_cells, want_racy = oracle_cells(oracle, p)
    assert cells_of(layout, touched) == want_cells
    assert cells_of(layout, racy) == want_racy and want_racy
