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
    pb, phb, lb, ib, tb, acc, racc, n = (int(x) for x in raw[:8])
    keys = raw[8:]
    assert len(keys) == n
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
    want = as_set(oracle.tuples(p.text, p.nthreads, p.cells, p.params))
    got = as_set(rows)
    if acc == racc:
        assert got == want
    else:
        assert got <= want and got


@pytest.mark.parametrize("seed", range(12))
def test_strided_range_keys_are_accesses(helper, tmp_path, oracle, seed):
    """Strides 2..8 (both signs), mixed with accesses the range pass leaves
    to the interpreter: every planned key is one of the protocol's
    accesses, and all of them when every access is a range access."""
    p = protogen.strided_small(seed)
    acc, racc, rows = planned_keys(helper, tmp_path, p)
    want = as_set(oracle.tuples(p.text, p.nthreads, p.cells, p.params))
    got = as_set(rows)
    if racc == 0:
        assert not got
    elif acc == racc:
        assert got == want
    else:
        assert got <= want and got
