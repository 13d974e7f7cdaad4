"""ctypes wrapper around the C oracle (``drf_oracle.c``).

Test infrastructure only: imported by the tests, by ``__graft_entry__.smoke``
and by the benchmark's CPU-baseline leg.  The product library never imports
it, and it imports nothing from the product package.

The oracle interprets protocol *text* with its own parser; see the header of
``drf_oracle.c`` for what it computes and which passage of the paper each
step follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "drf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS_NAMES = {
    0: "OK", -1: "INVALID_ARG", -2: "PARSE", -4: "UNBOUND_VAR", -5: "UNKNOWN_ARRAY",
    -6: "REBIND", -7: "SYNC_IN_UNSYNC", -8: "OVERFLOW", -9: "INDEX_OOB",
    -10: "DIV_ZERO", -12: "NOMEM",
}
VERDICTS = {-1: None, 0: "DRF", 1: "RACY", 2: "BARRIER_DIVERGENCE"}

METHOD_PAIRS = 0   # Definition 1 literally: every ordered pair of distinct threads
METHOD_CELLS = 1   # per-cell owner records
METHOD_EVAL = 2    # evaluation only (status, tuples, syncs)


class _Result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("verdict", ctypes.c_int32),
        ("phase", ctypes.c_uint32), ("loc", ctypes.c_uint32),
        ("index", ctypes.c_uint64),
        ("tid_i", ctypes.c_uint32), ("tid_j", ctypes.c_uint32),
        ("i_writes", ctypes.c_uint32), ("j_writes", ctypes.c_uint32),
        ("div_tid", ctypes.c_uint32), ("sync_count_0", ctypes.c_uint32),
        ("sync_count_div", ctypes.c_uint32), ("phases", ctypes.c_uint32),
        ("tuples", ctypes.c_uint64),
        ("err_tid", ctypes.c_uint32), ("pad0", ctypes.c_uint32),
        ("err_ordinal", ctypes.c_uint64),
    ]


class _Cell(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_uint32), ("t1", ctypes.c_uint32), ("w0", ctypes.c_uint32), ("w1", ctypes.c_uint32),
                ("cell_accesses", ctypes.c_uint64), ("total", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("pad", ctypes.c_uint32)]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (plain gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-Wall", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_check.restype = ctypes.c_int
            lib.oracle_check.argtypes = [
                ctypes.c_char_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                ctypes.c_uint32, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                ctypes.POINTER(_Result), ctypes.c_char_p, ctypes.c_int]
            lib.oracle_check_mt.restype = ctypes.c_int
            lib.oracle_check_mt.argtypes = [
                ctypes.c_char_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                ctypes.c_uint32, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                ctypes.POINTER(_Result), ctypes.c_char_p, ctypes.c_int]
            lib.oracle_tuples.restype = ctypes.c_int64
            lib.oracle_tuples.argtypes = [
                ctypes.c_char_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                ctypes.c_uint32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint64),
                ctypes.c_int64, ctypes.c_char_p, ctypes.c_int]
            lib.oracle_cell.restype = ctypes.c_int
            lib.oracle_cell.argtypes = [
                ctypes.c_char_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                ctypes.c_uint32, ctypes.POINTER(ctypes.c_int64), ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                ctypes.POINTER(_Cell), ctypes.c_char_p, ctypes.c_int]
            lib.oracle_validate.restype = ctypes.c_int
            lib.oracle_validate.argtypes = [
                ctypes.c_char_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                ctypes.c_char_p, ctypes.c_int]
            _lib = lib
    return _lib


def _arrays(cells, params):
    cells = [int(c) for c in cells]
    params = [int(p) for p in params]
    ca = (ctypes.c_uint64 * max(1, len(cells)))(*cells)
    pa = (ctypes.c_int64 * max(1, len(params)))(*params)
    return cells, params, ca, pa


def result_dict(r: _Result) -> dict:
    """The fields the tests compare, by name."""
    d = {"status": STATUS_NAMES.get(r.status, r.status), "verdict": VERDICTS.get(r.verdict)}
    if r.status != 0:
        d.update(err_tid=r.err_tid, err_ordinal=r.err_ordinal)
        return d
    d.update(tuples=r.tuples, phases=r.phases)
    if r.verdict == 1:
        d.update(phase=r.phase, loc=r.loc, index=r.index, tid_i=r.tid_i, tid_j=r.tid_j,
                 i_writes=bool(r.i_writes), j_writes=bool(r.j_writes))
    elif r.verdict == 2:
        d.update(div_tid=r.div_tid, sync_count_0=r.sync_count_0, sync_count_div=r.sync_count_div)
    return d


def check(text: str, nthreads: int, cells=(), params=(), method: int = METHOD_CELLS) -> dict:
    """Run the oracle on one protocol; returns the result as a dict."""
    lib = _load()
    cells, params, ca, pa = _arrays(cells, params)
    r = _Result()
    msg = ctypes.create_string_buffer(512)
    lib.oracle_check(text.encode(), nthreads, len(cells), ca, len(params), pa, method,
                     ctypes.byref(r), msg, len(msg))
    d = result_dict(r)
    if r.status != 0 and msg.value:
        d["message"] = msg.value.decode(errors="replace")
    return d


def host_cores() -> int:
    """Host threads the multithreaded checker uses by default: the cores
    this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def check_mt(text: str, nthreads: int, cells=(), params=(), workers: int | None = None) -> dict:
    """Method B (per-cell records) run on ``workers`` host threads (default:
    every core); the same result as ``check(..., METHOD_CELLS)``."""
    lib = _load()
    cells, params, ca, pa = _arrays(cells, params)
    r = _Result()
    msg = ctypes.create_string_buffer(512)
    lib.oracle_check_mt(text.encode(), nthreads, len(cells), ca, len(params), pa,
                        host_cores() if workers is None else int(workers), ctypes.byref(r), msg, len(msg))
    d = result_dict(r)
    if r.status != 0 and msg.value:
        d["message"] = msg.value.decode(errors="replace")
    return d


def tuples(text: str, nthreads: int, cells=(), params=(), cap: int | None = None) -> np.ndarray:
    """All accesses as an (n, 5) uint64 array: phase, loc, index, tid, mode."""
    lib = _load()
    cells, params, ca, pa = _arrays(cells, params)
    msg = ctypes.create_string_buffer(512)
    if cap is None:
        n = lib.oracle_tuples(text.encode(), nthreads, len(cells), ca, len(params), pa,
                              None, 0, msg, len(msg))
        if n < 0:
            raise ValueError(f"oracle_tuples: {STATUS_NAMES.get(n, n)} {msg.value.decode()}")
        cap = n
    rows = np.zeros((max(cap, 1), 5), dtype=np.uint64)
    n = lib.oracle_tuples(text.encode(), nthreads, len(cells), ca, len(params), pa,
                          rows.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), cap, msg, len(msg))
    if n < 0:
        raise ValueError(f"oracle_tuples: {STATUS_NAMES.get(n, n)} {msg.value.decode()}")
    return rows[:min(n, cap)]


def cell(text: str, nthreads: int, cells, params, phase: int, loc: int, index: int) -> dict:
    """Accessors of one cell, computed one thread at a time: the witness that
    Definition 1 (with the smallest-pair reading) gives for that cell, and the
    protocol's total access count."""
    lib = _load()
    cells, params, ca, pa = _arrays(cells, params)
    r = _Cell()
    msg = ctypes.create_string_buffer(256)
    lib.oracle_cell(text.encode(), nthreads, len(cells), ca, len(params), pa, phase, loc, index,
                    ctypes.byref(r), msg, len(msg))
    none = 0xFFFFFFFF
    d = {"status": STATUS_NAMES.get(r.status, r.status), "accesses": r.cell_accesses, "total": r.total}
    racy = r.w0 != none and r.t1 != none
    d["racy"] = racy
    if racy:
        if r.w0 == r.t0:
            d.update(tid_i=r.t0, tid_j=r.t1, i_writes=True, j_writes=(r.w1 == r.t1))
        else:
            d.update(tid_i=r.t0, tid_j=r.w0, i_writes=False, j_writes=True)
    return d


def validate(text: str):
    """(status name, declared arrays, declared params, message)."""
    lib = _load()
    na, npar = ctypes.c_int(), ctypes.c_int()
    msg = ctypes.create_string_buffer(512)
    st = lib.oracle_validate(text.encode(), ctypes.byref(na), ctypes.byref(npar), msg, len(msg))
    return STATUS_NAMES.get(st, st), na.value, npar.value, msg.value.decode(errors="replace")
