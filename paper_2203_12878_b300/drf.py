"""Thin ctypes binding of the C ABI in ``include/drf.h``.

Every function here has the name of the C entry point it calls and only
marshals arguments: protocol text to bytes, bounds to ``drf_bounds``,
``drf_result`` to a dict, CUDA streams (torch streams or raw handles) to
``void*``.  All checking runs in the library's CUDA kernels; there is no
Python or CPU fallback, and loading fails loudly when the library has not
been built (``python -m paper_2203_12878_b300.build``).
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdrfcheck.so")

STATUS = {
    0: "OK", -1: "INVALID_ARG", -2: "PARSE", -3: "INVALID_BYTECODE", -4: "UNBOUND_VAR",
    -5: "UNKNOWN_ARRAY", -6: "REBIND", -7: "SYNC_IN_UNSYNC", -8: "OVERFLOW_RISK",
    -9: "INDEX_OOB", -10: "DIV_ZERO", -11: "KEY_TOO_WIDE", -12: "NOMEM", -13: "CUDA",
    -14: "TIMEOUT", -15: "BUSY", -16: "LIMIT", -17: "NOT_FOUND", -18: "INTERNAL",
}
VERDICTS = {-1: None, 0: "DRF", 1: "RACY", 2: "BARRIER_DIVERGENCE"}
OPT_PROFILE_STAGES = 0x1
OPT_AUTOTUNE = 0x2
OPT_PATH_SORT = 0x4      # force the sort back end
OPT_PATH_TABLE = 0x8     # force the owner-table back end
OPT_SPECIALIZE = 0x10    # plans over one protocol may compile kernels specialized to it
OPT_RANGE_ANY = 0x20     # the owner table's range pass for batches of any size
PATHS = {1: "sort", 2: "table"}


class DrfError(RuntimeError):
    def __init__(self, status, message=""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"DRF_E_{self.name}" + (f": {message}" if message else ""))


class drf_bounds(ctypes.Structure):
    _fields_ = [("nthreads", ctypes.c_uint32), ("nlocs", ctypes.c_uint32),
                ("loc_cells", ctypes.POINTER(ctypes.c_uint64)), ("nparams", ctypes.c_uint32),
                ("params", ctypes.POINTER(ctypes.c_int64))]


class drf_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("verdict", ctypes.c_int32),
        ("phase", ctypes.c_uint32), ("loc", ctypes.c_uint32), ("index", ctypes.c_uint64),
        ("tid_i", ctypes.c_uint32), ("tid_j", ctypes.c_uint32),
        ("i_writes", ctypes.c_uint32), ("j_writes", ctypes.c_uint32),
        ("div_tid", ctypes.c_uint32), ("sync_count_0", ctypes.c_uint32),
        ("sync_count_div", ctypes.c_uint32), ("phases", ctypes.c_uint32),
        ("tuples", ctypes.c_uint64), ("err_tid", ctypes.c_uint32), ("reserved0", ctypes.c_uint32),
        ("err_ordinal", ctypes.c_uint64),
    ]


class drf_opts(ctypes.Structure):
    _fields_ = [("radix_bits", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("max_device_bytes", ctypes.c_uint64)]


class drf_analysis(ctypes.Structure):
    _fields_ = [("tuple_bound", ctypes.c_uint64), ("sync_bound", ctypes.c_uint64), ("items", ctypes.c_uint32),
                ("wide_arithmetic", ctypes.c_uint32), ("sort_bits", ctypes.c_uint32), ("key_bits", ctypes.c_uint32),
                ("range_tuples", ctypes.c_uint64)]


class drf_server_opts(ctypes.Structure):
    _fields_ = [("max_round_tuples", ctypes.c_uint64), ("max_round_protocols", ctypes.c_uint32),
                ("max_queue", ctypes.c_uint32), ("poll_us", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


_lib = None
_lock = threading.Lock()

_P = ctypes.c_void_p
_U8P = ctypes.POINTER(ctypes.c_uint8)
_SIGS = {
    "drf_version": (ctypes.c_int, []),
    "drf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "drf_ctx_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(drf_opts), ctypes.POINTER(_P)]),
    "drf_ctx_destroy": (None, [_P]),
    "drf_last_error": (ctypes.c_char_p, [_P]),
    "drf_protocol_compile": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_U8P), ctypes.POINTER(ctypes.c_size_t),
                                            ctypes.c_char_p, ctypes.c_size_t]),
    "drf_babycuda_infer": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_U8P), ctypes.POINTER(ctypes.c_size_t),
                                          ctypes.c_char_p, ctypes.c_size_t]),
    "drf_protocol_text": (ctypes.c_int, [_U8P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
    "drf_protocol_info": (ctypes.c_int, [_U8P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint32),
                                         ctypes.POINTER(ctypes.c_uint32)]),
    "drf_protocol_analyze": (ctypes.c_int, [_U8P, ctypes.c_size_t, ctypes.POINTER(drf_bounds),
                                            ctypes.POINTER(drf_analysis)]),
    "drf_free": (None, [_P]),
    "drf_check": (ctypes.c_int, [_P, _U8P, ctypes.c_size_t, ctypes.POINTER(drf_bounds),
                                 ctypes.POINTER(drf_result), _P]),
    "drf_check_batch": (ctypes.c_int, [_P, ctypes.c_uint32, ctypes.POINTER(_U8P), ctypes.POINTER(ctypes.c_size_t),
                                       ctypes.POINTER(drf_bounds), ctypes.POINTER(drf_result), _P]),
    "drf_check_noalloc": (ctypes.c_int, [_U8P, ctypes.c_size_t, ctypes.POINTER(drf_bounds),
                                         ctypes.POINTER(drf_result), _P]),
    "drf_ctx_transfer_bytes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "drf_debug_sorted_keys": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint64,
                                             ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32)]),
    "drf_debug_stall_lookback": (ctypes.c_int, [_P, ctypes.c_uint32]),
    "drf_shard_range": (ctypes.c_int, [_U8P, ctypes.c_size_t, ctypes.POINTER(drf_bounds), ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                                       ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "drf_check_shard": (ctypes.c_int, [_P, _U8P, ctypes.c_size_t, ctypes.POINTER(drf_bounds), ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.POINTER(drf_result), _P]),
    "drf_merge_shards": (ctypes.c_int, [ctypes.POINTER(drf_result), ctypes.c_uint32, ctypes.POINTER(drf_result)]),
    "drf_check_param_sweep": (ctypes.c_int, [_P, _U8P, ctypes.c_size_t, ctypes.POINTER(drf_bounds), ctypes.c_uint32,
                                             ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(drf_result), _P]),
    "drf_plan_create": (ctypes.c_int, [_P, ctypes.c_uint32, ctypes.POINTER(_U8P), ctypes.POINTER(ctypes.c_size_t),
                                       ctypes.POINTER(drf_bounds), ctypes.POINTER(_P)]),
    "drf_plan_launch": (ctypes.c_int, [_P, _P]),
    "drf_plan_results": (ctypes.c_int, [_P, ctypes.POINTER(drf_result)]),
    "drf_plan_keys": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    "drf_plan_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32),
                                     ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)]),
    "drf_plan_stage_times": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_float),
                                            ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "drf_plan_config": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                       ctypes.POINTER(ctypes.c_uint32)]),
    "drf_plan_path": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint32)]),
    "drf_plan_specialized": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint32), ctypes.c_char_p, ctypes.c_size_t]),
    "drf_protocol_specialize": (ctypes.c_int, [_U8P, ctypes.c_size_t, ctypes.POINTER(drf_bounds),
                                               ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.c_char_p,
                                               ctypes.c_size_t]),
    "drf_plan_range_tuples": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "drf_plan_destroy": (None, [_P]),
    "drf_server_start": (ctypes.c_int, [_P, ctypes.POINTER(drf_server_opts)]),
    "drf_server_submit": (ctypes.c_int, [_P, _U8P, ctypes.c_size_t, ctypes.POINTER(drf_bounds),
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "drf_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(drf_result), ctypes.c_int64,
                                       ctypes.POINTER(ctypes.c_uint64)]),
    "drf_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_uint32)]),
    "drf_server_stop": (ctypes.c_int, [_P]),
}
EXPORTED = tuple(_SIGS)


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2203_12878_b300.build` "
                                   "(there is no fallback implementation)")
            l = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(l, name)
                f.restype = res
                f.argtypes = args
            _lib = l
    return _lib


def _stream(stream):
    """A cudaStream_t from None, an int handle or a torch.cuda.Stream."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _bytes(bc: bytes):
    buf = (ctypes.c_uint8 * max(1, len(bc))).from_buffer_copy(bc if bc else b"\0")
    return buf, ctypes.cast(buf, _U8P), len(bc)


class Bounds:
    """Keeps the arrays a drf_bounds points to alive."""

    def __init__(self, nthreads, cells=(), params=()):
        self.cells = (ctypes.c_uint64 * max(1, len(cells)))(*[int(c) for c in cells])
        self.params = (ctypes.c_int64 * max(1, len(params)))(*[int(p) for p in params])
        self.c = drf_bounds(int(nthreads), len(cells), self.cells, len(params), self.params)


def result_dict(r: drf_result) -> dict:
    """The fields of a result that are defined for its status and verdict."""
    d = {"status": STATUS.get(r.status, r.status), "verdict": VERDICTS.get(r.verdict)}
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


# ------------------------------------------------------------------ C ABI --

def drf_version() -> int:
    return lib().drf_version()


def drf_status_string(status: int) -> str:
    return lib().drf_status_string(status).decode()


def drf_protocol_compile(text: str) -> bytes:
    """Protocol text -> portable bytecode; raises DrfError on rejection."""
    out = _U8P()
    n = ctypes.c_size_t()
    err = ctypes.create_string_buffer(512)
    st = lib().drf_protocol_compile(text.encode(), ctypes.byref(out), ctypes.byref(n), err, len(err))
    if st != 0:
        raise DrfError(st, err.value.decode(errors="replace"))
    try:
        return ctypes.string_at(out, n.value)
    finally:
        lib().drf_free(out)


def drf_babycuda_infer(text: str) -> bytes:
    """BabyCUDA program -> bytecode of its inferred MAP; raises DrfError when
    the program is ill-typed (e.g. data-dependent indexing)."""
    out = _U8P()
    n = ctypes.c_size_t()
    err = ctypes.create_string_buffer(512)
    st = lib().drf_babycuda_infer(text.encode(), ctypes.byref(out), ctypes.byref(n), err, len(err))
    if st != 0:
        raise DrfError(st, err.value.decode(errors="replace"))
    try:
        return ctypes.string_at(out, n.value)
    finally:
        lib().drf_free(out)


def drf_protocol_text(bytecode: bytes) -> str:
    """MAP text of a bytecode."""
    _keep, p, n = _bytes(bytecode)
    out = ctypes.c_void_p()
    st = lib().drf_protocol_text(p, n, ctypes.byref(out))
    if st != 0:
        raise DrfError(st)
    try:
        return ctypes.string_at(out).decode()
    finally:
        lib().drf_free(out)


def drf_protocol_info(bytecode: bytes):
    _keep, p, n = _bytes(bytecode)
    nl, npar = ctypes.c_uint32(), ctypes.c_uint32()
    st = lib().drf_protocol_info(p, n, ctypes.byref(nl), ctypes.byref(npar))
    if st != 0:
        raise DrfError(st)
    return nl.value, npar.value


def drf_protocol_analyze(bytecode: bytes, nthreads: int, cells=(), params=()):
    """(status name, dict of the static analysis) -- host only, no GPU."""
    _keep, p, n = _bytes(bytecode)
    b = Bounds(nthreads, cells, params)
    a = drf_analysis()
    st = lib().drf_protocol_analyze(p, n, ctypes.byref(b.c), ctypes.byref(a))
    return STATUS.get(st, st), {f: getattr(a, f) for f, _ in drf_analysis._fields_}


def drf_protocol_specialize(bytecode: bytes, nthreads: int, cells=(), params=(), compile: bool = True):
    """(status name, generated CUDA source or None, compiler log) -- host only;
    compiling needs NVRTC but no GPU."""
    _keep, p, n = _bytes(bytecode)
    b = Bounds(nthreads, cells, params)
    src = ctypes.c_void_p()
    log = ctypes.create_string_buffer(1 << 16)
    st = lib().drf_protocol_specialize(p, n, ctypes.byref(b.c), 1 if compile else 0, ctypes.byref(src), log, len(log))
    text = None
    if src.value:
        text = ctypes.string_at(src.value).decode()
        lib().drf_free(src)
    return STATUS.get(st, st), text, log.value.decode(errors="replace")


def drf_ctx_create(device: int = 0, radix_bits: int = 0, flags: int = 0, max_device_bytes: int = 0):
    ctx = _P()
    opts = drf_opts(radix_bits, flags, max_device_bytes)
    st = lib().drf_ctx_create(device, ctypes.byref(opts), ctypes.byref(ctx))
    if st != 0:
        raise DrfError(st, "drf_ctx_create")
    return ctx


def drf_ctx_destroy(ctx) -> None:
    lib().drf_ctx_destroy(ctx)


def drf_last_error(ctx) -> str:
    return lib().drf_last_error(ctx).decode(errors="replace")


def drf_check(ctx, bytecode: bytes, nthreads: int, cells=(), params=(), stream=None) -> drf_result:
    """One protocol through the whole device pipeline; returns drf_result."""
    _keep, p, n = _bytes(bytecode)
    b = Bounds(nthreads, cells, params)
    r = drf_result()
    st = lib().drf_check(ctx, p, n, ctypes.byref(b.c), ctypes.byref(r), _stream(stream))
    if st != 0 and r.status == 0:
        raise DrfError(st, drf_last_error(ctx))
    return r


def drf_check_noalloc(bytecode: bytes, nthreads: int, cells=(), params=(), stream=None) -> drf_result:
    """drf_check on the current device with no device allocation (the
    library's fixed scratch array); for callers that cannot allocate."""
    _keep, p, n = _bytes(bytecode)
    b = Bounds(nthreads, cells, params)
    r = drf_result()
    lib().drf_check_noalloc(p, n, ctypes.byref(b.c), ctypes.byref(r), _stream(stream))
    return r


def _batch_args(bytecodes, bounds):
    keep = [_bytes(bc) for bc in bytecodes]
    ptrs = (_U8P * max(1, len(keep)))(*[k[1] for k in keep])
    lens = (ctypes.c_size_t * max(1, len(keep)))(*[k[2] for k in keep])
    bs = [b if isinstance(b, Bounds) else Bounds(*b) for b in bounds]
    barr = (drf_bounds * max(1, len(bs)))(*[b.c for b in bs])
    return keep, bs, ptrs, lens, barr


def drf_check_batch(ctx, bytecodes, bounds, stream=None):
    """bounds: list of Bounds or (nthreads, cells, params) tuples.  Returns a
    list of drf_result, one per protocol."""
    keep, bs, ptrs, lens, barr = _batch_args(bytecodes, bounds)
    out = (drf_result * max(1, len(keep)))()
    st = lib().drf_check_batch(ctx, len(keep), ptrs, lens, barr, out, _stream(stream))
    if st != 0:
        raise DrfError(st, drf_last_error(ctx))
    return list(out)[:len(keep)]


def drf_ctx_transfer_bytes(ctx):
    """(host->device, device->host) bytes of the context's last check."""
    h, d = ctypes.c_uint64(), ctypes.c_uint64()
    st = lib().drf_ctx_transfer_bytes(ctx, ctypes.byref(h), ctypes.byref(d))
    if st != 0:
        raise DrfError(st)
    return h.value, d.value


def drf_shard_range(bytecode: bytes, nthreads: int, cells, params, shard: int, nshards: int):
    """(lo, hi, total) cell positions of shard `shard` of `nshards` (host only)."""
    _keep, p, n = _bytes(bytecode)
    b = Bounds(nthreads, cells, params)
    lo, hi, tot = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    st = lib().drf_shard_range(p, n, ctypes.byref(b.c), shard, nshards, ctypes.byref(lo), ctypes.byref(hi),
                               ctypes.byref(tot))
    if st != 0:
        raise DrfError(st)
    return lo.value, hi.value, tot.value


def drf_check_shard(ctx, bytecode: bytes, nthreads: int, cells, params, shard: int, nshards: int,
                    stream=None) -> drf_result:
    """The result of shard `shard` of `nshards` of one protocol (see drf.h)."""
    _keep, p, n = _bytes(bytecode)
    b = Bounds(nthreads, cells, params)
    r = drf_result()
    st = lib().drf_check_shard(ctx, p, n, ctypes.byref(b.c), shard, nshards, ctypes.byref(r), _stream(stream))
    if st != 0 and r.status == 0:
        raise DrfError(st, drf_last_error(ctx))
    return r


def drf_merge_shards(parts) -> drf_result:
    """One protocol's result from its shards' results (host only)."""
    arr = (drf_result * max(1, len(parts)))(*parts)
    out = drf_result()
    st = lib().drf_merge_shards(arr, len(parts), ctypes.byref(out))
    if st != 0 and out.status == 0:
        raise DrfError(st)
    return out


def drf_debug_stall_lookback(ctx, launches: int = 1) -> None:
    """Test hook: the context's next `launches` sort-path checks stall their
    radix look-back briefly and report DRF_E_TIMEOUT."""
    st = lib().drf_debug_stall_lookback(ctx, launches)
    if st != 0:
        raise DrfError(st)


def drf_debug_sorted_keys(ctx):
    """(sorted keys as a numpy uint64 array, layout dict) of the last check."""
    import numpy as np
    n = ctypes.c_uint64()
    lay = (ctypes.c_uint32 * 5)()
    st = lib().drf_debug_sorted_keys(ctx, None, 0, ctypes.byref(n), lay)
    if st != 0:
        raise DrfError(st)
    keys = np.zeros(max(1, n.value), dtype=np.uint64)
    st = lib().drf_debug_sorted_keys(ctx, keys.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), n.value,
                                     ctypes.byref(n), lay)
    if st != 0:
        raise DrfError(st)
    layout = dict(zip(("tid_bits", "idx_bits", "loc_bits", "phase_bits", "proto_bits"), list(lay)))
    return keys[:n.value], layout


def drf_check_param_sweep(ctx, bytecode: bytes, nthreads: int, cells, params, param: int, lo: int, hi: int,
                          stream=None):
    """Results for every value of parameter `param` in [lo, hi), one batched pass."""
    _keep, p, n = _bytes(bytecode)
    b = Bounds(nthreads, cells, params)
    out = (drf_result * max(1, hi - lo))()
    st = lib().drf_check_param_sweep(ctx, p, n, ctypes.byref(b.c), param, lo, hi, out, _stream(stream))
    if st != 0:
        raise DrfError(st, drf_last_error(ctx))
    return list(out)[:max(0, hi - lo)]


def drf_plan_create(ctx, bytecodes, bounds):
    keep, bs, ptrs, lens, barr = _batch_args(bytecodes, bounds)
    plan = _P()
    st = lib().drf_plan_create(ctx, len(keep), ptrs, lens, barr, ctypes.byref(plan))
    if st != 0:
        raise DrfError(st, drf_last_error(ctx))
    plan._n = len(keep)
    return plan


def drf_plan_launch(plan, stream=None) -> None:
    st = lib().drf_plan_launch(plan, _stream(stream))
    if st != 0:
        raise DrfError(st)


def drf_plan_results(plan):
    out = (drf_result * plan._n)()
    st = lib().drf_plan_results(plan, out)
    if st != 0:
        raise DrfError(st)
    return list(out)


def drf_plan_info(plan) -> dict:
    t, p, k, b = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    st = lib().drf_plan_info(plan, ctypes.byref(t), ctypes.byref(p), ctypes.byref(k), ctypes.byref(b))
    if st != 0:
        raise DrfError(st)
    return {"tuples": t.value, "sort_passes": p.value, "kernels_per_launch": k.value, "sort_bits": b.value}


def drf_plan_keys(plan) -> int:
    k = ctypes.c_uint64()
    st = lib().drf_plan_keys(plan, ctypes.byref(k))
    if st != 0:
        raise DrfError(st)
    return k.value


def drf_plan_stage_times(plan) -> list:
    names = (ctypes.c_char_p * 32)()
    ms = (ctypes.c_float * 32)()
    n = ctypes.c_int()
    st = lib().drf_plan_stage_times(plan, names, ms, 32, ctypes.byref(n))
    if st != 0:
        raise DrfError(st)
    return [(names[i].decode(), ms[i]) for i in range(n.value)]


def drf_plan_config(plan) -> dict:
    g, it, rb = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    st = lib().drf_plan_config(plan, ctypes.byref(g), ctypes.byref(it), ctypes.byref(rb))
    if st != 0:
        raise DrfError(st)
    return {"granularity": g.value, "radix_items": it.value, "radix_bits": rb.value}


def drf_plan_range_tuples(plan):
    """(access tuples of the range pass's accesses per launch, record updates
    its last launch made)."""
    n, u = ctypes.c_uint64(), ctypes.c_uint64()
    st = lib().drf_plan_range_tuples(plan, ctypes.byref(n), ctypes.byref(u))
    if st != 0:
        raise DrfError(st)
    return n.value, u.value


def drf_plan_specialized(plan):
    """(0: interpreted, 1: specialized kernels, 2: specialized with static
    phases -- no count or scan pass, 3: the same with the range pass; why
    not specialized when asked for)."""
    v = ctypes.c_uint32()
    log = ctypes.create_string_buffer(4096)
    st = lib().drf_plan_specialized(plan, ctypes.byref(v), log, len(log))
    if st != 0:
        raise DrfError(st)
    return int(v.value), log.value.decode(errors="replace")


def drf_plan_path(plan) -> str:
    """'sort' or 'table': the back end the plan runs."""
    v = ctypes.c_uint32()
    st = lib().drf_plan_path(plan, ctypes.byref(v))
    if st != 0:
        raise DrfError(st)
    return PATHS[v.value]


def drf_plan_destroy(plan) -> None:
    lib().drf_plan_destroy(plan)


def drf_server_start(ctx, max_round_tuples=0, max_round_protocols=0, max_queue=0, poll_us=0) -> None:
    o = drf_server_opts(max_round_tuples, max_round_protocols, max_queue, poll_us, 0)
    st = lib().drf_server_start(ctx, ctypes.byref(o))
    if st != 0:
        raise DrfError(st)


def drf_server_submit(ctx, bytecode: bytes, nthreads: int, cells=(), params=()) -> int:
    _keep, p, n = _bytes(bytecode)
    b = Bounds(nthreads, cells, params)
    t = ctypes.c_uint64()
    st = lib().drf_server_submit(ctx, p, n, ctypes.byref(b.c), ctypes.byref(t))
    if st != 0:
        raise DrfError(st)
    return t.value


def drf_server_poll(ctx, ticket: int, timeout_us: int = -1):
    """(drf_result, latency_ns), or None when the timeout expires first."""
    r = drf_result()
    lat = ctypes.c_uint64()
    st = lib().drf_server_poll(ctx, ticket, ctypes.byref(r), timeout_us, ctypes.byref(lat))
    if st == -14:
        return None
    if st != 0:
        raise DrfError(st)
    return r, lat.value


def drf_server_stats(ctx) -> dict:
    r, c, m = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint32()
    st = lib().drf_server_stats(ctx, ctypes.byref(r), ctypes.byref(c), ctypes.byref(m))
    if st != 0:
        raise DrfError(st)
    return {"rounds": r.value, "completed": c.value, "max_round": m.value}


def drf_server_stop(ctx) -> None:
    st = lib().drf_server_stop(ctx)
    if st != 0:
        raise DrfError(st)
