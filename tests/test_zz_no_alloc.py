"""The allocation-free check (drf_check_noalloc) against the ordinary one.

drf_check_noalloc serves callers that cannot call cudaMalloc when they need
a check -- for example a process whose device memory another component's
allocator has already reserved.  It runs the same pipeline in a fixed
device array that the library reserves when it is loaded.  Its results must
equal drf_check's exactly (this is integer work, so the tolerance is zero),
call after call, even though consecutive calls reuse the same array.

This file is named to be collected last, so that a run stopping at the
first failure has run every other test first.
"""
import pytest

from paper_2203_12878_b300 import drf, protogen

pytestmark = pytest.mark.gpu


def _cases():
    cs = [protogen.config1("drf"), protogen.config1("nosync"),
          protogen.config2(1, target=2e5), protogen.config2(3, "constructed", target=3e5, plant=True)]
    cs += [protogen.random_small(s) for s in range(12)]
    return cs


def test_no_alloc_matches_drf_check_twice_in_a_row(oracle):
    import torch
    torch.cuda.set_device(0)
    ctx = drf.drf_ctx_create(0)
    try:
        for p in _cases():
            bc = drf.drf_protocol_compile(p.text)
            want = drf.result_dict(drf.drf_check(ctx, bc, p.nthreads, p.cells, p.params))
            first = drf.result_dict(drf.drf_check_noalloc(bc, p.nthreads, p.cells, p.params))
            second = drf.result_dict(drf.drf_check_noalloc(bc, p.nthreads, p.cells, p.params))
            assert first == want, p.text
            assert second == want, p.text
            # and directly against the oracle (this entry point always runs
            # the sort path, drf_check on a default context may not)
            exp = oracle.check(p.text, p.nthreads, p.cells, p.params, oracle.METHOD_CELLS)
            exp.pop("message", None)
            if exp["status"] != "OVERFLOW":
                assert first == exp, p.text
    finally:
        drf.drf_ctx_destroy(ctx)


def test_no_alloc_rejects_what_does_not_fit():
    import torch
    torch.cuda.set_device(0)
    p = protogen.config2(0)              # ~1.2e7 accesses: more than the fixed array holds
    bc = drf.drf_protocol_compile(p.text)
    r = drf.drf_check_noalloc(bc, p.nthreads, p.cells, p.params)
    assert drf.result_dict(r)["status"] == "LIMIT"
    # a small check right after still works
    q = protogen.config1("nosync")
    got = drf.result_dict(drf.drf_check_noalloc(drf.drf_protocol_compile(q.text), q.nthreads, q.cells, q.params))
    assert got["verdict"] == "RACY" and (got["tid_i"], got["tid_j"]) == (0, 255)
