"""Run-time specialization, host side: the generated CUDA source of a
protocol's count, owner-table and witness kernels compiles with NVRTC for
sm_103a (no GPU needed), for protocols across the whole syntax."""
import ctypes.util
import random

import pytest

from paper_2203_12878_b300 import drf, protogen


def _nvrtc():
    try:
        ctypes.CDLL("libnvrtc.so.13")
        return True
    except OSError:
        return False


pytestmark = pytest.mark.skipif(not _nvrtc(), reason="NVRTC not installed")


def _protocols():
    ps = [protogen.config1("drf"), protogen.config1("nosync"), protogen.config2(0),
          protogen.config2(3, "constructed", target=3e5, plant=True),
          protogen.config4_one(random.Random(5), True), protogen.config4_one(random.Random(9), False)]
    ps += [protogen.random_small(s) for s in range(0, 400, 10)]
    return ps


@pytest.mark.parametrize("i", range(46))
def test_specialized_source_compiles(i):
    p = _protocols()[i]
    bc = drf.drf_protocol_compile(p.text)
    st, src, log = drf.drf_protocol_specialize(bc, p.nthreads, p.cells, p.params)
    if st == "LIMIT":            # no owner table (or too many shapes): the plan keeps the interpreter
        assert src is None
        return
    assert st == "OK", log
    for k in ("drf_count", "drf_table", "drf_cell"):
        assert f'extern "C" __global__ void __launch_bounds__(256) {k}(' in src


def test_wide_protocol_specializes_with_64bit_arithmetic():
    p = protogen.Protocol("array A;\nwr A[4294967295 + tid];\n", 2, [1 << 33], [])
    st, src, log = drf.drf_protocol_specialize(drf.drf_protocol_compile(p.text), p.nthreads, p.cells, p.params)
    assert st in ("OK", "LIMIT"), log
    if st == "OK":
        assert "int64_t v[" in src


def test_constants_are_baked_in():
    """Array sizes and table strides appear as literals in the source."""
    p = protogen.config1("drf")
    st, src, _ = drf.drf_protocol_specialize(drf.drf_protocol_compile(p.text), p.nthreads, p.cells, p.params,
                                             compile=False)
    assert st == "OK"
    assert "2048ull" in src      # the array's size bounds every index check


@pytest.mark.parametrize("seed", range(0, 60, 6))
def test_range_pass_source_compiles(seed):
    """Protocols whose accesses are mostly +-tid plus loop terms get the
    range pass (drf_range) beside the other kernels, and it compiles."""
    p = protogen.shifted_small(seed)
    st, src, log = drf.drf_protocol_specialize(drf.drf_protocol_compile(p.text), p.nthreads, p.cells, p.params)
    assert st == "OK", log


def test_grid_scale_protocol_gets_the_range_pass():
    """Every access of the grid-scale protocol at a * tid plus a function of
    the loop variables (the owned writes with a = +-1, the reads with a in
    -8..3, the tid-free read D[5x - 6] with a = 0) goes to the range pass:
    all of its 221,642,754 tuples but the two guarded writes of the planted
    race, which stay in the table pass."""
    p = protogen.config3(0, racy=True)
    st, a = drf.drf_protocol_analyze(drf.drf_protocol_compile(p.text), p.nthreads, p.cells, p.params)
    assert st == "OK"
    assert a["range_tuples"] == 221642754 - 2
    st, src, log = drf.drf_protocol_specialize(drf.drf_protocol_compile(p.text), p.nthreads, p.cells, p.params)
    assert st == "OK", log


def test_protocols_without_shifted_indices_get_no_range_pass():
    for text, T, n in (("array A;\nwr A[100 * tid];\n", 64, 6400),               # a coefficient above 64
                       ("array A;\nwr A[(64 * tid) % 65];\n", 100, 65),         # wraps more than 64 times
                       ("array A;\nwr A[tid * tid];\n", 64, 4096),                # not linear in tid
                       ("array A;\nforU x in 0 .. tid { wr A[tid + 64 * x]; }\n", 64, 64 * 64),   # bound reads tid
                       ("array A;\nforS x in 0 .. 4 { wr A[tid + 64 * x]; sync; }\n", 64, 256)):  # sync in the loop
        st, a = drf.drf_protocol_analyze(drf.drf_protocol_compile(text), T, [n], [])
        assert st == "OK" and a["range_tuples"] == 0, text
    st, a = drf.drf_protocol_analyze(drf.drf_protocol_compile("array A;\nforU x in 0 .. 4 { wr A[tid + 64 * x]; }\n"),
                                     64, [256], [])
    assert st == "OK" and a["range_tuples"] == 256          # counted at any size
    st, a = drf.drf_protocol_analyze(drf.drf_protocol_compile("array A;\nforU x in 0 .. 4 { wr A[(-3 * tid + x) % 200]; }\n"),
                                     64, [256], [])
    assert st == "OK" and a["range_tuples"] == 256          # stride -3, one wrap
    st, a = drf.drf_protocol_analyze(drf.drf_protocol_compile("array A;\nrd A[(6 * tid + 1) % 4096];\n"),
                                     853, [4096], [])
    assert st == "OK" and a["range_tuples"] == 853          # stride 6, two wraps
