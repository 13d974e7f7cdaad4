"""Host-side pieces of the benchmark line that need no GPU."""
import os
import sys

import pytest

sys.path.insert(0, os.path.join(os.path.dirname(__file__), ".."))
import bench  # noqa: E402


@pytest.mark.parametrize("sort_bits, passes, per_tuple", [
    (29, 4, 80),     # the grid-scale protocol: phase 3 + array 2 + index 24 bits
    (32, 4, 80),     # four whole digits
    (33, 5, 96),     # one bit more takes a fifth pass
    (15, 2, 48),     # the 256-thread protocol: phase 4 + index 11 bits
    (0, 0, 16),      # nothing to sort: one key written and read
])
def test_materialize_scan_bytes(sort_bits, passes, per_tuple):
    m = bench.materialize_scan_fractions(1e9, sort_bits, 1000.0)
    assert m["reference_passes"] == passes
    assert m["reference_bytes_per_tuple"] == per_tuple


def test_materialize_scan_fractions():
    # 10^12 tuples/s at 80 B per tuple is 80 TB/s, ten times an 8 TB/s copy;
    # at the 16 B lower bound it is 16 TB/s, twice that copy
    m = bench.materialize_scan_fractions(1e12, 29, 8000.0)
    assert m["pipeline_frac"] == pytest.approx(10.0)
    assert m["lower_bound_frac"] == pytest.approx(2.0)
    # a throughput exactly at the lower bound's bandwidth
    m = bench.materialize_scan_fractions(8000e9 / 16, 20, 8000.0)
    assert m["lower_bound_frac"] == pytest.approx(1.0)
    assert m["pipeline_frac"] == pytest.approx(4.0)      # 16 * (1 + 3) / 16
