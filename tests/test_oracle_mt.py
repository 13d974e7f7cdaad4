"""The oracle's multithreaded driver of method B (per-cell records, host
threads over thread-id ranges and then over shards of consecutive cells)
against the single-threaded method B it runs the steps of: every result
field equal, for every worker count, on protocols covering evaluation errors
(smallest failing tid and its ordinal), barrier divergence, races and
race-free protocols."""
import pytest

from paper_2203_12878_b300 import protogen


def _strip(d):
    d = dict(d)
    d.pop("message", None)
    return d


@pytest.mark.parametrize("workers", [1, 2, 3, 8])
def test_mt_equals_single_thread_random_small(oracle, workers):
    statuses = set()
    for s in range(1500):
        p = protogen.random_small(s)
        a = _strip(oracle.check(p.text, p.nthreads, p.cells, p.params, oracle.METHOD_CELLS))
        b = _strip(oracle.check_mt(p.text, p.nthreads, p.cells, p.params, workers))
        assert a == b, (s, p.text, a, b)
        statuses.add((a["status"], a.get("verdict")))
    # the sample reaches every kind of outcome
    assert {("OK", "DRF"), ("OK", "RACY"), ("OK", "BARRIER_DIVERGENCE"), ("INDEX_OOB", None)} <= statuses


def test_mt_equals_single_thread_batched_family(oracle):
    for p in protogen.config4(master_seed=3, count=40):
        a = _strip(oracle.check(p.text, p.nthreads, p.cells, p.params, oracle.METHOD_CELLS))
        b = _strip(oracle.check_mt(p.text, p.nthreads, p.cells, p.params, 5))
        assert a == b, (p.text, a, b)


@pytest.mark.parametrize("racy", [False, True])
def test_mt_equals_single_thread_grid_shape(oracle, racy):
    # the grid-scale shape (4 arrays of 2^24 cells, 8 phases) at 2048 threads
    p = protogen.config3(1, racy=racy)
    p = protogen.Protocol(p.text, 2048, p.cells, p.params, p.meta)
    a = _strip(oracle.check(p.text, p.nthreads, p.cells, p.params, oracle.METHOD_CELLS))
    b = _strip(oracle.check_mt(p.text, p.nthreads, p.cells, p.params, 6))
    assert a == b


def test_mt_matches_pairwise_definition(oracle):
    # and, through method B, Definition 1 taken literally on tiny protocols
    for s in range(400):
        p = protogen.random_small(10_000 + s)
        a = _strip(oracle.check(p.text, p.nthreads, p.cells, p.params, oracle.METHOD_PAIRS))
        b = _strip(oracle.check_mt(p.text, p.nthreads, p.cells, p.params, 4))
        assert a == b, (p.text, a, b)
