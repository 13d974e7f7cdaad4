import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as o
    o.build()
    return o


_GRID = {}


@pytest.fixture(scope="session")
def grid_expected(oracle):
    """The oracle's result (method B over every thread of the whole protocol,
    run on all host cores) for the grid-scale protocol of a seed and
    variant, computed once per session."""
    from paper_2203_12878_b300 import protogen

    def get(seed, racy):
        key = (seed, racy)
        if key not in _GRID:
            p = protogen.config3(seed, racy=racy)
            d = oracle.check_mt(p.text, p.nthreads, p.cells, p.params)
            d.pop("message", None)
            _GRID[key] = d
        return _GRID[key]
    return get
