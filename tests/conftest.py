import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


_OPS = {}


@pytest.fixture(scope="session")
def oracle_ops():
    """Cached oracle operators per (k, p)."""
    from oracle import tables

    def get(k, p):
        if (k, p) not in _OPS:
            _OPS[(k, p)] = tables.Ops(k, p)
        return _OPS[(k, p)]
    return get
