import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libmtf")
    config.addinivalue_line("markers", "slow: longer CPU test (still part of the default suite)")


_cache = {}


@pytest.fixture(scope="session")
def oracle_cache():
    """Session cache of assembled oracle systems keyed by a name."""
    return _cache
