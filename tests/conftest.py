import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


_CACHE = {}


@pytest.fixture(scope="session")
def datasets():
    """Session cache of generated workloads (cfg3 takes ~10 s to draw)."""
    import gen

    def get(name, **kw):
        key = (name, tuple(sorted(kw.items())))
        if key not in _CACHE:
            _CACHE[key] = getattr(gen, name)(**kw)
        return _CACHE[key]

    return get
