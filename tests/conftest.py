import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 and the CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def cases():
    """Seeded synthetic cases, drawn once per session."""
    from gen import make_config
    store = {}

    def get(cfg, **kw):
        key = (cfg, tuple(sorted(kw.items())))
        if key not in store:
            store[key] = make_config(cfg, **kw)
        return store[key]
    return get
