import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~10 s")


def pytest_collection_finish(session):
    # start the slow oracle solves that selected tests will need, so that they run in the
    # background while the tests before them run (see oracle_cache.py)
    import oracle_cache
    for name, fragment in oracle_cache.NEEDED_BY.items():
        if any(fragment in item.nodeid for item in session.items):
            oracle_cache.start(name)


def pytest_sessionfinish(session, exitstatus):
    import oracle_cache
    oracle_cache.stop_all()
