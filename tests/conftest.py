import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def _modules(session):
    seen = {}
    for item in session.items:
        mod = getattr(item, "module", None)
        if mod is not None:
            seen.setdefault(id(mod), mod)
    return list(seen.values())


def pytest_collection_finish(session):
    """Let selected test modules start CPU work that they will need later (the
    final-time oracle runs) before the first test runs."""
    if session.config.option.collectonly:
        return
    for mod in _modules(session):
        start = getattr(mod, "start_early", None)
        if callable(start):
            start()


def pytest_sessionfinish(session, exitstatus):
    for mod in _modules(session):
        stop = getattr(mod, "stop_early", None)
        if callable(stop):
            stop()
