"""Shared fixtures. GPU tests are marked `gpu`; everything else runs on the CPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


_cache = {}


def cached_system(name, fn):
    if name not in _cache:
        _cache[name] = fn()
    return _cache[name]


@pytest.fixture(scope="session")
def small_water():
    from paper_1904_08756_gb300 import synth
    return cached_system("small_water", synth.small_water)
