"""Shared pytest configuration.

``-m gpu`` tests need a GB300 and the CUDA library; ``-m "not gpu"`` tests run
on any CPU (oracle pins, host logic, C-ABI export checks).
"""
import functools
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@functools.lru_cache(maxsize=None)
def oracle_swe(level: int):
    from oracle.swe import make_swe
    return make_swe(level)


@pytest.fixture(scope="session")
def swe_factory():
    return oracle_swe
