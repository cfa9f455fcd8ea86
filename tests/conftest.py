"""Shared pytest configuration.

Markers: `gpu` marks tests that need a CUDA device (GB300); everything else
runs on the CPU.  The repo root is put on sys.path so that tests can import
the package, the oracle (test infrastructure) and the workload generators.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a)")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle

    oracle.build()
    return oracle
