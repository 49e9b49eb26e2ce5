"""Shared pytest configuration.

Markers:
  gpu  -- needs a CUDA device and the compiled library (run with -m gpu).
Tests without the marker run on the CPU only (oracle pins, host logic, the
C-ABI symbol check).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the compiled sm_103a library")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as O
    O.build()
    return O
