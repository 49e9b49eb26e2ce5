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


@pytest.fixture(scope="session")
def gpu():
    """The compiled library plus torch on cuda:0 (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_16862_gb300 import build
    build.build()
    from paper_2403_16862_gb300 import _binding
    _binding.load()
    torch.cuda.set_device(0)
    return torch.device("cuda:0")
