"""Shared test configuration.

Tests marked `gpu` need a CUDA device and the compiled library; everything else
runs on the CPU (`pytest -m "not gpu"`).
"""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled libdmp")
    config.addinivalue_line("markers", "slow: long-running (minutes)")


@pytest.fixture(scope="session")
def golden_dir():
    return GOLDEN


@pytest.fixture(scope="session")
def dmp():
    """The compiled library's binding, on a CUDA device. Fails (does not skip)
    when the library cannot be built or loaded: there is no fallback path."""
    import torch

    from paper_2407_13299_gb300 import build
    from paper_2407_13299_gb300 import dmp as binding

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    binding.lib()
    return binding
