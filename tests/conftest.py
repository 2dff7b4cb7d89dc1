import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and libpakr.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def cuda_lib():
    """libpakr.so loaded on a machine with a GPU; the CUDA path has no fallback."""
    import torch

    from paper_2607_03987_gb300 import _build, pakr

    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    _build.build()
    return pakr.lib()
