import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def cuda_lib():
    """The product library (C-ABI), loaded once; skips when no GPU is visible."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_01177_gb300 import tor
    return tor


@pytest.fixture(scope="session", autouse=True)
def _built_library():
    """Compile the product library if it is missing or stale (nvcc only, no GPU needed), so CPU
    tests of host code that goes through it (partial sums, conversions) run from a fresh tree."""
    from paper_2009_01177_gb300 import build
    build.build()
