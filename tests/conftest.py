import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a B300 (CUDA) device")
    config.addinivalue_line("markers", "slow: long CPU-side test")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu():
    """The product binding on cuda:0.  A GPU test must never fall back to
    the CPU: without a device it fails loudly."""
    if not cuda_available():
        pytest.fail("this test needs a CUDA device")
    import paper_1912_07423_b300 as snn
    return snn
