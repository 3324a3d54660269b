import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libss")
    config.addinivalue_line("markers", "slow: longer CPU/GPU cases")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def ss():
    """The C-ABI binding, built for sm_103a; GPU tests only."""
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_1804_07135_gb300 import binding
    binding.load()
    return binding
