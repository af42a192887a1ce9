import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libdbp")
    config.addinivalue_line("markers", "slow: longer CPU-only oracle checks")


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def dbp_lib():
    """The built C-ABI library (built on demand)."""
    from paper_1507_00921_gb300 import _lib
    return _lib.load()
