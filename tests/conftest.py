import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def native():
    """The built native library's binding (builds it in-tree when missing)."""
    import paper_2010_00520_gb300 as F
    if not os.path.exists(F.LIB_PATH):
        from paper_2010_00520_gb300 import build
        build.build()
    F.lib()
    return F


@pytest.fixture(scope="session")
def cuda(native):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return torch
