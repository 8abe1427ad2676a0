import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: long-running oracle case")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def lib():
    """The CUDA library, built in place if needed (compiles on a CPU-only box too)."""
    from paper_1206_3215_gb300 import build as _b  # noqa: F401
    import paper_1206_3215_gb300.build as B
    B.build()
    import paper_1206_3215_gb300 as P
    P.load_library()
    return P


@pytest.fixture(scope="session")
def cuda_device(lib):
    import torch
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    torch.cuda.init()
    return torch.device("cuda:0")
