import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels through the C ABI)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def lqlib():
    """The built liblqcd.so through its Python binding (built here if missing)."""
    from paper_1105_2279_gb300 import build
    build.build_library()
    import paper_1105_2279_gb300 as lq
    lq.capi()
    return lq


@pytest.fixture(scope="session")
def gpu(lqlib):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but CUDA is not available")
    torch.cuda.init()
    return lqlib
