import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="session")
def skel():
    """The CUDA library binding, built if needed; GPU tests only."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2104_05877_gb300 as sk
    if not os.path.exists(sk.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    sk.lib()
    return sk


@pytest.fixture(scope="session")
def dev():
    import torch
    return torch.device("cuda:0")
