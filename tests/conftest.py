import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    import oracle

    return oracle.default()


@pytest.fixture(scope="session")
def rlib():
    """The product's binding, with the CUDA library built in-tree if stale."""
    from paper_1402_3392_b300 import build

    build.build()
    from paper_1402_3392_b300 import rans

    return rans


@pytest.fixture(scope="session")
def cuda(rlib):
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU test collected without a CUDA device")
    return torch.device("cuda:0")
