import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def oracle():
    import oracle as _oracle
    _oracle._load()
    return _oracle


@pytest.fixture(scope="session")
def wavelib():
    """The built CUDA library's binding (builds it if needed)."""
    from paper_1806_08299_gb300 import build, wave
    build.build()
    wave._lib()
    return wave


@pytest.fixture(scope="session")
def cuda(wavelib):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected without a CUDA device")
    return torch.device("cuda:0")
