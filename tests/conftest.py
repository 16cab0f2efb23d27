import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the sm_103a library")
    config.addinivalue_line("markers", "slow: long CPU run of the oracle (still part of the CPU suite)")


@pytest.fixture(scope="session")
def torch_threads():
    import torch
    return torch.get_num_threads()
