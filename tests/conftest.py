import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def bmg():
    """The CUDA library's Python binding; fails loudly when it cannot load."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_05279_gb300 as pkg
    return pkg
