import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled library")
    config.addinivalue_line("markers", "slow: long CPU test")
    config.addinivalue_line("markers", "mutation: plants a mistake in a copy of the oracle (opt-in)")


@pytest.fixture(scope="session")
def dp():
    """The CUDA library binding; GPU tests only."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_14675_gb300 import dp as _dp
    _dp.load()
    return _dp
