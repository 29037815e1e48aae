import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libpcr")


@pytest.fixture(scope="session")
def gpu():
    """Skip unless CUDA is present; build (if needed) and load the CUDA library."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_02681_gb300 import pcr
    pcr.load()
    return pcr
