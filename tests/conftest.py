import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: oracle cases that take tens of seconds on one core")


@pytest.fixture(scope="session")
def pxa_lib():
    """Build (if stale) and load libpxa.so; the CUDA path has no fallback."""
    from paper_2004_00546_gb300 import build, pxa

    build.build()
    return pxa.load()


@pytest.fixture(scope="session")
def cuda_ok(pxa_lib):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return pxa_lib
