import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 and the CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def tiny():
    from paper_2310_03505_gb300 import scenes
    return scenes.config_tiny()


@pytest.fixture(scope="session")
def rrlib():
    """Build (if needed) and load the CUDA library; GPU tests only."""
    import torch
    from paper_2310_03505_gb300 import build, rr
    build.build()
    lib = rr.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    return lib
