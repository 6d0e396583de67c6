import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.dirname(os.path.abspath(__file__))
for p in (ROOT, TESTS):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle._lib()
    return oracle


@pytest.fixture(scope="session")
def gpu():
    """The CUDA library and torch on cuda:0; fails (does not skip) without a GPU."""
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1406_7808_gb300 import build, srfmg
    build.build()
    srfmg.load()
    torch.cuda.set_device(0)
    return srfmg
