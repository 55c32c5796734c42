import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libfhr")
    config.addinivalue_line("markers", "slow: long-running oracle case")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.lib()
    # every oracle sum is taken in a fixed order, so the thread count changes only the time
    oracle.set_threads(len(os.sched_getaffinity(0)))
    return oracle


@pytest.fixture(scope="session")
def lib_path():
    from paper_2410_22500_gb300 import build

    return build.build()


@pytest.fixture(scope="session")
def fx(lib_path):
    """A libfhr context on cuda:0 (GPU tests only; fails loudly without a GPU)."""
    import torch
    from paper_2410_22500_gb300 import fhr

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    ctx = fhr.Context(0)
    yield ctx
    torch.cuda.synchronize()
    ctx.close()
