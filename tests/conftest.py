import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def gpu():
    """Build and load libslr for the GPU tests; skip where no GPU is present.
    On a GPU machine a missing or broken library fails the test loudly."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_04567_gb300 import build, slr
    build.build()
    slr.load()
    torch.cuda.set_device(0)
    return slr


def run_solver(slr, stencil, u, aux=None, max_iters=1000, **fields):
    """Run one solve through the C ABI; returns (state on host, Result)."""
    s = slr.Solver(stencil, u, aux, **fields)
    s.run(max_iters)
    r = s.result()
    s.close()
    return u.cpu().numpy(), r
