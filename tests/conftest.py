import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def gpu_lib():
    """Build (if needed) and load libskmmse.so; skip cleanly only when there is no GPU."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_11226_gb300 import build, skmmse
    build.build()
    return skmmse.load()


@pytest.fixture(scope="session")
def gpu_ctx(gpu_lib):
    from paper_2205_11226_gb300 import skmmse
    ctx = skmmse.Context()
    yield ctx
    ctx.close()
