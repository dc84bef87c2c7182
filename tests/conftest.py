import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    # the autotuner's shape cache: a fresh file per test session, so jobs created without
    # a launch shape take the library's default unless a test fills the cache itself
    import tempfile
    os.environ["PRDPT_AUTOTUNE_CACHE"] = os.path.join(tempfile.mkdtemp(prefix="prdpt_tune_"), "autotune.json")
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library; GPU tests skip on a machine without a GPU and fail loudly
    if the GPU exists but the library cannot be loaded."""
    if not cuda_available():
        pytest.skip("no CUDA device")
    from paper_2211_17263_gb300 import capi
    return capi.load()
