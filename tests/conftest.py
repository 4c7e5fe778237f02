import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def hms_ctx():
    """One library context on cuda:0 for the GPU tests."""
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_1208_4093_gb300 import capi
    ctx = capi.hms_context_create(0)
    yield ctx
    capi.hms_context_destroy(ctx)
