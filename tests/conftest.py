import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


_BUILT = False


def ensure_built():
    """Compile the oracle and the CUDA library (no-op when up to date)."""
    global _BUILT
    if not _BUILT:
        import oracle
        from paper_2104_08865_gb300 import build as _b
        oracle.build()
        _b.build()
        _BUILT = True


@pytest.fixture(scope="session")
def built():
    ensure_built()
    return True
