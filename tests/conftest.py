import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: slower CPU test (still part of the CPU suite)")


def pytest_collection_modifyitems(config, items):
    # GPU tests cannot run without a device; skip them cleanly on CPU-only hosts
    # unless the caller explicitly selected them with -m gpu.
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


@pytest.fixture(scope="session")
def libtsm():
    """The CUDA library, built in-tree if it is not there yet (nvcc cross-compiles)."""
    from paper_1211_0126_gb300 import build, tsm
    if not os.path.exists(tsm.LIB_PATH):
        build.build()
    return tsm.library()


@pytest.fixture(scope="module")
def ctx(libtsm):
    from paper_1211_0126_gb300 import tsm
    c = tsm.Context(0)
    yield c
    c.close()
