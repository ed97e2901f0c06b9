"""Shared test configuration: markers, GPU gating and small graph helpers."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (runs the library's kernels)")
    config.addinivalue_line("markers", "slow: full-size workloads (minutes)")


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _cuda_ok():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def gclib():
    """The CUDA library, built in-tree if needed (fails loudly when it cannot be built)."""
    from paper_1509_08267_gb300 import _build
    import paper_1509_08267_gb300 as gc
    _build.build()
    return gc
