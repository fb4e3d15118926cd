import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")
    config.addinivalue_line("markers", "long: full-length parity run of many minutes (runs with CLOT_LONG_TESTS=1)")


def pytest_collection_modifyitems(config, items):
    if os.environ.get("CLOT_LONG_TESTS") != "1":
        skip_long = pytest.mark.skip(reason="full-length run: set CLOT_LONG_TESTS=1")
        for it in items:
            if "long" in it.keywords:
                it.add_marker(skip_long)
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)
