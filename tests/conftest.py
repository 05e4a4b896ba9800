import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU-only oracle runs")


def pytest_collection_modifyitems(config, items):
    # long oracle runs (minutes of SuperLU work) run only when asked for
    if os.environ.get("STDG_SLOW_TESTS"):
        return
    skip = pytest.mark.skip(reason="slow oracle run: set STDG_SLOW_TESTS=1")
    for item in items:
        if "slow" in item.keywords:
            item.add_marker(skip)
