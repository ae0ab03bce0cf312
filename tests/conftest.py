import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")

import pytest


@pytest.fixture(scope="session")
def libbpx():
    """Builds libbpx.so in-tree if needed and returns the binding module."""
    from paper_1904_11563_gb300 import build as _build
    _build.build()
    from paper_1904_11563_gb300 import bpx
    bpx.lib()
    return bpx
