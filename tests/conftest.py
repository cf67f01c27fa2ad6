import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_sessionstart(session):
    """Build the in-tree CUDA library once if it is missing (nvcc cross-compiles without a GPU)."""
    from paper_2406_18479_gb300 import build
    if not os.path.exists(build.LIB):
        try:
            build.nvcc()
        except RuntimeError:
            return          # no toolchain: the tests that need the library fail loudly
        build.build()
