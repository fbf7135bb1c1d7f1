import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the native library")
    config.addinivalue_line("markers", "slow: a longer CPU test (still part of the default run)")


@pytest.fixture(scope="session")
def native():
    """The ctypes binding of libdgk, built in-tree first if needed (nvcc cross-compiles
    without a GPU)."""
    from paper_1311_7477_gb300 import build as _build
    _build.build()
    from paper_1311_7477_gb300 import dg
    return dg
