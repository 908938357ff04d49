import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the C-ABI kernels)")
    config.addinivalue_line("markers", "slow: larger CPU cases")


@pytest.fixture(scope="session")
def dgsl_lib():
    """Build (if stale) and load libdgsl.so."""
    from paper_2401_17806_gb300 import build, dgsl
    build.build()
    return dgsl.load()
