import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session", autouse=True)
def _library_current():
    """Rebuilds libamrmhd.so when a source is newer than it (nvcc cross-compiles
    without a GPU), so that no test loads a stale library."""
    from paper_1110_1616_gb300 import build
    if not build.up_to_date() and shutil.which(build.NVCC):
        build.build()
    yield
