import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


import pytest


def _stale(lib, srcdirs):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    for d in srcdirs:
        for f in os.listdir(d):
            if os.path.getmtime(os.path.join(d, f)) > t:
                return True
    return False


@pytest.fixture(scope="session")
def built_lib():
    """The in-tree CUDA library, (re)built by nvcc when missing or stale."""
    from paper_1702_04728_gb300 import build, binding
    if _stale(build.LIB, [build.CSRC, os.path.join(ROOT, "include")]):
        build.build()
    return binding.lib()
