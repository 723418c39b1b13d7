import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def small_phantom():
    from phantom import SMALL, make_lung_phantom
    return make_lung_phantom(SMALL)


@pytest.fixture(scope="session")
def full_phantom():
    from phantom import FULL, make_lung_phantom
    return make_lung_phantom(FULL)
