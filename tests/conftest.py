import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU case")


@pytest.fixture(scope="session")
def small_wl():
    import synth
    return synth.preset("small", seed=1)


@pytest.fixture(scope="session")
def small_set(small_wl):
    import oracle
    return oracle.ClipSet(small_wl)
