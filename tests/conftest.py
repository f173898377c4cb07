import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libcrmc.so")
    config.addinivalue_line("markers", "slow: long CPU statistical test")


@pytest.fixture(autouse=True)
def _no_plant():
    """Every test starts and ends with an unmodified oracle."""
    import oracle
    oracle.plant("none")
    yield
    oracle.plant("none")
