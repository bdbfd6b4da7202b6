import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (sm_103a); parity tests of the CUDA path")
    config.addinivalue_line(
        "markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle as O
    O.lib()
    return O


@pytest.fixture(scope="session")
def fq():
    """The CUDA library's Python binding (built in-tree if needed)."""
    from paper_2604_06947_gb300 import fqnm
    fqnm.load()
    return fqnm
