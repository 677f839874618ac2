import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300); runs through the C-ABI library")
    config.addinivalue_line("markers", "slow: test that takes more than ~20 s")


@pytest.fixture(scope="session")
def ora():
    from oracle import oracle as O
    O.load()
    return O


@pytest.fixture(scope="session")
def synth():
    from paper_1407_7595_gb300 import synth as S
    return S
