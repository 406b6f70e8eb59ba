"""Shared test configuration.

``-m "not gpu"`` runs the oracle pins, the host-side logic and the library
load/symbol checks on any machine; ``-m gpu`` runs the parity tests of the CUDA
library against the oracle on a B300.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.lib()
    return oracle
