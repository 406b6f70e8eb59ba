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


@pytest.fixture(scope="session")
def bfx():
    """The CUDA library binding (built in-tree if a source is newer than it)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1904_06376_b300 import build as _b

    _b.build()
    import paper_1904_06376_b300 as lib

    lib.lib()
    return lib


@pytest.fixture(autouse=True)
def _no_device_error(request):
    """Every GPU test must leave the device error word clear."""
    yield
    if request.node.get_closest_marker("gpu") is None:
        return
    import torch

    if not torch.cuda.is_available():
        return
    import paper_1904_06376_b300 as lib

    torch.cuda.synchronize()
    assert lib.device_error() == 0, "a bounded device-side wait expired"
