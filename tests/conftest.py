import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300); parity tests through the C-ABI")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~20 s")


_BOXES = {}


@pytest.fixture(scope="session")
def obox():
    """Session cache of oracle fold libraries: obox((3, 3, 3))."""
    import oracle

    def get(dims):
        dims = tuple(dims)
        if dims not in _BOXES:
            _BOXES[dims] = oracle.Box(dims)
        return _BOXES[dims]

    return get
