import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def rng():
    import numpy as np
    return np.random.default_rng(2408)


@pytest.fixture(scope="session")
def lib():
    """The compiled C-ABI library through its Python binding (built on demand)."""
    from paper_2408_07436_gb300 import build as b
    b.build()
    from paper_2408_07436_gb300 import m2l
    return m2l
