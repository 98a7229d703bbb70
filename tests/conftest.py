import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def O():
    """The FP64 CPU oracle (built on first use)."""
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def caption():
    import lbinputs
    return dict(lbinputs.CAPTION)
