import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def ctx():
    """A libdl context on cuda:0 (GPU tests only)."""
    from paper_1608_00139_gb300 import build as libbuild
    from paper_1608_00139_gb300 import dl
    libbuild.build()
    c = dl.Context(0)
    yield c
    c.close()
