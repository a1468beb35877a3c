import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU-side oracle runs")


@pytest.fixture(scope="session")
def built_lib():
    """Build (if needed) and load the CUDA library; GPU tests only."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_2212_04415_gb300 as pd
    return pd


@pytest.fixture(scope="session")
def oracle_lib():
    from oracle import core
    core.build()
    return core
