import os
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the compiled libbh.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def exact_tables(orc):
    """Oracle tables at the paper's sizes (512x512 D, 64x32 U)."""
    return orc.tables_exact(512, 64, 32, 1e-3)


@pytest.fixture(scope="session")
def colour_tables(orc):
    return orc.colour_table(64, 32, 64), orc.disc_colour_table(1024)
