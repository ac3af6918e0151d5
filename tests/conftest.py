import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TABLE = os.path.join(ROOT, "tables", "cbc_korobov_a2_s10.txt")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built extension")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def genvec_table():
    from oracle import load_genvec_table
    return load_genvec_table(TABLE)


def golden(name):
    return os.path.join(ROOT, "tests", "golden", name)
