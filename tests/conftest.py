import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than ~10 s on one CPU core")


def read_table(name):
    """Rows (exponent, pi value) of a golden table file."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                e, v = line.split()
                rows.append((int(e), int(v)))
    return rows


@pytest.fixture(scope="session")
def pi_pow10():
    return dict(read_table("pi_pow10.txt"))


@pytest.fixture(scope="session")
def pi_pow2():
    return dict(read_table("pi_pow2.txt"))
