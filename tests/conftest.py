import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built liblbm.so")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


def golden(name):
    """Parse tests/golden/<name>: lines 'key = v1 v2 ...  # citation'."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, vals = line.split("=", 1)
            out[key.strip()] = [float(v) for v in vals.split()]
    return out


@pytest.fixture(scope="session")
def paper_values():
    return golden("paper_printed_values.txt")
