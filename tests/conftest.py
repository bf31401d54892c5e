import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_kv(name):
    """key = value lines of a fixture under tests/golden ('#' starts a comment)."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = (s.strip() for s in line.split("=", 1))
                out[k] = float(v)
    return out


def golden_rows(name):
    """';'-separated rows of a fixture under tests/golden."""
    with open(os.path.join(GOLDEN, name)) as fh:
        return [[c.strip() for c in line.split(";")] for line in fh
                if line.strip() and not line.lstrip().startswith("#")]
