import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session", autouse=True)
def _oracle_built():
    from oracle import build

    build.build()


def read_golden(name):
    """Parse a tests/golden fixture: 'key v1 v2 ...' lines, '#' comments."""
    path = os.path.join(ROOT, "tests", "golden", name)
    out = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        out[k] = v
    return out


def read_golden_cases(name):
    path = os.path.join(ROOT, "tests", "golden", name)
    cases = {}
    cur = None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        if k == "case":
            cur = cases.setdefault(v[0], {})
            continue
        cur[k] = v
    return cases
