import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def _load_builder(path, name):
    import importlib.util

    spec = importlib.util.spec_from_file_location(name, path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


# Build both shared libraries before any test imports them (nvcc cross-compiles
# the sm_103a library without a GPU; gcc builds the oracle).
_load_builder(os.path.join(ROOT, "paper_2604_01397_b300", "build.py"), "_exz_lib_build").build()
_load_builder(os.path.join(ROOT, "oracle", "build.py"), "_exz_oracle_build").build()


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
