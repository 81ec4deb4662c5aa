"""Compile a planted mistake into a temporary copy of the oracle library (never
into the committed oracle) and swap it in for the duration of a test."""
import contextlib
import ctypes
import os
import shutil
import subprocess
import tempfile

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "exactz_oracle.c")
ENTRY_POINTS = ("oracle_mesh", "oracle_classify", "oracle_cp_order", "oracle_correct",
                "oracle_requests", "oracle_correct_events", "oracle_requests_events", "oracle_correct_ex",
                "oracle_requests_ex")


@contextlib.contextmanager
def mutant(monkeypatch, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    tmp = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        path = os.path.join(tmp, "mutant.c")
        open(path, "w").write(src.replace(old, new))
        so = os.path.join(tmp, "libmutant.so")
        subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                        "-mfpmath=sse", path, "-o", so, "-lm"], check=True)
        real = oracle.lib()
        L = ctypes.CDLL(so)
        for fn in ENTRY_POINTS:
            getattr(L, fn).argtypes = getattr(real, fn).argtypes
            getattr(L, fn).restype = getattr(real, fn).restype
        with monkeypatch.context() as m:
            m.setattr(oracle, "_lib", L)
            yield
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
