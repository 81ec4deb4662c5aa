"""The C-ABI library builds, loads and exports every entry point its header
declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(exactz_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    from conftest import _load_builder

    path = _load_builder(os.path.join(ROOT, "paper_2604_01397_b300", "build.py"), "_b").build()
    L = ctypes.CDLL(path)
    names = _declared()
    assert "exactz_correct" in names and "exactz_correct_batch" in names
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_package_import_loads_native_library():
    import paper_2604_01397_b300 as ez

    assert "sm_103a" in ez.version()
    assert ez._native.lib() is ez._native.lib()


def test_no_device_is_an_error_not_a_fallback():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2604_01397_b300 as ez

    L = ez._native.lib()
    d = (ez._native.Dims * 1)(ez._native.Dims(4, 4, 4))
    assert not L.exactz_workspace_create(1, d)
    res = ez._native.Result()
    rc = L.exactz_correct(None, None, ez._native.Dims(4, 4, 4), ctypes.c_float(0.1), None, None, None, 0,
                          ctypes.byref(res), None)
    assert rc == ez._native.EXACTZ_ENODEV


def test_default_opts():
    import paper_2604_01397_b300 as ez

    o = ez._native.Opts()
    ez._native.lib().exactz_default_opts(ctypes.byref(o))
    assert (o.N, o.mode, o.max_iters, o.want_edit_list) == (5, 2, 1000000, 1)
    assert (o.events, o.direction) == (ez.EVENTS["reformulated"], ez.DIRECTIONS["decreasing"])


def test_binding_constants_match_the_header():
    """Every EXACTZ_* value the Python binding uses equals the header's
    #define: return codes, loop modes, event constraints, edit directions."""
    import paper_2604_01397_b300 as ez

    txt = open(os.path.join(ROOT, "include", "exactz.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define\s+(EXACTZ_[A-Z_]+)\s+\(?(-?\d+)\)?", txt)}
    N = ez._native
    for name in ("OK", "EINVAL", "ENONFINITE", "EBOUND", "ENOMEM", "ECAP", "ENODEV", "ESIZE"):
        assert getattr(N, "EXACTZ_" + name) == defs["EXACTZ_" + name], name
    modes = {"plain": "EXACTZ_MODE_PLAIN", "frontier": "EXACTZ_MODE_FRONTIER", "graph": "EXACTZ_MODE_GRAPH",
             "fused": "EXACTZ_MODE_FUSED"}
    assert set(ez.api.MODES) == set(modes)
    for k, d in modes.items():
        assert ez.api.MODES[k] == defs[d], k
    assert ez.EVENTS["reformulated"] == defs["EXACTZ_EVENTS_REFORMULATED"]
    assert ez.EVENTS["original"] == defs["EXACTZ_EVENTS_ORIGINAL"]
    assert ez.DIRECTIONS["decreasing"] == defs["EXACTZ_EDITS_DECREASING"]
    assert ez.DIRECTIONS["increasing"] == defs["EXACTZ_EDITS_INCREASING"]


def test_oracle_and_library_share_no_code():
    # the oracle is plain C compiled by gcc; the library is CUDA; neither
    # includes, imports or links the other
    osrc = open(os.path.join(ROOT, "oracle", "exactz_oracle.c")).read()
    assert "#include \"" not in osrc
    for fn in os.listdir(os.path.join(ROOT, "paper_2604_01397_b300", "csrc")):
        src = open(os.path.join(ROOT, "paper_2604_01397_b300", "csrc", fn)).read()
        assert "oracle" not in src.lower() or "oracle's notes" in src
    for fn in ("api.py", "_native.py", "__init__.py"):
        src = open(os.path.join(ROOT, "paper_2604_01397_b300", fn)).read()
        assert "import oracle" not in src and "from oracle" not in src


def test_ctypes_structs_match_the_header(tmp_path):
    # compile a C program against include/exactz.h and compare every struct's
    # size and field offsets with the ctypes mirror used by the binding
    import subprocess

    import paper_2604_01397_b300._native as N

    structs = {"exactz_dims": N.Dims, "exactz_opts": N.Opts, "exactz_edit": N.Edit, "exactz_result": N.Result,
               "exactz_stats": N.Stats, "exactz_tuning": N.Tuning, "exactz_server_config": N.ServerConfig,
               "exactz_server_info": N.ServerInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "exactz.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out if line}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
