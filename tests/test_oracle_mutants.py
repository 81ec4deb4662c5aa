"""The pins have teeth: plausible mistakes planted in a temporary copy of the
oracle's source (never in the committed oracle) must each fail a pin.

Each mutant is compiled with gcc into a temporary directory, swapped in for
the oracle library, and run through the hand-derived runs, the independent
classifier and the fixpoint / topology properties on small fields.
"""
import numpy as np
import pytest

import oracle
from oracle import topology as T
import synth
from conftest import read_golden
from fixpoint import check_fixpoint
from mutant_util import mutant

MUTANTS = {
    "R1-down-targets-g-min": ("mark(req, C->inc ? dng : C->dnf[p]);", "mark(req, C->inc ? dng : dng);"),
    "R1-up-targets-f-max": ("mark(req, C->inc ? C->upf[p] : upg);", "mark(req, C->inc ? C->upf[p] : C->upf[p]);"),
    "R2-raises-wrong-end": ("mark(req, (below_f != C->inc) ? nb[j] : p);",
                            "mark(req, (below_f != C->inc) ? p : nb[j]);"),
    "R2-only-f-saddles": ("if (saddle_f || saddle_g) {", "if (saddle_f) {"),
    "R3-wrong-target": ("C->o[q + 1];\n    if (prec(g, b, a)) mark(req, C->inc ? b : a);",
                        "C->o[q + 1];\n    if (prec(g, b, a)) mark(req, C->inc ? b : b);"),
    "R3-dropped": ("C->o[q + 1];\n    if (prec(g, b, a)) mark(req, C->inc ? b : a);",
                   "C->o[q + 1];\n    if (0 && prec(g, b, a)) mark(req, C->inc ? b : a);"),
    "SoS-reversed": ("(h[a] == h[b] && a < b)", "(h[a] == h[b] && a > b)"),
    "floor-wrong": ("float floor_x = inc ? f[x] + xi : f[x] - xi;", "float floor_x = inc ? f[x] + xi : f[x] - 2.0f * xi;"),
    "delta-wrong": ("const float delta = xi / (float)N;", "const float delta = xi / (float)(N + 1);"),
    "mesh-wrong-cube-corner": ("int c[3] = {-(s & 1), -((s >> 1) & 1), -((s >> 2) & 1)};",
                               "int c[3] = {-(s & 1), -((s >> 1) & 1), -((s >> 1) & 1)};"),
    "mesh-anti-diagonal": ("v[m][perm[t][m - 1]] += 1;",
                           "v[m][perm[t][m - 1]] += (perm[t][m - 1] == 2 && m == 1) ? -1 : 1;"),
    "join-threshold": ("if (cL >= 2) t |= T_JOIN;", "if (cL >= 3) t |= T_JOIN;"),
    "lossless-skipped": ("            } else {\n                g[x] = floor_x;",
                         "            } else {\n                g[x] = g[x] - delta;"),
}


def _mesh_ok():
    off, edges = oracle.mesh()
    assert {tuple(int(c) for c in o) for o in off} == set(T.OFFSETS)
    assert len(edges) == 36


def _golden_ok():
    for name in ("cascade_1d.txt", "lossless_1d.txt", "stuck_1d.txt"):
        c = read_golden(name)
        dims = tuple(int(x) for x in c["dims"])
        f = np.array([float(x) for x in c["f"]], np.float32)
        fh = np.array([float(x) for x in c["fhat"]], np.float32)
        r = oracle.correct(f, fh, float(c["xi"][0]), dims=dims, N=int(c["N"][0]), max_iters=200)
        assert np.array_equal(r["g"], np.array([float(x) for x in c["g"]], np.float32))
        assert r["iterations"] == int(c["iterations"][0])
        assert r["status"] == int(c["status"][0])


def _classify_ok():
    rng = np.random.default_rng(2)
    for dims in [(6, 5, 4), (7, 7, 1)]:
        h = rng.integers(0, 4, int(np.prod(dims))).astype(np.float32)
        up, dn, ty = oracle.classify(h, dims)
        c = T.classify(T.Grid(dims), h)
        assert np.array_equal(up, c["up"]) and np.array_equal(dn, c["down"])
        assert np.array_equal(ty, c["type"])


def _fields_ok():
    for dims, seed, recipe, rel in [((10, 9, 8), 3, "quantised", 1e-2),
                                    ((12, 11, 10), 4, "uniform", 1e-2),
                                    ((16, 16, 1), 5, "quantised", 3e-2)]:
        f, fh, xi = synth.make_case("bumps", dims, seed, rel, recipe, n_bumps=6, sigma=(1.5, 3.0))
        f, fh = f.numpy().reshape(-1), fh.numpy().reshape(-1)
        r = oracle.correct(f, fh, xi, dims=dims, max_iters=500)
        assert r["status"] == oracle.CONVERGED
        check_fixpoint(f, fh, xi, 5, r["g"], r["k"], r["status"], r["residual"], dims)
        assert T.recalls(T.Grid(dims), f, r["g"]) == dict(cp=1.0, eg=1.0, ct=1.0)


def _detected() -> bool:
    for check in (_mesh_ok, _golden_ok, _classify_ok, _fields_ok):
        try:
            check()
        except (AssertionError, ValueError):
            return True
    return False


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, monkeypatch):
    with mutant(monkeypatch, name, *MUTANTS[name]):
        assert _detected(), f"planted mistake {name!r} passed every pin"


def test_unmutated_copy_passes():
    assert not _detected()
