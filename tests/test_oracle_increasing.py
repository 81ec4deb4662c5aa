"""Pins of the oracle's increasing-edit mode (the paper's framework supports
increasing as well as decreasing monotone edits, Sec. 4.2; edits of Sec. 3.3
mirrored: g <- fl(g + Delta) up to the lossless bound fl(f + xi), every rule
raising the vertex that must be higher).

* the point-reflection / negation identity: with R the reflection v -> n-1-v
  (which maps the Freudenthal mesh onto itself and reverses the index order,
  so that negating the values reverses the simulation-of-simplicity order),
  the increasing correction of (f, f_hat) equals -R of the decreasing
  correction of (-R f, -R f_hat) in every output, for both constraint sets;
* the hand-derived 1D runs, mirrored;
* fixpoint invariants and the brute-force topology of increasing results;
* planted mistakes in the increasing branches each fail one of the above.
"""
import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden
from oracle import topology as T
from mutant_util import mutant


def _mirror(a):
    return (-np.asarray(a, np.float32).reshape(-1)[::-1]).astype(np.float32)


def _same_mirrored(inc, dec, N):
    # -R of the decreasing result; signed zeros compare equal (the order treats them alike)
    assert np.array_equal(inc["g"], _mirror(dec["g"]))
    assert np.array_equal(inc["k"], dec["k"][::-1])
    for key in ("iterations", "status", "residual", "n_edits", "n_lossless"):
        assert inc[key] == dec[key], key
    # an increasing edit never produces -0 (g + Delta, f + xi with positive Delta, xi)
    edited = inc["k"] > 0
    assert not np.any(np.signbit(inc["g"][edited]) & (inc["g"][edited] == 0))


FIELDS = [((24, 20, 1), 6, "uniform", 2e-2), ((14, 13, 12), 14, "quantised", 3e-2),
          ((18, 16, 14), 17, "uniform", 4e-2), ((40, 1, 1), 7, "uniform", 5e-2), ((10, 9, 8), 3, "quantised", 1e-2)]


def _case(dims, seed, recipe, rel):
    f, fh, xi = synth.make_case("bumps", dims, seed, rel, recipe, n_bumps=8, sigma=(1.5, 3.0))
    return f.numpy().reshape(-1), fh.numpy().reshape(-1), xi


def _identity_ok(events):
    for dims, seed, recipe, rel in FIELDS:
        f, fh, xi = _case(dims, seed, recipe, rel)
        inc = oracle.correct(f, fh, xi, dims=dims, events=events, increasing=True)
        dec = oracle.correct(_mirror(f), _mirror(fh), xi, dims=dims, events=events)
        _same_mirrored(inc, dec, 5)


@pytest.mark.parametrize("events", [False, True])
def test_reflection_identity(events):
    _identity_ok(events)


def test_heavy_ties_identity():
    dims = (37, 11, 9)
    rng = np.random.default_rng(5)
    n = int(np.prod(dims))
    f = rng.integers(0, 5, n).astype(np.float32)
    xi = 0.75
    fh = np.clip(f + rng.integers(-1, 2, n).astype(np.float32) * np.float32(0.5), f - np.float32(xi),
                 f + np.float32(xi)).astype(np.float32)
    for events in (False, True):
        inc = oracle.correct(f, fh, xi, dims=dims, events=events, increasing=True)
        dec = oracle.correct(_mirror(f), _mirror(fh), xi, dims=dims, events=events)
        _same_mirrored(inc, dec, 5)


def _golden_ok():
    for name in ("cascade_1d.txt", "lossless_1d.txt", "stuck_1d.txt"):
        c = read_golden(name)
        dims = tuple(int(x) for x in c["dims"])
        arr = lambda key: np.array([float(x) for x in c[key]], np.float32)  # noqa: E731
        N = int(c["N"][0])
        r = oracle.correct(_mirror(arr("f")), _mirror(arr("fhat")), float(c["xi"][0]), dims=dims, N=N,
                           increasing=True)
        assert np.array_equal(r["g"], _mirror(arr("g")))
        assert np.array_equal(r["k"], np.array([int(x) for x in c["k"]], np.uint8)[::-1])
        assert r["iterations"] == int(c["iterations"][0]) and r["status"] == int(c["status"][0])


def test_golden_runs_mirrored():
    _golden_ok()


def _fixpoint_ok():
    for dims, seed, recipe, rel in FIELDS[:3]:
        f, fh, xi = _case(dims, seed, recipe, rel)
        N = 5
        r = oracle.correct(f, fh, xi, dims=dims, increasing=True)
        g, k = r["g"], r["k"]
        ceil = (f + np.float32(xi)).astype(np.float32)
        assert np.all(g >= fh) and np.all(g <= ceil)
        # replay: k increments of Delta from f_hat, or the bound fl(f + xi)
        assert np.array_equal(oracle.decode_stream(fh, k, ceil[k == N + 1], xi, N, increasing=True), g)
        if r["status"] == oracle.CONVERGED:
            _, cnt = oracle.requests(f, g, dims, increasing=True)
            assert cnt == 0
            assert T.recalls(T.Grid(dims), f, g) == dict(cp=1.0, eg=1.0, ct=1.0)


def test_fixpoint_and_topology():
    _fixpoint_ok()


INC_MUTANTS = {
    "inc-R1-up-raises-g-max": ("mark(req, C->inc ? C->upf[p] : upg);", "mark(req, C->inc ? upg : upg);"),
    "inc-R1-down-raises-f-min": ("mark(req, C->inc ? dng : C->dnf[p]);",
                                 "mark(req, C->inc ? C->dnf[p] : C->dnf[p]);"),
    "inc-R2-raises-lower": ("mark(req, (below_f != C->inc) ? nb[j] : p);", "mark(req, below_f ? nb[j] : p);"),
    "inc-R3-raises-lower": ("C->o[q + 1];\n    if (prec(g, b, a)) mark(req, C->inc ? b : a);",
                            "C->o[q + 1];\n    if (prec(g, b, a)) mark(req, C->inc ? a : a);"),
    "inc-bound-below": ("float floor_x = inc ? f[x] + xi : f[x] - xi;", "float floor_x = inc ? f[x] - xi : f[x] - xi;"),
    "inc-step-down": ("float t = inc ? g[x] + delta : g[x] - delta;", "float t = inc ? g[x] - delta : g[x] - delta;"),
    "inc-C3-join-raises-g-selection": ("mark(req, C->inc ? C->sel_min[q] : best);", "mark(req, C->inc ? best : best);"),
    "inc-C3-split-raises-f-selection": ("mark(req, C->inc ? best : C->sel_max[q]);",
                                        "mark(req, C->inc ? C->sel_max[q] : C->sel_max[q]);"),
}


def _detected() -> bool:
    for check in (lambda: _identity_ok(False), lambda: _identity_ok(True), _golden_ok, _fixpoint_ok):
        try:
            check()
        except (AssertionError, ValueError):
            return True
    return False


@pytest.mark.parametrize("name", sorted(INC_MUTANTS))
def test_planted_mistake_is_caught(name, monkeypatch):
    with mutant(monkeypatch, name, *INC_MUTANTS[name]):
        assert _detected(), f"planted mistake {name!r} passed every pin"
