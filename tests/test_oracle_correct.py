"""Pins of the oracle's correction (Algorithm 1; Sec. 3.3, 4.2, 4.3, 4.4).

* hand-derived runs (tests/golden): exact g, k, iterations, status;
* closed forms: f_hat == f and f_hat == fl(f - xi) (no ties) need 0 passes;
* fixpoint invariants on random fields (request set empty, identical
  steepest neighbours / types / CP order, floor <= g <= f_hat, replay);
* the paper's guarantee: CP / EG / CT recall 1 by brute-force extremum graphs
  and union-find merge trees (Sec. 5.3, Obs. 5);
* the iteration bound of Thm. 4.1 with the lossless edit counted;
* worklist mode == plain mode bit for bit; input validation; the cap.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import topology as T
from conftest import read_golden
from fixpoint import check_fixpoint


def _golden(name):
    c = read_golden(name)
    dims = tuple(int(x) for x in c["dims"])
    arr = lambda key: np.array([float(x) for x in c[key]], np.float32)  # noqa: E731
    return dims, float(c["xi"][0]), int(c["N"][0]), arr("f"), arr("fhat"), c


@pytest.mark.parametrize("name", ["cascade_1d.txt", "lossless_1d.txt", "stuck_1d.txt"])
@pytest.mark.parametrize("worklist", [False, True])
def test_golden_runs(name, worklist):
    dims, xi, N, f, fhat, c = _golden(name)
    r = oracle.correct(f, fhat, xi, dims=dims, N=N, worklist=worklist)
    assert np.array_equal(r["g"], np.array([float(x) for x in c["g"]], np.float32))
    assert np.array_equal(r["k"], np.array([int(x) for x in c["k"]], np.uint8))
    assert r["iterations"] == int(c["iterations"][0])
    assert r["status"] == int(c["status"][0])
    assert r["residual"] == int(c["residual"][0])


def _case(dims, seed, recipe, rel, n_bumps=6, sigma=(1.5, 3.0), noise=0.01):
    f, fh, xi = synth.make_case("bumps", dims, seed, rel, recipe, n_bumps=n_bumps,
                                sigma=sigma, noise_std=noise)
    return f.numpy().reshape(-1), fh.numpy().reshape(-1), xi


def test_identity_needs_no_pass():
    f, _, xi = _case((9, 8, 7), 1, "uniform", 1e-2)
    r = oracle.correct(f, f, xi, dims=(9, 8, 7))
    assert r["iterations"] == 0 and r["status"] == oracle.CONVERGED and r["n_edits"] == 0


def test_all_at_floor_needs_no_pass():
    # distinct, well separated values: fl(f - xi) keeps f's strict order
    dims = (6, 5, 4)
    rng = np.random.default_rng(3)
    f = (rng.permutation(120).astype(np.float32) * np.float32(0.5))
    xi = 0.1
    fhat = (f - np.float32(xi)).astype(np.float32)
    r = oracle.correct(f, fhat, xi, dims=dims)
    assert r["iterations"] == 0 and r["n_edits"] == 0


CASES = [
    ((10, 9, 8), 3, "quantised", 1e-2),
    ((12, 11, 10), 4, "uniform", 1e-2),
    ((16, 16, 1), 5, "quantised", 3e-2),
    ((24, 20, 1), 6, "uniform", 2e-2),
    ((40, 1, 1), 7, "uniform", 5e-2),
    ((64, 1, 1), 8, "quantised", 5e-2),
    ((9, 9, 9), 9, "quantised", 5e-3),
    ((5, 13, 7), 10, "uniform", 3e-2),
]


@pytest.mark.parametrize("dims,seed,recipe,rel", CASES)
def test_fixpoint_and_topology(dims, seed, recipe, rel):
    f, fhat, xi = _case(dims, seed, recipe, rel)
    r = oracle.correct(f, fhat, xi, dims=dims)
    assert r["status"] in (oracle.CONVERGED, oracle.STUCK)
    check_fixpoint(f, fhat, xi, 5, r["g"], r["k"], r["status"], r["residual"], dims)
    grid = T.Grid(dims)
    if r["status"] == oracle.CONVERGED:
        rec = T.recalls(grid, f, r["g"])
        assert rec == dict(cp=1.0, eg=1.0, ct=1.0), rec
    # Thm. 4.1 with the lossless (N+1)-th edit, on the rule-complete graph
    vb = T.vulnerability(grid, f, fhat, xi)
    assert r["iterations"] <= 6 * vb["Dmax"]
    if vb["Dmax"] == 0:
        assert r["iterations"] == 0


@pytest.mark.parametrize("dims,seed,recipe,rel", CASES)
@pytest.mark.parametrize("N", [1, 5, 8])
def test_worklist_equals_plain(dims, seed, recipe, rel, N):
    f, fhat, xi = _case(dims, seed, recipe, rel)
    a = oracle.correct(f, fhat, xi, dims=dims, N=N)
    b = oracle.correct(f, fhat, xi, dims=dims, N=N, worklist=True)
    assert np.array_equal(a["g"].view(np.uint32), b["g"].view(np.uint32))
    assert np.array_equal(a["k"], b["k"])
    for key in ("iterations", "status", "residual"):
        assert a[key] == b[key]


def test_other_N_values_reach_fixpoints():
    f, fhat, xi = _case((10, 10, 6), 12, "quantised", 2e-2)
    for N in (1, 2, 3, 10):
        r = oracle.correct(f, fhat, xi, dims=(10, 10, 6), N=N)
        check_fixpoint(f, fhat, xi, N, r["g"], r["k"], r["status"], r["residual"], (10, 10, 6))


def test_iteration_cap():
    f, fhat, xi = _case((12, 11, 10), 4, "uniform", 1e-2)
    full = oracle.correct(f, fhat, xi, dims=(12, 11, 10))
    assert full["iterations"] > 2
    for wl in (False, True):
        r = oracle.correct(f, fhat, xi, dims=(12, 11, 10), max_iters=2, worklist=wl)
        assert r["status"] == oracle.ITER_LIMIT and r["iterations"] == 2 and r["residual"] > 0
    r0 = oracle.correct(f, fhat, xi, dims=(12, 11, 10), max_iters=0)
    assert r0["status"] == oracle.ITER_LIMIT and r0["iterations"] == 0 and r0["n_edits"] == 0


def test_input_validation():
    f = np.linspace(0, 1, 27, dtype=np.float32)
    ok = f.copy()
    assert oracle.correct_rc(f, ok, 0.1, dims=(3, 3, 3)) == 0
    bad = f.copy()
    bad[5] = np.nan
    assert oracle.correct_rc(f, bad, 0.1, dims=(3, 3, 3)) == -2
    bad = f.copy()
    bad[5] = np.inf
    assert oracle.correct_rc(bad, ok, 0.1, dims=(3, 3, 3)) == -2
    bad = f.copy()
    bad[7] += np.float32(0.2)
    assert oracle.correct_rc(f, bad, 0.1, dims=(3, 3, 3)) == -3
    assert oracle.correct_rc(f, ok, 0.0, dims=(3, 3, 3)) == -1
    assert oracle.correct_rc(f, ok, -1.0, dims=(3, 3, 3)) == -1
    assert oracle.correct_rc(f[:1], ok[:1], 0.1, dims=(1, 1, 1)) == -1


def test_generators_respect_the_bound():
    for recipe in ("quantised", "uniform"):
        f, fh, xi = synth.make_case("bumps", (20, 18, 16), 4, 1e-3, recipe)
        x = torch.tensor(xi, dtype=torch.float32)
        assert bool(((fh >= f - x) & (fh <= f + x)).all())
        assert oracle.correct_rc(f.numpy().reshape(-1), fh.numpy().reshape(-1), xi,
                                 dims=(20, 18, 16)) == 0
