"""Pins of the oracle's original event constraints (Sec. 4.2: saddle ordering,
C2, and merge / split events of the extremum graph, C3) and of the elder-rule
branch decomposition used to check them.

* branch pairs: a 1D field paired by hand; on random fields every pair is an
  extremum and a saddle of the independent classifier, one pair per extremum
  but the global one;
* worked examples on two- and three-well fields, each request set derived by
  hand from the rule: the join saddle's selection is the larger minimum, the
  split saddle's the smaller maximum, and a swap of two minima that no saddle
  pairs is left alone (while the reformulated constraints of Sec. 4.3 request
  it);
* corrections: every field converges, the fixpoint invariants hold with the
  saddle order in place of the full critical-point order, the brute-force
  merge trees and extremum graphs of f and g agree, and so does the extremum
  each saddle selects over the extremum graph of f;
* planted mistakes in the event rules each fail one of the above.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import topology as T
from fixpoint import check_fixpoint
from mutant_util import mutant


def _wells(nx, ny, wells):
    """Sum of negative Gaussian wells (centre x, depth) along the row y = 3."""
    x, y = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    f = np.zeros((ny, nx))
    for cx, depth in wells:
        f -= depth * np.exp(-((x - cx) ** 2 + (y - 3) ** 2) / 4.0)
    return f.astype(np.float32).reshape(-1), (nx, ny, 1)


def _requested(f, g, dims, events=True):
    req, cnt = oracle.requests(f, g, dims, events=events)
    assert cnt == int(req.sum())
    return set(int(v) for v in np.nonzero(req)[0])


# ----------------------------------------------------------------- branch pairs

def test_branch_pairs_by_hand_1d():
    # f = 3 0 2 1 4: minima 1, 3 meet at 2 (the younger, 3, dies there);
    # maxima 0, 2, 4: 2 dies where it meets 4's component (vertex 3), then 0 at 1
    f = np.array([3, 0, 2, 1, 4], np.float32)
    assert T.branch_pairs(T.Grid((5, 1, 1)), f) == {("j", 3, 2), ("s", 2, 3), ("s", 0, 1)}


@pytest.mark.parametrize("dims,seed", [((9, 8, 7), 1), ((17, 15, 1), 2), ((40, 1, 1), 3)])
def test_branch_pairs_invariants(dims, seed):
    h = np.random.default_rng(seed).integers(0, 6, int(np.prod(dims))).astype(np.float32)
    G = T.Grid(dims)
    ty = T.classify(G, h)["type"]
    pairs = T.branch_pairs(G, h)
    join = [(b, s) for k, b, s in pairs if k == "j"]
    split = [(b, s) for k, b, s in pairs if k == "s"]
    assert len(join) == int(np.count_nonzero(ty & oracle.T_MIN)) - 1
    assert len(split) == int(np.count_nonzero(ty & oracle.T_MAX)) - 1
    # in 1D a link is two points, so a merge vertex is typed as the extremum
    line = dims[1] == dims[2] == 1
    jt, st = (oracle.T_MAX, oracle.T_MIN) if line else (oracle.T_JOIN, oracle.T_SPLIT)
    assert all(ty[b] & oracle.T_MIN and ty[s] & jt for b, s in join)
    assert all(ty[b] & oracle.T_MAX and ty[s] & st for b, s in split)
    assert len({b for b, _ in join}) == len(join) and len({b for b, _ in split}) == len(split)


# ------------------------------------------------------------- worked examples

def test_two_wells_field_layout():
    f, dims = _wells(13, 7, [(3, 1.0), (9, 0.8)])
    _, _, ty = oracle.classify(f, dims)
    assert ty[42] == oracle.T_MIN and ty[48] == oracle.T_MIN
    assert ty[45] & oracle.T_JOIN
    assert ("j", 48, 45) in T.branch_pairs(T.Grid(dims), f)


def test_join_event_requests_the_g_selection():
    # EGP pairs the join saddle 45 with the larger of its minima, 48 (-0.8 vs
    # -1.0).  Sinking 48 below 42 makes 42 the larger in g: C3 requests 42.
    f, dims = _wells(13, 7, [(3, 1.0), (9, 0.8)])
    g = f.copy()
    g[48] = -1.2
    assert _requested(f, g, dims) == {42}


def test_split_event_requests_the_f_selection():
    # -f: maxima 42 (1.0) and 48 (0.8); EGP pairs the split saddle 45 with the
    # smaller, 48.  Raising 48 above 42 makes 42 the smaller in g: C3 requests
    # 48, the f-selection, which lies below 42 in f.
    f, dims = _wells(13, 7, [(3, 1.0), (9, 0.8)])
    h = -f
    g = h.copy()
    g[48] = 1.2
    assert _requested(h, g, dims) == {48}


def test_saddle_order_requests_the_lower_in_f():
    # saddles in f order: 45 (-0.190) < 3 (-0.105) < ...; sinking the boundary
    # saddle 3 to -0.2 keeps every neighbour relation but reverses the pair
    f, dims = _wells(13, 7, [(3, 1.0), (9, 0.8)])
    g = f.copy()
    g[3] = -0.2
    assert _requested(f, g, dims) == {45}


def test_unpaired_minima_order_is_free():
    # wells A = 60 (-0.9), B = 66 (-1.0), C = 72 (-0.8); saddle 63 pairs A,
    # saddle 69 pairs C.  C sunk between B and A keeps both selections: no event
    # request, while the reformulated constraint on the sorted critical points
    # requests A, the lower of the reversed pair (A, C).
    f, dims = _wells(19, 7, [(3, 0.9), (9, 1.0), (15, 0.8)])
    assert {p for p in T.branch_pairs(T.Grid(dims), f) if p[0] == "j"} == {("j", 60, 63), ("j", 72, 69)}
    g = f.copy()
    g[72] = -0.95
    assert _requested(f, g, dims) == set()
    assert _requested(f, g, dims, events=False) == {60}


# ----------------------------------------------------------------- corrections

FIELDS = [((24, 20, 1), 6, "uniform", 2e-2), ((16, 16, 1), 5, "quantised", 3e-2),
          ((32, 28, 1), 13, "quantised", 5e-2), ((14, 13, 12), 14, "quantised", 3e-2),
          ((18, 16, 14), 17, "uniform", 4e-2)]


def _correct(dims, seed, recipe, rel):
    f, fh, xi = synth.make_case("bumps", dims, seed, rel, recipe, n_bumps=8, sigma=(1.5, 3.0))
    f, fh = f.numpy().reshape(-1), fh.numpy().reshape(-1)
    return f, fh, xi, oracle.correct(f, fh, xi, dims=dims, events=True)


def _fields_ok():
    for dims, seed, recipe, rel in FIELDS:
        f, fh, xi, r = _correct(dims, seed, recipe, rel)
        assert r["status"] == oracle.CONVERGED
        check_fixpoint(f, fh, xi, 5, r["g"], r["k"], r["status"], r["residual"], dims, events=True)
        G = T.Grid(dims)
        assert T.recalls(G, f, r["g"]) == dict(cp=1.0, eg=1.0, ct=1.0)
        eg = T.extremum_graph(G, f)
        assert T.event_selections(eg, f) == T.event_selections(eg, r["g"])


def test_corrections_preserve_events():
    _fields_ok()


def test_reformulated_corrections_preserve_branch_pairs():
    # the full critical-point order (Sec. 4.3) also fixes which extremum each
    # saddle is paired with by the elder rule; the event constraints fix the
    # selections over the extremum graph only
    for dims, seed, recipe, rel in FIELDS:
        f, fh, xi = synth.make_case("bumps", dims, seed, rel, recipe, n_bumps=8, sigma=(1.5, 3.0))
        f, fh = f.numpy().reshape(-1), fh.numpy().reshape(-1)
        r = oracle.correct(f, fh, xi, dims=dims)
        G = T.Grid(dims)
        assert T.branch_pairs(G, f) == T.branch_pairs(G, r["g"])


def test_fhat_equal_f_needs_no_pass():
    f, fh, xi = synth.make_case("bumps", (12, 11, 10), 4, 1e-2, "uniform", n_bumps=6, sigma=(1.5, 3.0))
    f = f.numpy().reshape(-1)
    r = oracle.correct(f, f, xi, dims=(12, 11, 10), events=True)
    assert r["iterations"] == 0 and r["status"] == oracle.CONVERGED and r["n_edits"] == 0


# ------------------------------------------------------------ planted mistakes

EVENT_MUTANTS = {
    "C3-join-dropped": ("        if (best != C->sel_min[q]) mark(req, C->inc ? C->sel_min[q] : best);",
                        "        if (0 && best != C->sel_min[q]) mark(req, C->inc ? C->sel_min[q] : best);"),
    "C3-join-targets-f-selection": ("mark(req, C->inc ? C->sel_min[q] : best);",
                                    "mark(req, C->inc ? C->sel_min[q] : C->sel_min[q]);"),
    "C3-split-dropped": ("        if (best != C->sel_max[q]) mark(req, C->inc ? best : C->sel_max[q]);",
                         "        if (0 && best != C->sel_max[q]) mark(req, C->inc ? best : C->sel_max[q]);"),
    "C3-split-targets-g-selection": ("mark(req, C->inc ? best : C->sel_max[q]);", "mark(req, C->inc ? best : best);"),
    "C2-dropped": ("    if (prec(g, b, a)) mark(req, C->inc ? b : a);\n}\n\n/* C3",
                   "    if (0 && prec(g, b, a)) mark(req, C->inc ? b : a);\n}\n\n/* C3"),
    "EGP-selects-smallest-minimum": (
        "                    if (prec(C->f, best, e[i])) best = e[i];\n                C->sel_min[q] = best;",
        "                    if (prec(C->f, e[i], best)) best = e[i];\n                C->sel_min[q] = best;"),
    "EG-join-paths-ascend": ("const int64_t m = path_end(C->dnf, end_dn, nb[j]);",
                             "const int64_t m = path_end(C->upf, end_dn, nb[j]);"),
    "EG-split-paths-from-below": ("                if (!prec(C->f, s, nb[j])) continue;",
                                  "                if (!prec(C->f, nb[j], s)) continue;"),
    "EG-path-memo-keeps-first-step": ("        end[w] = m;\n        if (w == u) break;",
                                      "        end[w] = step[w];\n        if (w == u) break;"),
}


def _detected() -> bool:
    checks = (test_branch_pairs_by_hand_1d, test_join_event_requests_the_g_selection,
              test_split_event_requests_the_f_selection, test_saddle_order_requests_the_lower_in_f,
              test_unpaired_minima_order_is_free, _fields_ok)
    for check in checks:
        try:
            check()
        except (AssertionError, ValueError):
            return True
    return False


@pytest.mark.parametrize("name", sorted(EVENT_MUTANTS))
def test_planted_event_mistake_is_caught(name, monkeypatch):
    with mutant(monkeypatch, name, *EVENT_MUTANTS[name]):
        assert _detected(), f"planted mistake {name!r} passed every pin"
