"""Pins of the oracle's critical-point classification and CP order (Sec. 3.2,
Sec. 4.3): hand-classified vertices, an independent Python classifier,
union-find sublevel components, and numpy lexsort for the sorted order."""
import numpy as np
import pytest

import oracle
from oracle import topology as T
from conftest import read_golden_cases


def test_hand_classified_vertices():
    for name, c in read_golden_cases("classify_hand.txt").items():
        dims = tuple(int(x) for x in c["dims"])
        h = np.array([float(x) for x in c["values"]], np.float32)
        v = int(c["vertex"][0])
        _, _, ty = oracle.classify(h, dims)
        assert ty[v] == int(c["type"][0]), name


@pytest.mark.parametrize("dims", [(6, 5, 4), (7, 7, 1), (9, 1, 1), (4, 4, 4), (1, 5, 6)])
@pytest.mark.parametrize("levels", [3, 1000])
def test_against_independent_classifier(dims, levels):
    rng = np.random.default_rng(levels + sum(dims))
    n = int(np.prod(dims))
    h = rng.integers(0, levels, n).astype(np.float32)
    up, dn, ty = oracle.classify(h, dims)
    c = T.classify(T.Grid(dims), h)
    assert np.array_equal(up, c["up"])
    assert np.array_equal(dn, c["down"])
    assert np.array_equal(ty, c["type"])


def test_negative_zero_equals_zero():
    # IEEE compare: -0 == +0, so the index decides, exactly as for equal values
    dims = (4, 3, 2)
    rng = np.random.default_rng(5)
    h = rng.choice(np.array([0.0, -0.0, 1.0], np.float32), 24)
    h2 = np.abs(h)
    for a, b in zip(oracle.classify(h, dims), oracle.classify(h2, dims)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("seed", range(4))
def test_union_find_agrees_with_link_components(seed):
    """Sweeping vertices up in order, a vertex with no lower neighbour starts a
    sublevel component iff it is a minimum, and a vertex merging two or more
    sublevel components must have a disconnected lower link (a join saddle)."""
    dims = (6, 6, 5)
    rng = np.random.default_rng(seed)
    n = int(np.prod(dims))
    h = rng.integers(0, 6, n).astype(np.float32)
    _, _, ty = oracle.classify(h, dims)
    grid = T.Grid(dims)
    r = T.ranks(h)
    parent = {}

    def find(a):
        while parent[a] != a:
            a = parent[a]
        return a

    for v in np.argsort(r, kind="stable"):
        v = int(v)
        roots = {find(u) for u in grid.neighbours(v) if u in parent}
        parent[v] = v
        assert (len(roots) == 0) == bool(ty[v] & oracle.T_MIN)
        if len(roots) >= 2:
            assert ty[v] & oracle.T_JOIN
        for q in roots:
            parent[q] = v


def test_constant_field_has_two_critical_points():
    for dims in [(3, 3, 3), (5, 4, 1), (7, 1, 1)]:
        h = np.full(int(np.prod(dims)), 3.5, np.float32)
        _, _, ty = oracle.classify(h, dims)
        n = h.size
        assert ty[0] == oracle.T_MIN and ty[n - 1] == oracle.T_MAX
        assert np.count_nonzero(ty) == 2


@pytest.mark.parametrize("levels", [4, 100000])
def test_cp_order_is_value_then_index(levels):
    dims = (7, 6, 5)
    rng = np.random.default_rng(levels)
    h = rng.integers(0, levels, int(np.prod(dims))).astype(np.float32)
    o = oracle.cp_order(h, dims)
    _, _, ty = oracle.classify(h, dims)
    cps = np.nonzero(ty)[0]
    expect = cps[np.lexsort((cps, h[cps]))]
    assert np.array_equal(o, expect)
