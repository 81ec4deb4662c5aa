"""Pins of the oracle's mesh (the Freudenthal triangulation, Sec. 3 PL field).

The oracle derives neighbours and link edges from explicit tetrahedra; these
tests compare that with the closed-form description (offsets with all
components in {0,1} or all in {0,-1}; a link edge joins two neighbours whose
difference is itself an offset) and with topological facts: the link of an
interior vertex of a triangulated 3-manifold is a 2-sphere (Euler
characteristic 2), of a boundary vertex a disk (1), and in 2D a hexagon.
"""
import itertools

import numpy as np

import oracle
from oracle import topology as T


def _triangles(edges, verts):
    es = {frozenset(e) for e in edges}
    return [t for t in itertools.combinations(verts, 3)
            if all(frozenset(p) in es for p in itertools.combinations(t, 2))]


def test_offsets_match_closed_form():
    off, _ = oracle.mesh()
    assert len(off) == 14
    assert {tuple(int(c) for c in o) for o in off} == set(T.OFFSETS)


def test_link_edges_match_difference_rule():
    off, edges = oracle.mesh()
    tet = {frozenset((tuple(off[a]), tuple(off[b]))) for a, b in edges}
    rule = {frozenset((T.OFFSETS[a], T.OFFSETS[b])) for a, b in T.link_edges_by_rule()}
    assert len(tet) == 36
    assert tet == rule


def test_interior_link_is_a_sphere():
    off, edges = oracle.mesh()
    verts = list(range(len(off)))
    tris = _triangles([tuple(e) for e in edges], verts)
    assert len(tris) == 24  # 24 tetrahedra around an interior vertex
    assert len(verts) - len(edges) + len(tris) == 2
    # every link edge lies on exactly two link triangles (closed surface)
    for e in edges:
        assert sum(1 for t in tris if e[0] in t and e[1] in t) == 2


def test_boundary_links_are_disks():
    off, edges = oracle.mesh()
    for keep in ([0, 1, 2], [0, 1], [0]):  # face, edge, corner vertices
        # restrict to offsets not leaving the half-spaces x>=0 (face), x,y>=0 (edge), ...
        verts = [s for s in range(len(off)) if all(off[s][a] >= 0 for a in keep)]
        es = [tuple(e) for e in edges if e[0] in verts and e[1] in verts]
        tris = _triangles(es, verts)
        assert len(verts) - len(es) + len(tris) == 1


def test_2d_link_is_a_hexagon():
    off, edges = oracle.mesh()
    verts = [s for s in range(len(off)) if off[s][2] == 0]
    es = [tuple(e) for e in edges if e[0] in verts and e[1] in verts]
    assert len(verts) == 6 and len(es) == 6
    deg = {v: 0 for v in verts}
    for a, b in es:
        deg[a] += 1
        deg[b] += 1
    assert set(deg.values()) == {2}


def test_neighbour_sets_against_tiny_box():
    # brute force: the neighbours the oracle uses give the same steepest
    # vertices as a search over the closed-form neighbour lists
    rng = np.random.default_rng(11)
    for dims in [(2, 2, 2), (3, 2, 4), (5, 1, 3), (1, 4, 4)]:
        n = int(np.prod(dims))
        h = rng.standard_normal(n).astype(np.float32)
        up, dn, _ = oracle.classify(h, dims)
        c = T.classify(T.Grid(dims), h)
        assert np.array_equal(up, c["up"]) and np.array_equal(dn, c["down"])
