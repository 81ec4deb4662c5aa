"""Brute-force topology tools for tiny fields -- TEST INFRASTRUCTURE ONLY.

These are deliberately independent of ``exactz_oracle.c``: the mesh here comes
from the closed-form description of the Freudenthal triangulation (two grid
vertices are adjacent iff their difference is a non-zero vector whose
components are all in {0, 1} or all in {0, -1}), the order is a numpy lexsort
on (value, index), and the structures are built from their definitions:

* critical points by link components (Sec. 3.2, Step 1);
* extremum graphs by following steepest-descent / -ascent integral paths from
  the neighbours of every saddle (Sec. 3.1, Sec. 3.2 Step 1);
* join / split trees by a union-find sweep of the sublevel / superlevel sets
  (Sec. 3.1, merge trees; the contour tree is their combination), and their
  branch decompositions by the elder rule of the same sweep (the pairs that
  Extremum Graph Pairing extracts, Sec. 3.2 Step 2);
* weak / strong / reduced vulnerability graphs and the longest path D_max of
  Thm. 4.1 (Sec. 4.4).
Pure Python loops: use on fields of at most a few thousand vertices.
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Set, Tuple

import numpy as np

OFFSETS = [d for d in itertools.product((-1, 0, 1), repeat=3)
           if d != (0, 0, 0) and (all(c >= 0 for c in d) or all(c <= 0 for c in d))]
_OFFSET_SET = set(OFFSETS)


def link_edges_by_rule() -> List[Tuple[int, int]]:
    """Edges (a, b) of the interior link: b - a is itself a neighbour offset."""
    out = []
    for a in range(len(OFFSETS)):
        for b in range(a + 1, len(OFFSETS)):
            d = tuple(OFFSETS[b][c] - OFFSETS[a][c] for c in range(3))
            if d in _OFFSET_SET:
                out.append((a, b))
    return out


class Grid:
    def __init__(self, dims):
        self.nx, self.ny, self.nz = (int(d) for d in dims)
        self.n = self.nx * self.ny * self.nz
        nb = np.full((self.n, len(OFFSETS)), -1, np.int64)
        for v in range(self.n):
            x, y, z = v % self.nx, (v // self.nx) % self.ny, v // (self.nx * self.ny)
            for s, (dx, dy, dz) in enumerate(OFFSETS):
                X, Y, Z = x + dx, y + dy, z + dz
                if 0 <= X < self.nx and 0 <= Y < self.ny and 0 <= Z < self.nz:
                    nb[v, s] = X + self.nx * (Y + self.ny * Z)
        self.nb = nb
        self.adj = np.zeros((len(OFFSETS), len(OFFSETS)), bool)
        for a, b in link_edges_by_rule():
            self.adj[a, b] = self.adj[b, a] = True

    def neighbours(self, v):
        return [int(u) for u in self.nb[v] if u >= 0]


def ranks(h: np.ndarray) -> np.ndarray:
    """Position of every vertex in the order by (value, index)."""
    h = np.asarray(h, np.float32).reshape(-1)
    # +0.0 / -0.0 compare equal; lexsort on float values already treats them equal
    # only if they sort as equal, so normalise the sign of zero first.
    hv = np.where(h == 0, np.float32(0), h)
    order = np.lexsort((np.arange(h.size), hv))
    r = np.empty(h.size, np.int64)
    r[order] = np.arange(h.size)
    return r


def _components(adj, slots: List[int]) -> int:
    slots = list(slots)
    seen = set()
    c = 0
    for s in slots:
        if s in seen:
            continue
        c += 1
        stack = [s]
        seen.add(s)
        while stack:
            u = stack.pop()
            for t in slots:
                if t not in seen and adj[u, t]:
                    seen.add(t)
                    stack.append(t)
    return c


def classify(grid: Grid, h) -> Dict[str, np.ndarray]:
    """up/down (steepest vertex of the closed neighbourhood), cL, cU, type bits."""
    r = ranks(h)
    n = grid.n
    up = np.arange(n)
    dn = np.arange(n)
    cL = np.zeros(n, np.int64)
    cU = np.zeros(n, np.int64)
    ty = np.zeros(n, np.uint8)
    for v in range(n):
        lows, highs = [], []
        for s in range(len(OFFSETS)):
            u = grid.nb[v, s]
            if u < 0:
                continue
            if r[u] > r[up[v]]:
                up[v] = u
            if r[u] < r[dn[v]]:
                dn[v] = u
            (lows if r[u] < r[v] else highs).append(s)
        cL[v] = _components(grid.adj, lows)
        cU[v] = _components(grid.adj, highs)
        if cL[v] == 0:
            ty[v] = 1
        elif cU[v] == 0:
            ty[v] = 2
        else:
            ty[v] = (4 if cL[v] >= 2 else 0) | (8 if cU[v] >= 2 else 0)
    return dict(up=up, down=dn, cL=cL, cU=cU, type=ty, rank=r)


def extremum_graph(grid: Grid, h) -> Set[Tuple[int, int, str]]:
    """Edges (saddle, extremum, 'join'|'split'): a join saddle s reaches minimum
    m if the steepest-descent path from some lower neighbour of s ends at m;
    split saddles likewise reach maxima by steepest ascent."""
    c = classify(grid, h)
    r = c["rank"]
    up, dn, ty = c["up"], c["down"], c["type"]
    edges = set()
    for s in range(grid.n):
        if ty[s] & 4:
            for u in grid.neighbours(s):
                if r[u] < r[s]:
                    v = u
                    while dn[v] != v:
                        v = int(dn[v])
                    edges.add((s, v, "join"))
        if ty[s] & 8:
            for u in grid.neighbours(s):
                if r[u] > r[s]:
                    v = u
                    while up[v] != v:
                        v = int(up[v])
                    edges.add((s, v, "split"))
    return edges


def _merge_tree(grid: Grid, r: np.ndarray, ascending: bool) -> Set[Tuple[int, int]]:
    order = np.argsort(r if ascending else -r, kind="stable")
    parent = {}
    node = {}

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    arcs = set()
    for v in order:
        v = int(v)
        roots = {find(u) for u in grid.neighbours(v) if u in parent}
        parent[v] = v
        if not roots:
            node[v] = v
            continue
        if len(roots) >= 2:
            for q in roots:
                arcs.add((node[q], v))
        for q in roots:
            parent[q] = v
        node[v] = v if len(roots) >= 2 else node[next(iter(roots))]
    return arcs


def join_tree(grid: Grid, h) -> Set[Tuple[int, int]]:
    """Arcs of the join tree (sublevel sets merging), as (lower node, merge vertex)."""
    return _merge_tree(grid, ranks(h), ascending=True)


def split_tree(grid: Grid, h) -> Set[Tuple[int, int]]:
    """Arcs of the split tree (superlevel sets merging when sweeping down)."""
    return _merge_tree(grid, ranks(h), ascending=False)


def _branch_pairs(grid: Grid, r: np.ndarray, ascending: bool) -> Set[Tuple[int, int]]:
    """Elder rule on the sweep: where components meet, the one born at the
    oldest extremum (lowest rank going up, highest going down) survives and every
    other is paired with the meeting vertex as (its birth extremum, vertex)."""
    order = np.argsort(r if ascending else -r, kind="stable")
    key = r if ascending else -r
    parent = {}
    birth = {}

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    pairs = set()
    for v in order:
        v = int(v)
        roots = {find(u) for u in grid.neighbours(v) if u in parent}
        parent[v] = v
        if not roots:
            birth[v] = v
            continue
        elder = min(roots, key=lambda q: key[birth[q]])
        if len(roots) >= 2:
            for q in roots:
                if q != elder:
                    pairs.add((birth[q], v))
        for q in roots:
            parent[q] = v
        birth[v] = birth[elder]
    return pairs


def branch_pairs(grid: Grid, h) -> Set[Tuple[str, int, int]]:
    """Branches of the join ('j': minimum, join saddle) and split ('s': maximum,
    split saddle) trees, as extracted by Extremum Graph Pairing."""
    r = ranks(h)
    return ({("j",) + p for p in _branch_pairs(grid, r, True)} |
            {("s",) + p for p in _branch_pairs(grid, r, False)})


def event_selections(eg, h) -> Dict[Tuple[str, int], int]:
    """The two selections of the merge / split event constraints (Sec. 4.2,
    C3) over the links of extremum graph eg, ranked by h: per saddle with two
    or more linked extrema, its largest minimum ('join') or smallest maximum
    ('split'); per extremum, its lowest join saddle ('min') or highest split
    saddle ('max')."""
    r = ranks(h)
    by_saddle: Dict[Tuple[str, int], Set[int]] = {}
    by_ext: Dict[Tuple[str, int], Set[int]] = {}
    for s, e, kind in eg:
        by_saddle.setdefault((kind, s), set()).add(e)
        by_ext.setdefault(("min" if kind == "join" else "max", e), set()).add(s)
    out = {}
    for (kind, s), es in by_saddle.items():
        if len(es) >= 2:
            pick = max if kind == "join" else min
            out[(kind, s)] = pick(es, key=lambda v: r[v])
    for (kind, e), ss in by_ext.items():
        pick = min if kind == "min" else max
        out[(kind, e)] = pick(ss, key=lambda v: r[v])
    return out


def recalls(grid: Grid, f, g) -> Dict[str, float]:
    """CP / EG / CT recall of g against f (Sec. 5.1 metrics)."""
    cf, cg = classify(grid, f), classify(grid, g)
    cps = np.nonzero(cf["type"])[0]
    cp_rec = float(np.mean(cg["type"][cps] == cf["type"][cps])) if cps.size else 1.0
    ef, eg = extremum_graph(grid, f), extremum_graph(grid, g)
    eg_rec = len(ef & eg) / len(ef) if ef else 1.0
    tf = {("j",) + a for a in join_tree(grid, f)} | {("s",) + a for a in split_tree(grid, f)}
    tg = {("j",) + a for a in join_tree(grid, g)} | {("s",) + a for a in split_tree(grid, g)}
    ct_rec = len(tf & tg) / len(tf) if tf else 1.0
    return dict(cp=cp_rec, eg=eg_rec, ct=ct_rec)


def compared_pairs(grid: Grid, f, literal: bool = False) -> Set[Tuple[int, int]]:
    """Unordered pairs of vertices whose order some rule compares.

    literal=True  (paper-literal reading of "adjacent"): mesh edges plus pairs
                  of critical points adjacent in f's sorted order.
    literal=False (rule-complete reading): any two members of one closed
                  neighbourhood (rule R1 compares the steepest candidates of a
                  star, which need not be mesh-adjacent), plus the same
                  critical-point pairs.
    """
    pairs = set()
    for v in range(grid.n):
        nb = grid.neighbours(v)
        if literal:
            for u in nb:
                pairs.add((min(u, v), max(u, v)))
        else:
            star = nb + [v]
            for a, b in itertools.combinations(star, 2):
                pairs.add((min(a, b), max(a, b)))
    c = classify(grid, f)
    cps = [int(v) for v in np.nonzero(c["type"])[0]]
    cps.sort(key=lambda v: c["rank"][v])
    for a, b in zip(cps, cps[1:]):
        pairs.add((min(a, b), max(a, b)))
    return pairs


def vulnerability(grid: Grid, f, fhat, xi: float, literal: bool = False) -> Dict[str, object]:
    """G_V, G_S, G_R and D_max (longest path, counted in vertices, from a seed
    endpoint) of Sec. 4.4.  Edges point from the higher to the lower vertex in f.
    G_S keeps u->v when f_hat_v >= fl(f_u - xi) (u can still be lowered to v);
    seeds are G_S edges already flipped in f_hat."""
    f = np.asarray(f, np.float32).reshape(-1)
    fhat = np.asarray(fhat, np.float32).reshape(-1)
    rf, rh = ranks(f), ranks(fhat)
    xi32 = np.float32(xi)
    floor = (f - xi32).astype(np.float32)
    ev, es, seeds = [], [], []
    thr = 2.0 * float(xi) * (1 + 1e-6) + 4 * float(np.spacing(np.float32(np.max(np.abs(f)) + xi)))
    for a, b in compared_pairs(grid, f, literal):
        u, v = (a, b) if rf[a] > rf[b] else (b, a)
        if abs(float(f[u]) - float(f[v])) <= thr:
            ev.append((u, v))
        if fhat[v] >= floor[u]:
            es.append((u, v))
            if rh[u] < rh[v]:
                seeds.append((u, v))
    seed_nodes = {x for e in seeds for x in e}
    out_edges: Dict[int, List[int]] = {}
    for u, v in es:
        out_edges.setdefault(u, []).append(v)
    # reachable from the seed endpoints in G_S
    reach = set(seed_nodes)
    stack = list(seed_nodes)
    while stack:
        u = stack.pop()
        for v in out_edges.get(u, []):
            if v not in reach:
                reach.add(v)
                stack.append(v)
    # longest path in vertices, processing vertices from high to low f (topological)
    dep = {v: 1 for v in seed_nodes}
    for u in sorted(reach, key=lambda x: -rf[x]):
        if u not in dep:
            continue
        for v in out_edges.get(u, []):
            if v in reach and dep.get(v, 0) < dep[u] + 1:
                dep[v] = dep[u] + 1
    dmax = max(dep.values()) if dep else 0
    gv_nodes = {x for e in ev for x in e}
    gs_nodes = {x for e in es for x in e}
    return dict(GV=len(gv_nodes), GS=len(gs_nodes), GR=len(reach), seeds=len(seeds), Dmax=dmax)
