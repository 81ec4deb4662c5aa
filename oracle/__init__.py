"""The oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow CPU implementation of the EXaCTz correction (Algorithm 1 with the
EG constraints of Sec. 4.2 and either the reformulated event constraints of
Sec. 4.3 or the saddle-ordering and original merge / split event constraints of
Sec. 4.2) plus brute-force topology tools (``oracle.topology``).  Only ``tests/``, the
smoke check and the benchmark's CPU-baseline leg import this package; the
library under ``paper_2604_01397_b300`` never does, and the two share no code.

Parity status per function (each pin lives under ``tests/``):
  correct       pinned: hand-computed 1D cascades (tests/golden), closed forms
                (f_hat == f, f_hat == floor), fixpoint invariants, brute-force
                extremum graphs and merge trees of the result, the iteration
                bound of Thm. 4.1, plain == worklist.
  classify      pinned: mesh derived from tetrahedra vs. the offset-difference
                rule and Euler characteristics; hand-built saddles; union-find
                component counts.
  cp_order      pinned: equals numpy lexsort on (value, index).
  requests      pinned through ``correct`` (R empty at a converged fixpoint).
  edit_stream, decode_stream
                pinned: decoding a correction's own stream gives its g bit for
                bit (hand-derived golden runs, random fields, several N);
                lossless count and passes follow Appendix C's trade-off in N.
  correct(increasing=True), requests(increasing=True)
                pinned: the point-reflection / negation identity against the
                decreasing mode, fixpoint invariants mirrored, brute-force
                topology of results, planted mistakes
                (tests/test_oracle_increasing.py).
  correct(events=True), requests(events=True)
                pinned: brute-force extremum graphs, merge and split trees and
                event selections of converged results, fixpoint invariants
                with the saddle order, hand-derived request sets on two- and
                three-well fields, planted mistakes (tests/test_oracle_events.py).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CONVERGED, STUCK, ITER_LIMIT = 1, 2, 3
STATUS_NAMES = {1: "CONVERGED", 2: "STUCK", 3: "ITER_LIMIT"}
T_MIN, T_MAX, T_JOIN, T_SPLIT = 1, 2, 4, 8

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        L.oracle_mesh.argtypes = [P, P, P, P]
        L.oracle_classify.argtypes = [P, i64, i64, i64, P, P, P]
        L.oracle_cp_order.argtypes = [P, i64, i64, i64, P]
        L.oracle_cp_order.restype = i64
        L.oracle_correct.argtypes = [P, P, i64, i64, i64, ctypes.c_float, ctypes.c_int,
                                     i64, ctypes.c_int, P, P, P]
        L.oracle_requests.argtypes = [P, P, i64, i64, i64, P, P]
        L.oracle_correct_events.argtypes = [P, P, i64, i64, i64, ctypes.c_float, ctypes.c_int, i64, P, P, P]
        L.oracle_requests_events.argtypes = [P, P, i64, i64, i64, P, P]
        L.oracle_correct_ex.argtypes = [P, P, i64, i64, i64, ctypes.c_float, ctypes.c_int, i64, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, P, P, P]
        L.oracle_requests_ex.argtypes = [P, P, i64, i64, i64, ctypes.c_int, ctypes.c_int, P, P]
        _lib = L
    return _lib


def _f32(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return a


def _dims_of(a: np.ndarray, dims):
    if dims is not None:
        nx, ny, nz = (int(d) for d in dims)
    else:
        shp = a.shape
        if len(shp) == 3:
            nz, ny, nx = shp
        elif len(shp) == 2:
            nz, (ny, nx) = 1, shp
        else:
            nz, ny, nx = 1, 1, shp[0]
    assert nx * ny * nz == a.size
    return nx, ny, nz


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def mesh():
    """(offsets [n_off, 3], link edges [n_edges, 2]) derived from tetrahedra."""
    off = np.zeros(96, np.int32)
    edg = np.zeros(512, np.int32)
    no = ctypes.c_int()
    ne = ctypes.c_int()
    lib().oracle_mesh(_p(off), ctypes.byref(no), _p(edg), ctypes.byref(ne))
    return off[: 3 * no.value].reshape(-1, 3).copy(), edg[: 2 * ne.value].reshape(-1, 2).copy()


def classify(h, dims=None):
    """Per vertex: up (int64 vertex id), down, type bits (T_MIN|T_MAX|T_JOIN|T_SPLIT)."""
    h = _f32(h)
    nx, ny, nz = _dims_of(h, dims)
    n = h.size
    up = np.empty(n, np.int64)
    dn = np.empty(n, np.int64)
    ty = np.empty(n, np.uint8)
    rc = lib().oracle_classify(_p(h), nx, ny, nz, _p(up), _p(dn), _p(ty))
    if rc != 0:
        raise ValueError(f"oracle_classify failed: {rc}")
    return up, dn, ty


def cp_order(f, dims=None) -> np.ndarray:
    """Critical points of f sorted ascending by (value, index)."""
    f = _f32(f)
    nx, ny, nz = _dims_of(f, dims)
    out = np.empty(f.size, np.int64)
    c = lib().oracle_cp_order(_p(f), nx, ny, nz, _p(out))
    if c < 0:
        raise ValueError(f"oracle_cp_order failed: {c}")
    return out[:c].copy()


def correct(f, fhat, xi: float, dims=None, N: int = 5, max_iters: int = 1 << 30,
            worklist: bool = False, events: bool = False, increasing: bool = False,
            edit_list: bool = True) -> dict:
    """Run the correction to its fixpoint.  Returns g, k, iterations, residual,
    status, n_edits, n_lossless and the edit list (ascending index).
    events=True: the saddle-ordering and original event constraints replace the
    reformulated ones (every rule is evaluated in full each pass).
    increasing=True: monotone increasing edits (every rule raises the vertex
    that must be higher; g <- fl(g + Delta) up to the lossless bound fl(f + xi)).
    edit_list=False: leave out the edit_* arrays (the caller derives the edits
    from k and g; saves host memory on very large fields)."""
    f = _f32(f)
    fhat = _f32(fhat)
    nx, ny, nz = _dims_of(f, dims)
    n = f.size
    g = np.empty(n, np.float32)
    k = np.empty(n, np.uint8)
    info = np.zeros(5, np.int64)
    if increasing:
        rc = lib().oracle_correct_ex(_p(f.reshape(-1)), _p(fhat.reshape(-1)), nx, ny, nz,
                                     ctypes.c_float(np.float32(xi)), int(N), int(max_iters), int(bool(worklist)),
                                     int(bool(events)), 1, _p(g), _p(k), _p(info))
    elif events:
        rc = lib().oracle_correct_events(_p(f.reshape(-1)), _p(fhat.reshape(-1)), nx, ny, nz,
                                         ctypes.c_float(np.float32(xi)), int(N), int(max_iters),
                                         _p(g), _p(k), _p(info))
    else:
        rc = lib().oracle_correct(_p(f.reshape(-1)), _p(fhat.reshape(-1)), nx, ny, nz,
                                  ctypes.c_float(np.float32(xi)), int(N), int(max_iters),
                                  int(bool(worklist)), _p(g), _p(k), _p(info))
    if rc != 0:
        raise ValueError(f"oracle_correct failed: {rc}")
    out = dict(g=g, k=k, iterations=int(info[0]), residual=int(info[1]),
               status=int(info[2]), n_edits=int(info[3]), n_lossless=int(info[4]))
    if edit_list:
        idx = np.nonzero(k)[0]
        out.update(edit_idx=idx.astype(np.int64), edit_k=k[idx].copy(),
                   edit_lossless=(k[idx] == N + 1), edit_value=g[idx].copy())
    return out


def correct_rc(f, fhat, xi: float, dims=None, N: int = 5) -> int:
    """Return code only (for input-validation tests)."""
    f = _f32(f)
    fhat = _f32(fhat)
    nx, ny, nz = _dims_of(f, dims)
    n = f.size
    g = np.empty(n, np.float32)
    k = np.empty(n, np.uint8)
    info = np.zeros(5, np.int64)
    return lib().oracle_correct(_p(f.reshape(-1)), _p(fhat.reshape(-1)), nx, ny, nz,
                                ctypes.c_float(np.float32(xi)), int(N), 1 << 30, 0,
                                _p(g), _p(k), _p(info))


def edit_stream(res: dict, N: int = 5):
    """The stored form of a correction result (Sec. 3.3: step edits plus the
    lossless values): the edit count k of every vertex (uint8; N + 1 marks the
    lossless bound) and the lossless values fl(f - xi) in index order."""
    k = np.asarray(res["k"], np.uint8)
    return k.copy(), np.asarray(res["g"], np.float32)[k == N + 1].copy()


def decode_stream(fhat, kcodes, lossless, xi: float, N: int = 5, increasing: bool = False) -> np.ndarray:
    """g from the stored form (Sec. 3.3): f_hat after k decrements g <- fl(g - Delta)
    (increments with increasing=True) with Delta = fl(xi / N), or the next
    lossless value where k = N + 1."""
    fhat = _f32(fhat).reshape(-1)
    k = np.asarray(kcodes, np.uint8).reshape(-1)
    if k.size != fhat.size or np.any(k > N + 1):
        raise ValueError("one edit count per vertex, each at most N + 1")
    delta = np.float32(np.float32(xi) / np.float32(N))
    g = fhat.copy()
    for step in range(N):
        m = k > step
        m &= k <= N
        g[m] = ((g[m] + delta) if increasing else (g[m] - delta)).astype(np.float32)
    lossless = np.asarray(lossless, np.float32).reshape(-1)
    sel = np.nonzero(k == N + 1)[0]
    if lossless.size != sel.size:
        raise ValueError("one lossless value per vertex with k = N + 1")
    g[sel] = lossless
    return g


def requests(f, g, dims=None, events: bool = False, increasing: bool = False):
    """Full request set R (bool per vertex) of the edited field g."""
    f = _f32(f)
    g = _f32(g)
    nx, ny, nz = _dims_of(f, dims)
    req = np.empty(f.size, np.uint8)
    cnt = ctypes.c_int64()
    if increasing:
        rc = lib().oracle_requests_ex(_p(f.reshape(-1)), _p(g.reshape(-1)), nx, ny, nz, int(bool(events)), 1,
                                      _p(req), ctypes.byref(cnt))
    else:
        fn = lib().oracle_requests_events if events else lib().oracle_requests
        rc = fn(_p(f.reshape(-1)), _p(g.reshape(-1)), nx, ny, nz, _p(req), ctypes.byref(cnt))
    if rc != 0:
        raise ValueError(f"oracle_requests failed: {rc}")
    return req.astype(bool), int(cnt.value)
