"""Properties every correction result must have, at any size (Sec. 3.3, 4.2-4.4).

Used on oracle results (to pin the oracle) and on CUDA results at sizes where
the oracle is too slow to run the whole correction.
"""
import numpy as np

import oracle


def replay(fhat, k, f, xi, N):
    """g implied by (f_hat, k): k successive fl(g - Delta) steps from f_hat, or
    the lossless bound fl(f - xi) when k == N + 1 (Sec. 3.3)."""
    xi32 = np.float32(xi)
    delta = np.float32(xi32 / np.float32(N))
    g = fhat.astype(np.float32).copy()
    for step in range(N):
        m = (k > step) & (k <= N)
        g[m] = (g[m] - delta).astype(np.float32)
    floor = (f - xi32).astype(np.float32)
    g[k == N + 1] = floor[k == N + 1]
    return g


def check_fixpoint(f, fhat, xi, N, g, k, status, residual=None, dims=None, full=True, events=False):
    """events=True: the result of the original event constraints, which fix the
    order of the saddles (C2) rather than of every critical point."""
    f = np.asarray(f, np.float32).reshape(-1)
    fhat = np.asarray(fhat, np.float32).reshape(-1)
    g = np.asarray(g, np.float32).reshape(-1)
    k = np.asarray(k, np.uint8).reshape(-1)
    xi32 = np.float32(xi)
    floor = (f - xi32).astype(np.float32)
    assert np.all(k <= N + 1), "k exceeds N + 1"
    assert np.all(g >= floor), "g below fl(f - xi)"
    assert np.all(g <= fhat), "g above f_hat (edits only decrease)"
    assert np.array_equal(g.view(np.uint32), replay(fhat, k, f, xi, N).view(np.uint32)), \
        "g is not the bitwise replay of (f_hat, k)"
    # pointwise bound in float64, allowing the single rounding of fl(f +- xi)
    d = g.astype(np.float64) - f.astype(np.float64)
    tol = np.spacing(np.abs(f).astype(np.float32) + xi32).astype(np.float64)
    assert np.all(d >= -float(xi32) - tol) and np.all(d <= float(xi32) + tol)
    if full:
        req, cnt = oracle.requests(f, g, dims, events=events)
        if status == oracle.CONVERGED:
            assert cnt == 0
            up_f, dn_f, ty_f = oracle.classify(f, dims)
            up_g, dn_g, ty_g = oracle.classify(g, dims)
            assert np.array_equal(up_f, up_g) and np.array_equal(dn_f, dn_g)
            assert np.array_equal(ty_f, ty_g)
            o = oracle.cp_order(f, dims)
            if events:
                o = o[(ty_f[o] & (oracle.T_JOIN | oracle.T_SPLIT)) != 0]
            gv = g[o]
            # strictly increasing in the g-order, ties broken by index
            ok = (gv[1:] > gv[:-1]) | ((gv[1:] == gv[:-1]) & (o[1:] > o[:-1]))
            assert np.all(ok)
        elif status == oracle.STUCK:
            assert cnt > 0 and np.all(k[req] == N + 1)
        if residual is not None and status != oracle.ITER_LIMIT:
            assert residual == cnt
