"""Canonical digests of a correction result, shared by the script that writes
the full-size oracle digests (``make_fullsize.py``) and the GPU tests that
compare the CUDA path with them.  Test infrastructure only: it holds no step
of the correction, only byte layouts and SHA-256.

An edit list is hashed as 16-byte little-endian records in ascending vertex
index, the layout of ``exactz_edit``: uint64 index, float32 value (its bits),
uint8 edit count k, uint8 lossless flag (k == N + 1), uint16 zero.
"""
from __future__ import annotations

import hashlib

import numpy as np

REC = np.dtype([("idx", "<u8"), ("value", "<f4"), ("k", "u1"), ("lossless", "u1"), ("reserved", "<u2")])
CHUNK = 1 << 25


def sha_array(a: np.ndarray) -> str:
    """SHA-256 of the array's bytes in C order."""
    a = np.ascontiguousarray(a)
    h = hashlib.sha256()
    flat = a.reshape(-1)
    for s in range(0, flat.size, CHUNK):
        h.update(memoryview(flat[s:s + CHUNK]).cast("B"))
    return h.hexdigest()


def _records(idx, value, k, lossless) -> np.ndarray:
    r = np.zeros(len(idx), REC)
    r["idx"] = idx
    r["value"] = value
    r["k"] = k
    r["lossless"] = lossless
    return r


def sha_edits_from_kg(k: np.ndarray, g: np.ndarray, N: int) -> str:
    """Digest of the edit list of a result given per vertex as edit counts k and
    values g: every vertex with k > 0, in index order."""
    h = hashlib.sha256()
    k = k.reshape(-1)
    g = g.reshape(-1)
    for s in range(0, k.size, CHUNK):
        kc = k[s:s + CHUNK]
        loc = np.nonzero(kc)[0]
        if loc.size:
            r = _records(loc.astype(np.uint64) + np.uint64(s), g[s:s + CHUNK][loc], kc[loc], kc[loc] == N + 1)
            h.update(memoryview(r).cast("B"))
    return h.hexdigest()


def sha_edits(idx, value, k, lossless) -> str:
    """Digest of an edit list given as four arrays (already in index order)."""
    h = hashlib.sha256()
    for s in range(0, len(idx), CHUNK):
        r = _records(idx[s:s + CHUNK], value[s:s + CHUNK], k[s:s + CHUNK], lossless[s:s + CHUNK])
        h.update(memoryview(r).cast("B"))
    return h.hexdigest()


def xi_bits(xi: float) -> str:
    return "0x%08x" % int(np.array([xi], np.float32).view(np.uint32)[0])
