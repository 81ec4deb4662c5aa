"""Python front end of the CUDA library: torch tensors in, torch tensors out.

Every function marshals arguments to the C ABI (include/exactz.h) and reads
the results back; all computation runs in the library's kernels.  Fields are
float32 tensors of shape (nz, ny, nx) (or flat with explicit dims), contiguous,
on a CUDA device; the current torch stream is used unless one is given.
"""
from __future__ import annotations

import ctypes
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import _native as N

MODES = {"plain": N.MODE_PLAIN, "frontier": N.MODE_FRONTIER, "graph": N.MODE_GRAPH, "fused": N.MODE_FUSED}
# event constraints: the global order of all critical points (Sec. 4.3), or the
# saddle order and extremum-graph merge / split events (Sec. 4.2)
EVENTS = {"reformulated": 0, "original": 1}
# edit direction: monotone decreasing (the paper's choice) or increasing edits
DIRECTIONS = {"decreasing": 0, "increasing": 1}
STATUS = {N.CONVERGED: "CONVERGED", N.STUCK: "STUCK", N.ITER_LIMIT: "ITER_LIMIT"}


class ExactzError(RuntimeError):
    def __init__(self, rc: int, where: str):
        super().__init__(f"{where}: {N.ERROR_NAMES.get(rc, rc)} ({rc})")
        self.rc = rc


def version() -> str:
    return N.lib().exactz_version().decode()


def dims_of(t: torch.Tensor, dims=None):
    if dims is not None:
        nx, ny, nz = (int(d) for d in dims)
    elif t.dim() == 3:
        nz, ny, nx = t.shape
    elif t.dim() == 2:
        nz, (ny, nx) = 1, t.shape
    elif t.dim() == 1:
        nz, ny, nx = 1, 1, t.shape[0]
    else:
        raise ValueError("field must be 1D, 2D or 3D")
    if nx * ny * nz != t.numel():
        raise ValueError("dims do not match the tensor size")
    return int(nx), int(ny), int(nz)


def _check(t: torch.Tensor, name: str, host: bool = False):
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 tensor")
    if host and t.is_cuda:
        raise ValueError(f"{name} must be a host tensor for host_buffers")
    if not host and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (no CPU fallback)")


def make_opts(N_steps: int = 5, mode: str = "graph", max_iters: int = 1_000_000,
              want_edit_list: bool = True, profile: bool = False, events: str = "reformulated",
              direction: str = "decreasing") -> N.Opts:
    o = N.Opts()
    N.lib().exactz_default_opts(ctypes.byref(o))
    o.N = int(N_steps)
    o.mode = MODES[mode] if isinstance(mode, str) else int(mode)
    o.max_iters = int(max_iters)
    o.want_edit_list = int(bool(want_edit_list))
    o.profile = int(bool(profile))
    o.events = EVENTS[events] if isinstance(events, str) else int(events)
    o.direction = DIRECTIONS[direction] if isinstance(direction, str) else int(direction)
    return o


def default_edits_cap(n: int) -> int:
    return n if n <= (1 << 26) else n // 4


def decode_edits(buf: torch.Tensor, count: int) -> Dict[str, torch.Tensor]:
    """Split a (cap, 16) uint8 record buffer into idx / value / k / lossless
    (strided views into buf, no copies: they change when buf is reused) and
    the records themselves."""
    count = min(int(count), buf.shape[0])
    b = buf[:count]
    return dict(idx=b.view(torch.int64)[:, 0], value=b.view(torch.float32)[:, 2], k=b[:, 12],
                lossless=b[:, 13].view(torch.bool), records=b)


def _result_dict(r: N.Result) -> dict:
    return dict(iterations=int(r.iterations), n_edits=int(r.n_edits), n_lossless=int(r.n_lossless),
                residual=int(r.residual_violations), n_critical=int(r.n_critical), status=int(r.status),
                status_name=STATUS.get(int(r.status), N.ERROR_NAMES.get(int(r.status), str(r.status))))


def _stream(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Workspace:
    """Device workspace planned for a list of field dims (x, y, z sizes)."""

    def __init__(self, dims_list: Sequence[Sequence[int]]):
        self.dims_list = [tuple(int(v) for v in d) for d in dims_list]
        arr = (N.Dims * len(self.dims_list))(*[N.Dims(*d) for d in self.dims_list])
        self._h = N.lib().exactz_workspace_create(len(self.dims_list), arr)
        if not self._h:
            raise ExactzError(N.EXACTZ_ENOMEM, "exactz_workspace_create")

    def stats(self) -> dict:
        """Launch count, passes and (with profile=True) per-stage device ms of the last call."""
        st = N.Stats()
        N.lib().exactz_ws_stats(self._h, ctypes.byref(st))
        return dict(kernel_launches=int(st.kernel_launches), passes=int(st.passes),
                    total_critical=int(st.total_critical), sum_requests=int(st.sum_requests),
                    sum_tiles=int(st.sum_tiles), sum_pairs=int(st.sum_pairs),
                    stage_ms={k: float(v) for k, v in zip(N.STAGES, st.stage_ms)},
                    loop_kernel_ms={k: float(v) for k, v in zip(("check", "pairs", "apply"), st.loop_kernel_ms)},
                    loop_passes=int(st.loop_passes), sum_visits=int(st.sum_visits))

    def tuning(self) -> dict:
        t = N.Tuning()
        N.lib().exactz_ws_get_tuning(self._h, ctypes.byref(t))
        return {k: getattr(t, k) for k, _ in N.Tuning._fields_}

    def set_tuning(self, stencil_blocks_per_sm=48, apply_blocks_per_sm=32, pairs_blocks_per_sm=8,
                   chunked_schedule=0):
        t = N.Tuning(stencil_blocks_per_sm, apply_blocks_per_sm, pairs_blocks_per_sm, chunked_schedule, 0.0)
        rc = N.lib().exactz_ws_set_tuning(self._h, ctypes.byref(t))
        if rc != N.EXACTZ_OK:
            raise ExactzError(rc, "exactz_ws_set_tuning")

    def autotune(self, fs, fhats, xis, dims=None, N_steps: int = 5, mode: str = "graph", repeats: int = 2,
                 stream=None, events: str = "reformulated", direction: str = "decreasing") -> dict:
        """Pick the launch schedule for these fields by timing whole corrections."""
        nf = len(fs)
        dl = [dims_of(fs[i], dims[i] if dims else None) for i in range(nf)]
        t = N.Tuning()
        o = make_opts(N_steps, mode, 1_000_000, False, events=events, direction=direction)
        rc = N.lib().exactz_ws_autotune(
            self._h, nf, N.ptr_array([x.data_ptr() for x in fs]), N.ptr_array([x.data_ptr() for x in fhats]),
            (N.Dims * nf)(*[N.Dims(*d) for d in dl]), (ctypes.c_float * nf)(*[float(np.float32(x)) for x in xis]),
            ctypes.byref(o), ctypes.c_void_p(_stream(stream)), int(repeats), ctypes.byref(t))
        if rc != N.EXACTZ_OK:
            raise ExactzError(rc, "exactz_ws_autotune")
        return {k: getattr(t, k) for k, _ in N.Tuning._fields_}

    @property
    def nbytes(self) -> int:
        return int(N.lib().exactz_workspace_bytes(self._h))

    def close(self):
        if getattr(self, "_h", None):
            N.lib().exactz_workspace_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def correct(self, fs: List[torch.Tensor], fhats: List[torch.Tensor], xis: Sequence[float],
                dims: Optional[List] = None, N_steps: int = 5, mode: str = "graph",
                max_iters: int = 1_000_000, edits: bool = True, edits_caps=None,
                g_out: Optional[List[torch.Tensor]] = None, edit_bufs: Optional[List[torch.Tensor]] = None,
                stream=None, host_buffers: bool = False, raise_on_error: bool = True,
                profile: bool = False, events: str = "reformulated", direction: str = "decreasing") -> List[dict]:
        nf = len(fs)
        dl = [dims_of(fs[i], dims[i] if dims else None) for i in range(nf)]
        for i in range(nf):
            _check(fs[i], "f", host_buffers)
            _check(fhats[i], "fhat", host_buffers)
        if g_out is None:
            g_out = [torch.empty_like(f) for f in fs]
        if edits and edit_bufs is None:
            caps = [default_edits_cap(f.numel()) if edits_caps is None else int(edits_caps[i])
                    for i, f in enumerate(fs)]
            dev = None if host_buffers else fs[0].device
            edit_bufs = [torch.empty((c, 16), dtype=torch.uint8, device=dev) for c in caps]
        caps = [b.shape[0] for b in edit_bufs] if edits else [0] * nf
        darr = (N.Dims * nf)(*[N.Dims(*d) for d in dl])
        xarr = (ctypes.c_float * nf)(*[float(np.float32(x)) for x in xis])
        carr = (ctypes.c_uint64 * nf)(*caps)
        res = (N.Result * nf)()
        o = make_opts(N_steps, mode, max_iters, edits, profile, events, direction)
        rc = N.lib().exactz_ws_correct(
            self._h, nf, N.ptr_array([t.data_ptr() for t in fs]), N.ptr_array([t.data_ptr() for t in fhats]),
            darr, xarr, ctypes.byref(o), N.ptr_array([t.data_ptr() for t in g_out]),
            N.ptr_array([b.data_ptr() for b in edit_bufs] if edits else [0] * nf), carr, res,
            ctypes.c_void_p(0 if host_buffers and not torch.cuda.is_available() else _stream(stream)),
            int(host_buffers))
        if rc not in (N.EXACTZ_OK, N.EXACTZ_ECAP) and raise_on_error:
            raise ExactzError(rc, "exactz_ws_correct")
        out = []
        for i in range(nf):
            d = _result_dict(res[i])
            d["rc"] = rc
            d["g"] = g_out[i]
            if edits:
                d["edits"] = decode_edits(edit_bufs[i], d["n_edits"])
                d["edits_truncated"] = d["n_edits"] > caps[i]
            out.append(d)
        return out

    def correct_sequence(self, fs: Sequence[torch.Tensor], fhats: Sequence[torch.Tensor], xis: Sequence[float],
                         g_outs: Sequence[torch.Tensor], edit_bufs: Optional[Sequence[torch.Tensor]] = None,
                         dims=None, N_steps: int = 5, mode: str = "graph", max_iters: int = 1_000_000,
                         stream=None, raise_on_error: bool = True, profile: bool = False,
                         events: str = "reformulated", direction: str = "decreasing") -> List[dict]:
        """Correct host-resident fields of one shape one after another
        (exactz_ws_correct_sequence): field i+1 is copied in and field i-1
        copied out while field i is corrected.  fs, fhats: pinned host float32
        tensors; g_outs[i] (and edit_bufs[i], records of 16 bytes) pinned host
        outputs, which fields may share (the last field written stays).
        Returns one result dict per field ("g" and "edits" view its buffers)."""
        n = len(fs)
        if not (len(fhats) == len(xis) == len(g_outs) == n) or (edit_bufs is not None and len(edit_bufs) != n):
            raise ValueError("fs, fhats, xis, g_outs (and edit_bufs) must have one entry per field")
        for i in range(n):
            _check(fs[i], "f", True)
            _check(fhats[i], "fhat", True)
        d = dims_of(fs[0], dims) if n else (1, 1, 1)
        nv = d[0] * d[1] * d[2]
        for i in range(n):
            if fs[i].numel() != nv or fhats[i].numel() != nv or g_outs[i].numel() != nv:
                raise ValueError(f"field {i}: f, fhat and g_out must hold {nv} values")
            if g_outs[i].is_cuda or g_outs[i].dtype != torch.float32 or not g_outs[i].is_contiguous():
                raise ValueError(f"field {i}: g_out must be a contiguous float32 host tensor")
            if edit_bufs is not None:
                b = edit_bufs[i]
                if b.is_cuda or b.dtype != torch.uint8 or b.dim() != 2 or b.shape[1] != 16 or not b.is_contiguous():
                    raise ValueError(f"field {i}: edit buffer must be a contiguous (cap, 16) uint8 host tensor")
        xarr = (ctypes.c_float * max(n, 1))(*[float(np.float32(x)) for x in xis])
        caps = [b.shape[0] for b in edit_bufs] if edit_bufs is not None else [0] * n
        carr = (ctypes.c_uint64 * max(n, 1))(*caps)
        res = (N.Result * max(n, 1))()
        o = make_opts(N_steps, mode, max_iters, edit_bufs is not None, profile, events, direction)
        rc = N.lib().exactz_ws_correct_sequence(
            self._h, n, N.ptr_array([t.data_ptr() for t in fs]), N.ptr_array([t.data_ptr() for t in fhats]),
            N.Dims(*d), xarr, ctypes.byref(o), N.ptr_array([t.data_ptr() for t in g_outs]),
            N.ptr_array([b.data_ptr() for b in edit_bufs] if edit_bufs is not None else [0] * n), carr, res,
            ctypes.c_void_p(_stream(stream)))
        if rc not in (N.EXACTZ_OK, N.EXACTZ_ECAP) and raise_on_error:
            raise ExactzError(rc, "exactz_ws_correct_sequence")
        out = []
        for i in range(n):
            r = _result_dict(res[i])
            r["rc"] = rc
            r["g"] = g_outs[i]
            if edit_bufs is not None:
                r["edits"] = decode_edits(edit_bufs[i], r["n_edits"])
                r["edits_truncated"] = r["n_edits"] > caps[i]
            out.append(r)
        return out

    def correct_batch_sequence(self, fs, fhats, xis, g_outs, edit_bufs=None, dims=None, N_steps: int = 5,
                               mode: str = "graph", max_iters: int = 1_000_000, stream=None,
                               raise_on_error: bool = True, events: str = "reformulated",
                               direction: str = "decreasing") -> List[List[dict]]:
        """Correct a sequence of batches of host-resident fields
        (exactz_ws_correct_batch_sequence): fs[s][j], fhats[s][j], xis[s][j],
        g_outs[s][j] (and edit_bufs[s][j]) for step s and field j, field j of
        every step having dims[j] (default: the shapes of fs[0]).  Step s+1 is
        copied in and step s-1 copied out while step s is corrected.  Host
        tensors as for correct_sequence.  Returns the result dicts per step."""
        ns = len(fs)
        nf = len(fs[0]) if ns else 0
        for name, arr in (("fhats", fhats), ("xis", xis), ("g_outs", g_outs)) + (
                (("edit_bufs", edit_bufs),) if edit_bufs is not None else ()):
            if len(arr) != ns or any(len(x) != nf for x in arr):
                raise ValueError(f"{name} must have one entry per step and field")
        if ns == 0:
            return []
        dl = [dims_of(fs[0][j], dims[j] if dims else None) for j in range(nf)]
        flat = lambda a: [x for step in a for x in step]  # noqa: E731
        F, H, X, G = flat(fs), flat(fhats), flat(xis), flat(g_outs)
        E = flat(edit_bufs) if edit_bufs is not None else None
        for i in range(ns * nf):
            nv = dl[i % nf][0] * dl[i % nf][1] * dl[i % nf][2]
            _check(F[i], "f", True)
            _check(H[i], "fhat", True)
            if F[i].numel() != nv or H[i].numel() != nv or G[i].numel() != nv:
                raise ValueError(f"item {i}: f, fhat and g_out must hold {nv} values")
            if G[i].is_cuda or G[i].dtype != torch.float32 or not G[i].is_contiguous():
                raise ValueError(f"item {i}: g_out must be a contiguous float32 host tensor")
            if E is not None:
                b = E[i]
                if b.is_cuda or b.dtype != torch.uint8 or b.dim() != 2 or b.shape[1] != 16 or not b.is_contiguous():
                    raise ValueError(f"item {i}: edit buffer must be a contiguous (cap, 16) uint8 host tensor")
        n = ns * nf
        xarr = (ctypes.c_float * n)(*[float(np.float32(x)) for x in X])
        caps = [b.shape[0] for b in E] if E is not None else [0] * n
        carr = (ctypes.c_uint64 * n)(*caps)
        res = (N.Result * n)()
        o = make_opts(N_steps, mode, max_iters, E is not None, False, events, direction)
        rc = N.lib().exactz_ws_correct_batch_sequence(
            self._h, ns, nf, (N.Dims * nf)(*[N.Dims(*d) for d in dl]), N.ptr_array([t.data_ptr() for t in F]),
            N.ptr_array([t.data_ptr() for t in H]), xarr, ctypes.byref(o), N.ptr_array([t.data_ptr() for t in G]),
            N.ptr_array([b.data_ptr() for b in E] if E is not None else [0] * n), carr, res,
            ctypes.c_void_p(_stream(stream)))
        if rc not in (N.EXACTZ_OK, N.EXACTZ_ECAP) and raise_on_error:
            raise ExactzError(rc, "exactz_ws_correct_batch_sequence")
        out = []
        for st in range(ns):
            row = []
            for j in range(nf):
                i = st * nf + j
                r = _result_dict(res[i])
                r["rc"] = rc
                r["g"] = G[i]
                if E is not None:
                    r["edits"] = decode_edits(E[i], r["n_edits"])
                    r["edits_truncated"] = r["n_edits"] > caps[i]
                row.append(r)
            out.append(row)
        return out


def correct(f: torch.Tensor, fhat: torch.Tensor, xi: float, dims=None, N_steps: int = 5,
            mode: str = "graph", max_iters: int = 1_000_000, edits: bool = True, edits_cap=None,
            stream=None, raise_on_error: bool = True, events: str = "reformulated",
            direction: str = "decreasing") -> dict:
    """Correct one field to its fixpoint (exactz_correct).  events: "reformulated"
    (all critical points keep their order) or "original" (saddle order and
    extremum-graph merge / split events); direction: "decreasing" or
    "increasing" monotone edits."""
    _check(f, "f")
    _check(fhat, "fhat")
    d = dims_of(f, dims)
    g = torch.empty_like(f)
    cap = default_edits_cap(f.numel()) if edits_cap is None else int(edits_cap)
    buf = torch.empty((cap if edits else 0, 16), dtype=torch.uint8, device=f.device)
    res = N.Result()
    o = make_opts(N_steps, mode, max_iters, edits, events=events, direction=direction)
    rc = N.lib().exactz_correct(ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(fhat.data_ptr()), N.Dims(*d),
                                ctypes.c_float(float(np.float32(xi))), ctypes.byref(o),
                                ctypes.c_void_p(g.data_ptr()),
                                ctypes.c_void_p(buf.data_ptr() if edits and cap else 0),
                                cap if edits else 0, ctypes.byref(res), ctypes.c_void_p(_stream(stream)))
    if rc not in (N.EXACTZ_OK, N.EXACTZ_ECAP) and raise_on_error:
        raise ExactzError(rc, "exactz_correct")
    out = _result_dict(res)
    out["rc"] = rc
    out["g"] = g
    if edits:
        out["edits"] = decode_edits(buf, out["n_edits"])
        out["edits_truncated"] = out["n_edits"] > cap
    return out


def correct_batch(fs, fhats, xis, dims=None, N_steps: int = 5, mode: str = "graph",
                  max_iters: int = 1_000_000, edits: bool = True, edits_caps=None, stream=None,
                  raise_on_error: bool = True, events: str = "reformulated",
                  direction: str = "decreasing") -> List[dict]:
    """Correct many independent fields in one run (exactz_correct_batch)."""
    nf = len(fs)
    dl = [dims_of(fs[i], dims[i] if dims else None) for i in range(nf)]
    for i in range(nf):
        _check(fs[i], "f")
        _check(fhats[i], "fhat")
    gs = [torch.empty_like(f) for f in fs]
    caps = [default_edits_cap(f.numel()) if edits_caps is None else int(edits_caps[i]) for i, f in enumerate(fs)]
    bufs = [torch.empty((c if edits else 0, 16), dtype=torch.uint8, device=fs[0].device) for c in caps]
    res = (N.Result * nf)()
    o = make_opts(N_steps, mode, max_iters, edits, events=events, direction=direction)
    rc = N.lib().exactz_correct_batch(
        nf, N.ptr_array([t.data_ptr() for t in fs]), N.ptr_array([t.data_ptr() for t in fhats]),
        (N.Dims * nf)(*[N.Dims(*d) for d in dl]), (ctypes.c_float * nf)(*[float(np.float32(x)) for x in xis]),
        ctypes.byref(o), N.ptr_array([t.data_ptr() for t in gs]),
        N.ptr_array([b.data_ptr() for b in bufs] if edits else [0] * nf),
        (ctypes.c_uint64 * nf)(*[c if edits else 0 for c in caps]), res, ctypes.c_void_p(_stream(stream)))
    if rc not in (N.EXACTZ_OK, N.EXACTZ_ECAP) and raise_on_error:
        raise ExactzError(rc, "exactz_correct_batch")
    out = []
    for i in range(nf):
        d = _result_dict(res[i])
        d["rc"] = rc
        d["g"] = gs[i]
        if edits:
            d["edits"] = decode_edits(bufs[i], d["n_edits"])
        out.append(d)
    return out


def _edit_records(edits) -> torch.Tensor:
    """A (count, 16) uint8 tensor of exactz_edit records from decode_edits' dict (or the records themselves)."""
    if isinstance(edits, torch.Tensor):
        return edits
    if "records" in edits:
        return edits["records"]
    n = edits["idx"].numel()
    dev = edits["idx"].device
    out = torch.zeros((n, 16), dtype=torch.uint8, device=dev)
    if n:
        out[:, 0:8] = edits["idx"].to(torch.int64).contiguous().view(torch.uint8).reshape(n, 8)
        out[:, 8:12] = edits["value"].to(torch.float32).contiguous().view(torch.uint8).reshape(n, 4)
        out[:, 12] = edits["k"].to(torch.uint8)
        out[:, 13] = edits["lossless"].to(torch.uint8)
    return out


def encode_edits(edits, n: int, N_steps: int = 5, stream=None) -> dict:
    """The stored form of a result's edits (exactz_encode_edits): "kcodes", one
    edit-count byte per vertex (0..N steps, N+1 = lossless bound), and
    "lossless", the lossless values in index order.  edits: the "edits" dict of
    a correction result (or its (count, 16) uint8 records), on the device."""
    rec = _edit_records(edits)
    dev = rec.device
    kcodes = torch.empty(int(n), dtype=torch.uint8, device=dev)
    ne = rec.shape[0]
    lossless = torch.empty(max(ne, 1), dtype=torch.float32, device=dev)
    nl = ctypes.c_uint64()
    rc = N.lib().exactz_encode_edits(ctypes.c_void_p(rec.data_ptr() if ne else 0), ne, int(n), int(N_steps),
                                     ctypes.c_void_p(kcodes.data_ptr()), ctypes.c_void_p(lossless.data_ptr()), ne,
                                     ctypes.byref(nl), ctypes.c_void_p(_stream(stream)))
    if rc != N.EXACTZ_OK:
        raise ExactzError(rc, "exactz_encode_edits")
    return dict(kcodes=kcodes, lossless=lossless[: nl.value])


def decode_edits_stream(fhat: torch.Tensor, kcodes: torch.Tensor, lossless: torch.Tensor, xi: float,
                        N_steps: int = 5, stream=None, direction: str = "decreasing") -> torch.Tensor:
    """g from f_hat and the stored edits (exactz_decode_edits)."""
    _check(fhat, "fhat")
    g = torch.empty_like(fhat)
    n = fhat.numel()
    if kcodes.numel() != n:
        raise ValueError("kcodes must hold one byte per vertex")
    rc = N.lib().exactz_decode_edits(ctypes.c_void_p(fhat.data_ptr()), n, ctypes.c_float(float(np.float32(xi))),
                                     int(N_steps), DIRECTIONS[direction], ctypes.c_void_p(kcodes.data_ptr()),
                                     ctypes.c_void_p(lossless.data_ptr() if lossless.numel() else 0),
                                     ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(_stream(stream)))
    if rc != N.EXACTZ_OK:
        raise ExactzError(rc, "exactz_decode_edits")
    return g


def classify(h: torch.Tensor, dims=None, stream=None):
    """Per-vertex descriptor (int32 bit fields, see exactz.h) and type of field h."""
    _check(h, "h")
    d = dims_of(h, dims)
    desc = torch.empty(h.numel(), dtype=torch.int32, device=h.device)
    ty = torch.empty(h.numel(), dtype=torch.uint8, device=h.device)
    rc = N.lib().exactz_classify(ctypes.c_void_p(h.data_ptr()), N.Dims(*d), ctypes.c_void_p(desc.data_ptr()),
                                 ctypes.c_void_p(ty.data_ptr()), ctypes.c_void_p(_stream(stream)))
    if rc != N.EXACTZ_OK:
        raise ExactzError(rc, "exactz_classify")
    return desc, ty


def cp_order(f: torch.Tensor, dims=None, stream=None) -> torch.Tensor:
    """Critical points of f sorted by (value, index), as int64 vertex indices."""
    _check(f, "f")
    d = dims_of(f, dims)
    out = torch.empty(f.numel(), dtype=torch.int64, device=f.device)
    cnt = ctypes.c_uint64()
    rc = N.lib().exactz_cp_order(ctypes.c_void_p(f.data_ptr()), N.Dims(*d), ctypes.c_void_p(out.data_ptr()),
                                 ctypes.byref(cnt), ctypes.c_void_p(_stream(stream)))
    if rc != N.EXACTZ_OK:
        raise ExactzError(rc, "exactz_cp_order")
    return out[: cnt.value]


def correct_noalloc(f: torch.Tensor, fhat: torch.Tensor, xi: float, g_out: torch.Tensor,
                    edit_buf: Optional[torch.Tensor] = None, dims=None, N_steps: int = 5,
                    mode: str = "frontier", max_iters: int = 1_000_000, stream=None,
                    raise_on_error: bool = True, direction: str = "decreasing") -> dict:
    """exactz_correct_noalloc: the correction for fields of at most 2^18 vertices
    using only the library's fixed device scratch, for callers that cannot
    allocate device memory during the call (an application that has reserved
    all device memory for its own pool, or a loop that cannot take the device
    synchronisation of cudaMalloc / cudaFree).  The passes are driven from the
    host: every pass synchronises the stream.  The caller provides the output
    g_out and, optionally, a (cap, 16) uint8 edit-record buffer; this function
    allocates nothing on the device."""
    _check(f, "f")
    _check(fhat, "fhat")
    _check(g_out, "g_out")
    d = dims_of(f, dims)
    cap = 0 if edit_buf is None else edit_buf.shape[0]
    res = N.Result()
    o = make_opts(N_steps, mode, max_iters, edit_buf is not None, direction=direction)
    rc = N.lib().exactz_correct_noalloc(
        ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(fhat.data_ptr()), N.Dims(*d),
        ctypes.c_float(float(np.float32(xi))), ctypes.byref(o), ctypes.c_void_p(g_out.data_ptr()),
        ctypes.c_void_p(edit_buf.data_ptr() if edit_buf is not None else 0), cap, ctypes.byref(res),
        ctypes.c_void_p(_stream(stream)))
    if rc not in (N.EXACTZ_OK, N.EXACTZ_ECAP) and raise_on_error:
        raise ExactzError(rc, "exactz_correct_noalloc")
    out = _result_dict(res)
    out["rc"] = rc
    out["g"] = g_out
    if edit_buf is not None:
        out["edits"] = decode_edits(edit_buf, out["n_edits"])
    return out


class Server:
    """Request server with continuous batching (exactz_server_*).

    Fields are submitted from host memory (float32 CPU tensors, ideally pinned)
    and corrected on the current CUDA device together with whatever else is
    resident; each result equals correct(..., mode="frontier") for the same
    input.  submit() returns a ticket; wait()/poll() return the result dict
    (g and the edit list as CPU tensors, latency_s from submission to results
    in host memory) once it is ready.
    """

    def __init__(self, budget_bytes: int, max_fields: int = 64, N_steps: int = 5,
                 max_iters: int = 1_000_000, edits: bool = True, direction: str = "decreasing"):
        cfg = N.ServerConfig()
        cfg.budget_bytes = int(budget_bytes)
        cfg.max_fields = int(max_fields)
        cfg.opts = make_opts(N_steps, "frontier", max_iters, edits, direction=direction)
        self._h = N.lib().exactz_server_create(ctypes.byref(cfg))
        if not self._h:
            raise ExactzError(N.EXACTZ_ENOMEM, "exactz_server_create")
        self.edits = bool(edits)
        self._live = {}

    def submit(self, f: torch.Tensor, fhat: torch.Tensor, xi: float, dims=None, edits_cap=None,
               g_out: Optional[torch.Tensor] = None, edit_buf: Optional[torch.Tensor] = None) -> int:
        """Queue one field; g_out / edit_buf (a (cap, 16) uint8 host tensor) are
        allocated here unless given."""
        _check(f, "f", host=True)
        _check(fhat, "fhat", host=True)
        d = dims_of(f, dims)
        g = torch.empty(f.shape, dtype=torch.float32, pin_memory=f.is_pinned()) if g_out is None else g_out
        _check(g, "g_out", host=True)
        if g.numel() < f.numel():
            raise ValueError("g_out is smaller than the field")
        if not self.edits:
            buf, cap = None, 0
        elif edit_buf is not None:
            if edit_buf.is_cuda or edit_buf.dtype != torch.uint8 or edit_buf.dim() != 2 or edit_buf.shape[1] != 16:
                raise ValueError("edit_buf must be a (cap, 16) uint8 host tensor")
            buf, cap = edit_buf, int(edit_buf.shape[0])
        else:
            cap = default_edits_cap(f.numel()) if edits_cap is None else int(edits_cap)
            buf = torch.empty((cap, 16), dtype=torch.uint8, pin_memory=f.is_pinned()) if cap else None
        t = ctypes.c_uint64()
        rc = N.lib().exactz_server_submit(self._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(fhat.data_ptr()),
                                          N.Dims(*d), ctypes.c_float(float(np.float32(xi))),
                                          ctypes.c_void_p(g.data_ptr()),
                                          ctypes.c_void_p(buf.data_ptr() if buf is not None else 0), cap,
                                          ctypes.byref(t))
        if rc != N.EXACTZ_OK:
            raise ExactzError(rc, "exactz_server_submit")
        # the buffers must outlive the request: keep them until its result is taken
        self._live[t.value] = (f, fhat, g, buf, cap)
        return int(t.value)

    def _finish(self, ticket: int, res: N.Result, lat: ctypes.c_double, decode: bool) -> dict:
        f, fhat, g, buf, cap = self._live.pop(ticket)
        out = _result_dict(res)
        out["g"] = g
        out["latency_s"] = float(lat.value)
        if buf is not None:
            out["edits_truncated"] = out["n_edits"] > cap
            out["edits"] = decode_edits(buf, out["n_edits"]) if decode else buf
        return out

    def poll(self, ticket: int, decode: bool = True) -> Optional[dict]:
        """The result if ready (else None); decode=False leaves the edit records raw."""
        res, lat = N.Result(), ctypes.c_double()
        rc = N.lib().exactz_server_poll(self._h, int(ticket), ctypes.byref(res), ctypes.byref(lat))
        if rc < 0:
            raise ExactzError(rc, "exactz_server_poll")
        return self._finish(ticket, res, lat, decode) if rc == 1 else None

    def wait(self, ticket: int, timeout_s: float = -1.0, decode: bool = True) -> Optional[dict]:
        res, lat = N.Result(), ctypes.c_double()
        rc = N.lib().exactz_server_wait(self._h, int(ticket), float(timeout_s), ctypes.byref(res),
                                        ctypes.byref(lat))
        if rc < 0:
            raise ExactzError(rc, "exactz_server_wait")
        return self._finish(ticket, res, lat, decode) if rc == 1 else None

    def cancel(self, ticket: int) -> bool:
        """Withdraw a request that is still queued (True); False when it was
        already admitted or finished (its result comes as usual)."""
        rc = N.lib().exactz_server_cancel(self._h, int(ticket))
        if rc < 0:
            raise ExactzError(rc, "exactz_server_cancel")
        if rc == 1:
            self._live.pop(int(ticket), None)
        return rc == 1

    def stats(self) -> dict:
        st = N.ServerInfo()
        N.lib().exactz_server_stats(self._h, ctypes.byref(st))
        return {k: getattr(st, k) for k, _ in N.ServerInfo._fields_ if k != "reserved"}

    def close(self):
        if getattr(self, "_h", None):
            N.lib().exactz_server_destroy(self._h)
            self._h = None
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
