"""The allocation-free entry point (exactz_correct_noalloc) gives the same
results as exactz_correct and as the oracle.

Some callers cannot allocate device memory in the middle of their work: an
application that reserved the whole device memory for its own pool up front
(a simulation or an in-situ analysis), where a cudaMalloc would fail or take
memory promised elsewhere, or a loop that cannot take the device
synchronisation that cudaMalloc / cudaFree may cause.  For them the library
keeps one fixed scratch array in static device storage, and this call carves
every buffer it needs from that array.  Its workspace refuses to grow (a grow
request fails with EXACTZ_ENOMEM), and the tests below also check that the
device's free memory does not change across a call.  This file is named so
that pytest collects it last; it passes alone and after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dev(a, dims):
    nx, ny, nz = dims
    return torch.from_numpy(np.ascontiguousarray(a, np.float32).reshape(nz, ny, nx)).cuda()


def _same(a, b):
    ga, gb = a["g"].reshape(-1).cpu().numpy(), b["g"].reshape(-1).cpu().numpy()
    assert np.array_equal(ga.view(np.uint32), gb.view(np.uint32))  # tolerance 0, as in every parity test
    for key in ("iterations", "status", "residual", "n_edits", "n_lossless", "n_critical"):
        assert a[key] == b[key], key
    for key in ("idx", "k", "lossless", "value"):
        x, y = a["edits"][key].cpu().numpy(), b["edits"][key].cpu().numpy()
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8)), key


def _same_as_oracle(a, ref):
    g = a["g"].reshape(-1).cpu().numpy()
    assert np.array_equal(g.view(np.uint32), ref["g"].view(np.uint32))
    for key in ("iterations", "status", "residual", "n_edits", "n_lossless"):
        assert a[key] == ref[key], key
    e = a["edits"]
    assert np.array_equal(e["idx"].cpu().numpy(), ref["edit_idx"])
    assert np.array_equal(e["k"].cpu().numpy(), ref["edit_k"])
    assert np.array_equal(e["value"].cpu().numpy().view(np.uint32), ref["edit_value"].view(np.uint32))


def _c_call(ez, f, fh, xi, dims, g, buf, opts):
    """exactz_correct_noalloc through the C ABI; returns (rc, exactz_result)."""
    res = ez._native.Result()
    rc = ez._native.lib().exactz_correct_noalloc(
        ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(fh.data_ptr()), ez._native.Dims(*dims),
        ctypes.c_float(float(np.float32(xi))), ctypes.byref(opts), ctypes.c_void_p(g.data_ptr()),
        ctypes.c_void_p(buf.data_ptr()), buf.shape[0], ctypes.byref(res),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, res


def _as_dict(ez, res, g, buf):
    return dict(g=g, iterations=res.iterations, status=res.status, residual=res.residual_violations,
                n_edits=res.n_edits, n_lossless=res.n_lossless, n_critical=res.n_critical,
                edits=ez.decode_edits(buf, res.n_edits))


def _case(dims, seed, recipe, rel, sigma):
    f, fh, xi = synth.make_case("bumps", dims, seed, rel, recipe, sigma=sigma)
    return f.numpy().reshape(-1), fh.numpy().reshape(-1), xi


def test_two_calls_in_a_row_match_the_allocating_entry_point():
    import paper_2604_01397_b300 as ez

    cases = [((40, 36, 30), 5, "uniform", 1e-2, (2.0, 5.0)),   # first call on the device: set-up
             ((64, 64, 64), 0, "quantised", 1e-3, (2.0, 8.0))]  # second call reuses the shared array
    runs = []
    for dims, seed, recipe, rel, sigma in cases:
        fn, hn, xi = _case(dims, seed, recipe, rel, sigma)
        f, fh = _dev(fn, dims), _dev(hn, dims)
        n = f.numel()
        runs.append((dims, fn, hn, xi, f, fh, ez.correct(f, fh, xi, mode="graph", edits_cap=n),
                     torch.empty_like(f), torch.empty((n, 16), dtype=torch.uint8, device="cuda")))
    opts = ez.make_opts(mode="frontier")
    for dims, fn, hn, xi, f, fh, ref, g, buf in runs:
        rc, res = _c_call(ez, f, fh, xi, dims, g, buf, opts)
        assert rc == 0
        got = _as_dict(ez, res, g, buf)
        _same(got, ref)
        _same_as_oracle(got, oracle.correct(fn, hn, xi, dims=dims))
        # the Python wrapper gives the same answer
        _same(ez.correct_noalloc(f, fh, xi, torch.empty_like(f), buf), ref)
    # with every kernel and the scratch loaded, further calls leave the
    # device's free memory unchanged (nothing allocated, by the library or torch)
    for dims, fn, hn, xi, f, fh, ref, g, buf in runs:
        torch.cuda.synchronize()
        free0, torch0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        rc, res = _c_call(ez, f, fh, xi, dims, g, buf, opts)
        torch.cuda.synchronize()
        free1, torch1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        assert rc == 0
        assert free1 == free0 and torch1 == torch0
        _same(_as_dict(ez, res, g, buf), ref)


@pytest.mark.parametrize("dims", [(48, 40, 33), (64, 64, 64), (1, 512, 512)],
                         ids=["ragged", "largest", "largest-one-vertex-rows"])
def test_increasing_edits_match_the_allocating_entry_point(dims):
    # the reflected -f, -f_hat live in the fixed scratch: still nothing
    # allocated, also for the largest accepted field (64^3 = 2^18 vertices) and
    # for the shape with the most row words per vertex (rows of one vertex)
    import paper_2604_01397_b300 as ez

    fn, hn, xi = _case(dims, 8, "uniform", 1e-2, (2.0, 5.0))
    f, fh = _dev(fn, dims), _dev(hn, dims)
    n = f.numel()
    ref = ez.correct(f, fh, xi, mode="graph", edits_cap=n, direction="increasing")
    g = torch.empty_like(f)
    buf = torch.empty((n, 16), dtype=torch.uint8, device="cuda")
    opts = ez.make_opts(mode="frontier", direction="increasing")
    assert _c_call(ez, f, fh, xi, dims, g, buf, opts)[0] == 0  # warm-up: kernels loaded
    torch.cuda.synchronize()
    free0, torch0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    rc, res = _c_call(ez, f, fh, xi, dims, g, buf, opts)
    torch.cuda.synchronize()
    free1, torch1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    assert rc == 0
    assert free1 == free0 and torch1 == torch0
    got = _as_dict(ez, res, g, buf)
    _same(got, ref)
    _same_as_oracle(got, oracle.correct(fn, hn, xi, dims=dims, increasing=True))
    # and a decreasing call right after it still matches
    _same(ez.correct_noalloc(f, fh, xi, torch.empty_like(f), buf), ez.correct(f, fh, xi, edits_cap=n))


def test_fields_beyond_the_limit_are_rejected():
    import paper_2604_01397_b300 as ez

    L = ez._native.lib()
    res = ez._native.Result()
    x = torch.zeros(8, device="cuda")
    rc = L.exactz_correct_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                  ez._native.Dims(65, 64, 64), ctypes.c_float(0.1), None,
                                  ctypes.c_void_p(x.data_ptr()), None, 0, ctypes.byref(res), None)
    assert rc == ez._native.EXACTZ_ESIZE
