"""The allocation-free entry point (exactz_correct_noalloc) gives the same
results as exactz_correct.

Some callers cannot allocate device memory in the middle of their work: code
that runs while a stream is being captured into a CUDA graph, applications that
reserve the whole device for their own pool, and loops that cannot afford the
device synchronisation cudaMalloc/cudaFree may cause.  For them the library
keeps one fixed scratch array in static device storage.  This file is named so
that pytest collects it last; it passes alone and after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

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


def test_two_calls_in_a_row_match_the_allocating_entry_point():
    import paper_2604_01397_b300 as ez

    cases = [((40, 36, 30), 5, "uniform", 1e-2, (2.0, 5.0)),   # first call on the device: set-up
             ((64, 64, 64), 0, "quantised", 1e-3, (2.0, 8.0))]  # second call reuses the shared array
    for dims, seed, recipe, rel, sigma in cases:
        f, fh, xi = synth.make_case("bumps", dims, seed, rel, recipe, sigma=sigma)
        f, fh = _dev(f.numpy(), dims), _dev(fh.numpy(), dims)
        n = f.numel()
        ref = ez.correct(f, fh, xi, mode="graph", edits_cap=n)
        g = torch.empty_like(f)
        buf = torch.empty((n, 16), dtype=torch.uint8, device="cuda")
        res = ez._native.Result()
        opts = ez.make_opts(mode="frontier")
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        rc = ez._native.lib().exactz_correct_noalloc(
            ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(fh.data_ptr()), ez._native.Dims(*dims),
            ctypes.c_float(float(np.float32(xi))), ctypes.byref(opts), ctypes.c_void_p(g.data_ptr()),
            ctypes.c_void_p(buf.data_ptr()), n, ctypes.byref(res),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before  # nothing allocated through torch either
        assert rc == 0
        got = dict(g=g, iterations=res.iterations, status=res.status, residual=res.residual_violations,
                   n_edits=res.n_edits, n_lossless=res.n_lossless, n_critical=res.n_critical,
                   edits=ez.decode_edits(buf, res.n_edits))
        _same(got, ref)
        # the Python wrapper gives the same answer
        _same(ez.correct_noalloc(f, fh, xi, torch.empty_like(f), buf), ref)


def test_increasing_edits_match_the_allocating_entry_point():
    # the reflected -f, -f_hat live in the fixed scratch: still nothing allocated
    import paper_2604_01397_b300 as ez

    dims = (48, 40, 33)
    f, fh, xi = synth.make_case("bumps", dims, 8, 1e-2, "uniform", sigma=(2.0, 5.0))
    f, fh = _dev(f.numpy(), dims), _dev(fh.numpy(), dims)
    n = f.numel()
    ref = ez.correct(f, fh, xi, mode="graph", edits_cap=n, direction="increasing")
    g = torch.empty_like(f)
    buf = torch.empty((n, 16), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    got = ez.correct_noalloc(f, fh, xi, g, buf, direction="increasing")
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
    _same(got, ref)
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
