"""Failure handling, injected on the host (no GPU fault is provoked).

* Allocation failures: the library's testing aid exactz_debug_fail_allocations
  makes chosen device allocations fail as out of memory (without calling
  cudaMalloc).  Every call must report it (EXACTZ_ENOMEM, or NULL from the
  create calls), free what it had allocated (the device's free memory is back
  where it was), and the library must work normally afterwards.
* The request server: waiting with a zero timeout on a request that is still
  queued returns at once without a result; a queued request can be withdrawn
  (exactz_server_cancel) and the server goes on serving the others, whose
  results equal the oracle's.
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


@pytest.fixture(autouse=True)
def _disarm():
    yield
    import paper_2604_01397_b300 as ez

    ez._native.lib().exactz_debug_fail_allocations(0, 0)


def _case(dims, seed=3, rel=1e-2):
    f, fh, xi = synth.make_case("bumps", dims, seed, rel, "uniform", sigma=(2.0, 5.0))
    return f.numpy().reshape(-1), fh.numpy().reshape(-1), xi


def _dev(a, dims):
    nx, ny, nz = dims
    return torch.from_numpy(np.ascontiguousarray(a, np.float32).reshape(nz, ny, nx)).cuda()


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _same_as_oracle(r, ref):
    g = r["g"].reshape(-1).cpu().numpy()
    assert np.array_equal(g.view(np.uint32), ref["g"].view(np.uint32))
    for key in ("iterations", "status", "residual", "n_edits", "n_lossless"):
        assert r[key] == ref[key], key


@pytest.mark.parametrize("skip", [0, 3, 12])
def test_workspace_create_reports_allocation_failure_and_leaks_nothing(skip):
    import paper_2604_01397_b300 as ez

    L = ez._native.lib()
    dims = (96, 64, 40)
    arr = (ez._native.Dims * 1)(ez._native.Dims(*dims))
    h = L.exactz_workspace_create(1, arr)  # warm-up: kernels and context loaded
    L.exactz_workspace_destroy(h)
    before = _free()
    L.exactz_debug_fail_allocations(skip, 1)
    assert not L.exactz_workspace_create(1, arr)
    assert _free() == before  # what was allocated before the failure was freed
    L.exactz_debug_fail_allocations(0, 0)
    fn, hn, xi = _case(dims)
    ws = ez.Workspace([dims])
    r = ws.correct([_dev(fn, dims)], [_dev(hn, dims)], [xi], mode="graph")[0]
    _same_as_oracle(r, oracle.correct(fn, hn, xi, dims=dims))
    ws.close()


def test_correct_reports_enomem_then_works():
    import paper_2604_01397_b300 as ez

    dims = (70, 50, 33)
    fn, hn, xi = _case(dims, seed=4)
    f, fh = _dev(fn, dims), _dev(hn, dims)
    ez.correct(f, fh, xi)  # warm-up
    before = _free()
    ez._native.lib().exactz_debug_fail_allocations(5, 1)
    with pytest.raises(ez.ExactzError) as e:
        ez.correct(f, fh, xi, edits=False)
    assert e.value.rc == ez._native.EXACTZ_ENOMEM
    assert _free() == before
    _same_as_oracle(ez.correct(f, fh, xi), oracle.correct(fn, hn, xi, dims=dims))


def test_server_create_reports_allocation_failure_and_leaks_nothing():
    import paper_2604_01397_b300 as ez

    ez.Server(budget_bytes=256 << 20, max_fields=4).close()  # warm-up
    before = _free()
    for skip in (0, 7, 20):
        ez._native.lib().exactz_debug_fail_allocations(skip, 1)
        with pytest.raises(ez.ExactzError):
            ez.Server(budget_bytes=256 << 20, max_fields=4)
        assert _free() == before
    ez._native.lib().exactz_debug_fail_allocations(0, 0)
    dims = (40, 30, 20)
    fn, hn, xi = _case(dims, seed=5)
    with ez.Server(budget_bytes=256 << 20, max_fields=4) as srv:
        r = srv.wait(srv.submit(torch.from_numpy(fn), torch.from_numpy(hn), xi, dims=dims))
    _same_as_oracle(r, oracle.correct(fn, hn, xi, dims=dims))


def _big_and_small():
    big = (256, 256, 256)
    f, fh, xi = synth.make_case("bumps", big, 7, 1e-4, "uniform", sigma=(2.0, 8.0))
    small = (48, 40, 36)
    fn, hn, xs = _case(small, seed=6)
    return (big, f.reshape(-1).pin_memory(), fh.reshape(-1).pin_memory(), xi), (small, fn, hn, xs)


def _until_resident(srv, limit_s=20.0):
    """Wait (bounded) until the server has admitted its first request."""
    import time

    t0 = time.perf_counter()
    while srv.stats()["resident"] == 0 and srv.stats()["completed"] == 0:
        assert time.perf_counter() - t0 < limit_s, "the first request was never admitted"
        time.sleep(0.0005)


def test_wait_with_zero_timeout_on_a_queued_request_returns_nothing():
    import paper_2604_01397_b300 as ez

    (bd, bf, bh, bxi), (sd, sf, sh, sxi) = _big_and_small()
    with ez.Server(budget_bytes=8 << 30, max_fields=1) as srv:  # one field at a time
        t1 = srv.submit(bf, bh, bxi, dims=bd)
        _until_resident(srv)
        t2 = srv.submit(torch.from_numpy(sf), torch.from_numpy(sh), sxi, dims=sd)
        # t2 waits for the only slot while t1 (256^3, milliseconds of passes) is corrected
        assert srv.wait(t2, timeout_s=0.0) is None
        assert srv.poll(t2) is None
        r2 = srv.wait(t2)
        r1 = srv.wait(t1)
    _same_as_oracle(r2, oracle.correct(sf, sh, sxi, dims=sd))
    assert r1["status"] in (oracle.CONVERGED, oracle.STUCK)


def test_cancel_a_queued_request():
    import paper_2604_01397_b300 as ez

    (bd, bf, bh, bxi), (sd, sf, sh, sxi) = _big_and_small()
    with ez.Server(budget_bytes=8 << 30, max_fields=1) as srv:
        t1 = srv.submit(bf, bh, bxi, dims=bd)
        _until_resident(srv)
        t2 = srv.submit(torch.from_numpy(sf), torch.from_numpy(sh), sxi, dims=sd)
        assert srv.cancel(t2)  # still queued behind t1: withdrawn
        with pytest.raises(ez.ExactzError):  # the ticket is gone
            srv.poll(t2)
        assert srv.stats()["cancelled"] == 1
        assert not srv.cancel(t1)  # admitted: never withdrawn mid-correction, its result comes
        r1 = srv.wait(t1)
        assert r1["status"] in (oracle.CONVERGED, oracle.STUCK)
        # the server goes on serving
        t3 = srv.submit(torch.from_numpy(sf), torch.from_numpy(sh), sxi, dims=sd)
        _same_as_oracle(srv.wait(t3), oracle.correct(sf, sh, sxi, dims=sd))
        st = srv.stats()
        assert st["error"] == 0 and st["completed"] == 2 and st["queued"] == 0
