"""The request server (continuous batching): every result is bit-identical to
the oracle's and to the same request run alone, whatever else is resident;
admission respects the slot count and the arena budget; oversized requests are
refused; an invalid request fails alone without disturbing the others; a
server for increasing edits matches the oracle's increasing mode."""
import threading

import numpy as np
import pytest
import torch

import synth
from gpu_util import assert_same, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01397_b300  # noqa: F401


def _fields(specs):
    out = []
    for dims, seed, recipe, rel in specs:
        f, fh, xi = synth.make_case("bumps", dims, seed, rel, recipe, n_bumps=max(2, int(np.prod(dims)) // 4096),
                                    sigma=(1.5, 4.0))
        out.append((dims, f.reshape(-1).contiguous().pin_memory(), fh.reshape(-1).contiguous().pin_memory(), xi))
    return out


# uneven sizes: partial tiles, 1D / 2D / 3D, a few thousand to a quarter million vertices
MIX = [((10, 9, 8), 3, "quantised", 1e-2), ((64, 64, 64), 21, "uniform", 1e-3),
       ((33, 17, 9), 22, "quantised", 1e-2), ((200, 1, 1), 23, "uniform", 5e-2),
       ((96, 80, 1), 24, "quantised", 2e-2), ((48, 40, 36), 25, "uniform", 1e-3),
       ((12, 11, 10), 4, "uniform", 1e-2), ((70, 50, 20), 26, "quantised", 3e-3),
       ((5, 13, 7), 10, "uniform", 3e-2), ((40, 40, 40), 27, "quantised", 1e-3)]


def _wait(s, t):
    r = s.wait(t, timeout_s=300.0)
    assert r is not None, "request did not finish within 300 s"
    return r


def _same(a, b):
    assert np.array_equal(a["g"].numpy().view(np.uint32), b["g"].numpy().view(np.uint32))
    for k in ("iterations", "status", "residual", "n_edits", "n_lossless", "n_critical"):
        assert a[k] == b[k], k
    for k in ("idx", "k", "lossless"):
        assert torch.equal(a["edits"][k], b["edits"][k])
    assert np.array_equal(a["edits"]["value"].numpy().view(np.uint32), b["edits"]["value"].numpy().view(np.uint32))


def _as_oracle_dict(r):
    out = dict(r)
    out["g"] = r["g"].reshape(-1)
    return out


def test_mix_equals_oracle_and_alone():
    import paper_2604_01397_b300 as ez

    fields = _fields(MIX)
    alone = []
    with ez.Server(budget_bytes=1 << 30, max_fields=1) as s:
        for dims, f, fh, xi in fields:
            alone.append(_wait(s, s.submit(f, fh, xi, dims=dims)))
        st = s.stats()
        assert st["max_resident"] == 1 and st["completed"] == len(fields)
    with ez.Server(budget_bytes=1 << 30, max_fields=6) as s:
        tickets = [s.submit(f, fh, xi, dims=dims) for dims, f, fh, xi in fields]
        mixed = [_wait(s, t) for t in tickets]
        st = s.stats()
        assert st["completed"] == len(fields) and st["error"] == 0
        assert 2 <= st["max_resident"] <= 6
    for (dims, f, fh, xi), a, m in zip(fields, alone, mixed):
        _same(a, m)
        ref = oracle_run(f.numpy(), fh.numpy(), xi, dims)
        assert_same(_as_oracle_dict(m), ref, f.numel())
        assert m["latency_s"] > 0


def test_server_equals_frontier_entry_point():
    import paper_2604_01397_b300 as ez

    fields = _fields(MIX[:4])
    with ez.Server(budget_bytes=1 << 30, max_fields=4, N_steps=3, max_iters=4) as s:
        tickets = [s.submit(f, fh, xi, dims=dims) for dims, f, fh, xi in fields]
        got = [_wait(s, t) for t in tickets]
    for (dims, f, fh, xi), m in zip(fields, got):
        r = ez.correct(f.cuda(), fh.cuda(), xi, dims=dims, N_steps=3, mode="frontier", max_iters=4)
        r = {**r, "g": r["g"].cpu(), "edits": {k: v.cpu() for k, v in r["edits"].items()}}
        _same(r, m)


def test_increasing_edits_equal_oracle():
    # a server created for increasing edits reflects each room's inputs at
    # admission and its g at retirement; results equal the oracle's native
    # increasing mode and the workspace's, whatever else is resident
    import paper_2604_01397_b300 as ez

    fields = _fields(MIX[:6])
    with ez.Server(budget_bytes=1 << 30, max_fields=4, direction="increasing") as s:
        tickets = [s.submit(f, fh, xi, dims=dims) for dims, f, fh, xi in fields]
        got = [_wait(s, t) for t in tickets]
        assert s.stats()["error"] == 0
    for (dims, f, fh, xi), m in zip(fields, got):
        ref = oracle_run(f.numpy(), fh.numpy(), xi, dims, increasing=True)
        assert_same(_as_oracle_dict(m), ref, f.numel())
        r = ez.correct(f.cuda(), fh.cuda(), xi, dims=dims, mode="frontier", direction="increasing")
        r = {**r, "g": r["g"].cpu(), "edits": {k: v.cpu() for k, v in r["edits"].items()}}
        _same(r, m)


def test_budget_limits_residency_and_refuses_oversized():
    import paper_2604_01397_b300 as ez

    with ez.Server(budget_bytes=96 << 20, max_fields=8) as s:
        cap = s.stats()["capacity_vertices"]
        # two 80^3 fields fit the arena at once, three do not
        assert 2 * 80 ** 3 <= cap < 3 * 80 ** 3
        big = torch.zeros(120 ** 3, dtype=torch.float32)
        with pytest.raises(ez.ExactzError, match="ESIZE"):
            s.submit(big, big, 0.1, dims=(120, 120, 120))
        fields = _fields([((80, 80, 80), 30 + i, "uniform", 1e-3) for i in range(5)])
        tickets = [s.submit(f, fh, xi, dims=dims, edits_cap=1 << 16) for dims, f, fh, xi in fields]
        got = [_wait(s, t) for t in tickets]
        st = s.stats()
        assert st["max_resident"] <= 2 and st["completed"] == 5
    for (dims, f, fh, xi), m in zip(fields, got):
        ref = oracle_run(f.numpy(), fh.numpy(), xi, dims)
        assert_same(_as_oracle_dict(m), ref, f.numel(), check_edits=False)


def test_invalid_request_fails_alone():
    import paper_2604_01397_b300 as ez

    fields = _fields(MIX[:3])
    dims, f, fh, xi = fields[1]
    bad = fh.clone()
    bad[7] = float("nan")
    out_of_bound = fh.clone()
    out_of_bound[3] = f[3] + 4 * xi
    with ez.Server(budget_bytes=256 << 20, max_fields=4) as s:
        t_ok0 = s.submit(*fields[0][1:3], fields[0][3], dims=fields[0][0])
        t_nan = s.submit(f, bad, xi, dims=dims)
        t_bnd = s.submit(f, out_of_bound, xi, dims=dims)
        t_ok2 = s.submit(*fields[2][1:3], fields[2][3], dims=fields[2][0])
        assert _wait(s, t_nan)["status"] == -2
        assert _wait(s, t_bnd)["status"] == -3
        for t, (dd, ff, hh, x) in ((t_ok0, fields[0]), (t_ok2, fields[2])):
            ref = oracle_run(ff.numpy(), hh.numpy(), x, dd)
            assert_same(_as_oracle_dict(_wait(s, t)), ref, ff.numel())
        with pytest.raises(ez.ExactzError, match="EINVAL"):
            s.submit(f, fh, 0.0, dims=dims)
        with pytest.raises(ez.ExactzError, match="EINVAL"):
            s.wait(123456)


def test_truncated_edit_list_and_poll():
    import paper_2604_01397_b300 as ez

    dims, f, fh, xi = _fields([MIX[1]])[0]
    ref = oracle_run(f.numpy(), fh.numpy(), xi, dims)
    assert ref["n_edits"] > 10
    with ez.Server(budget_bytes=256 << 20, max_fields=2) as s:
        t = s.submit(f, fh, xi, dims=dims, edits_cap=10)
        r = None
        for _ in range(200000):
            r = s.poll(t)
            if r is not None:
                break
        if r is None:
            r = _wait(s, t)
    assert r["edits_truncated"] and r["n_edits"] == ref["n_edits"]
    assert np.array_equal(r["edits"]["idx"].numpy(), ref["edit_idx"][:10])
    assert np.array_equal(r["g"].numpy().view(np.uint32), ref["g"].view(np.uint32))


def test_submissions_from_several_threads():
    import paper_2604_01397_b300 as ez

    fields = _fields(MIX[:8])
    results = [None] * len(fields)
    with ez.Server(budget_bytes=512 << 20, max_fields=5) as s:
        def worker(j0):
            for j in range(j0, len(fields), 2):
                dims, f, fh, xi = fields[j]
                results[j] = _wait(s, s.submit(f, fh, xi, dims=dims))

        th = [threading.Thread(target=worker, args=(j,)) for j in (0, 1)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert s.stats()["completed"] == len(fields)
    for (dims, f, fh, xi), m in zip(fields, results):
        ref = oracle_run(f.numpy(), fh.numpy(), xi, dims)
        assert_same(_as_oracle_dict(m), ref, f.numel())
