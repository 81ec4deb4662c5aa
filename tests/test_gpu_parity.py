"""Parity of the CUDA path (through the C ABI) with the oracle: bit-exact g,
edit list, iteration count, status and residual (tolerance 0), in all three
loop forms, on hand-derived runs, small random fields, ragged and degenerate
grids, the 64^3 workload and batches of uneven fields."""
import numpy as np
import pytest
import torch

import oracle
import synth
from conftest import read_golden
from gpu_util import assert_same, gpu_run, k_from_edits, oracle_run, to_dev

pytestmark = pytest.mark.gpu
MODES = ["plain", "frontier", "graph", "fused"]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01397_b300  # noqa: F401  (fails loudly if the library is missing)


def _golden(name):
    c = read_golden(name)
    dims = tuple(int(x) for x in c["dims"])
    arr = lambda key: np.array([float(x) for x in c[key]], np.float32)  # noqa: E731
    return dims, float(c["xi"][0]), int(c["N"][0]), arr("f"), arr("fhat"), c


@pytest.mark.parametrize("name", ["cascade_1d.txt", "lossless_1d.txt", "stuck_1d.txt"])
@pytest.mark.parametrize("mode", MODES)
def test_golden(name, mode):
    dims, xi, N, f, fh, c = _golden(name)
    r = gpu_run(f, fh, xi, dims, mode, N)
    assert np.array_equal(r["g"].reshape(-1).cpu().numpy(), np.array([float(x) for x in c["g"]], np.float32))
    assert np.array_equal(k_from_edits(r, f.size), np.array([int(x) for x in c["k"]], np.uint8))
    assert r["iterations"] == int(c["iterations"][0])
    assert r["status"] == int(c["status"][0])
    assert r["residual"] == int(c["residual"][0])


def _case(dims, seed, recipe, rel, kind="bumps", n_bumps=6, sigma=(1.5, 3.0)):
    f, fh, xi = synth.make_case(kind, dims, seed, rel, recipe, n_bumps=n_bumps, sigma=sigma)
    return f.numpy().reshape(-1), fh.numpy().reshape(-1), xi


CASES = [
    ((10, 9, 8), 3, "quantised", 1e-2),
    ((12, 11, 10), 4, "uniform", 1e-2),
    ((16, 16, 1), 5, "quantised", 3e-2),
    ((24, 20, 1), 6, "uniform", 2e-2),
    ((40, 1, 1), 7, "uniform", 5e-2),
    ((64, 1, 1), 8, "quantised", 5e-2),
    ((9, 9, 9), 9, "quantised", 5e-3),
    ((5, 13, 7), 10, "uniform", 3e-2),
]

# ragged and degenerate grids: partial tiles in every axis, nx = 1, two vertices,
# exact tile multiples, long thin boxes
EDGE = [(33, 5, 7), (65, 3, 2), (1, 7, 9), (2, 1, 1), (1, 1, 100), (100, 1, 1), (31, 31, 1),
        (32, 4, 4), (64, 8, 8), (97, 13, 11), (1, 40, 1), (3, 3, 3), (34, 6, 6)]


@pytest.mark.parametrize("dims,seed,recipe,rel", CASES)
@pytest.mark.parametrize("mode", MODES)
def test_small_fields(dims, seed, recipe, rel, mode):
    f, fh, xi = _case(dims, seed, recipe, rel)
    assert_same(gpu_run(f, fh, xi, dims, mode), oracle_run(f, fh, xi, dims), f.size)


@pytest.mark.parametrize("dims", EDGE)
@pytest.mark.parametrize("recipe", ["quantised", "uniform"])
def test_edge_grids(dims, recipe):
    n = int(np.prod(dims))
    f, fh, xi = _case(dims, 100 + n % 97, recipe, 3e-2, n_bumps=3, sigma=(1.0, 4.0))
    ref = oracle_run(f, fh, xi, dims)
    for mode in MODES:
        assert_same(gpu_run(f, fh, xi, dims, mode), ref, n)


@pytest.mark.parametrize("levels", [2, 5, 50])
def test_heavy_ties(levels):
    # integer-valued fields: many exact ties, resolved by index on both sides
    dims = (37, 11, 9)
    rng = np.random.default_rng(levels)
    n = int(np.prod(dims))
    f = rng.integers(0, levels, n).astype(np.float32)
    xi = 0.75
    fh = np.clip(f + rng.integers(-1, 2, n).astype(np.float32) * np.float32(0.5),
                 f - np.float32(xi), f + np.float32(xi)).astype(np.float32)
    ref = oracle_run(f, fh, xi, dims)
    for mode in MODES:
        assert_same(gpu_run(f, fh, xi, dims, mode), ref, n)


@pytest.mark.parametrize("N", [1, 3, 8])
def test_other_N(N):
    dims = (20, 18, 9)
    f, fh, xi = _case(dims, 21, "quantised", 2e-2)
    assert_same(gpu_run(f, fh, xi, dims, "graph", N=N), oracle_run(f, fh, xi, dims, N=N), f.size, N=N)


@pytest.mark.parametrize("mode", MODES)
def test_iteration_cap(mode):
    dims = (12, 11, 10)
    f, fh, xi = _case(dims, 4, "uniform", 1e-2)
    for cap in (0, 1, 2):
        assert_same(gpu_run(f, fh, xi, dims, mode, max_iters=cap), oracle_run(f, fh, xi, dims, max_iters=cap),
                    f.size)


@pytest.mark.parametrize("mode", MODES)
def test_workload_64(mode):
    f, fh, xi = synth.fields.workload_case("bumps64")
    f, fh = f.numpy().reshape(-1), fh.numpy().reshape(-1)
    assert_same(gpu_run(f, fh, xi, (64, 64, 64), mode), oracle_run(f, fh, xi, (64, 64, 64)), f.size)


def test_validation_errors():
    import paper_2604_01397_b300 as ez

    dims = (8, 8, 8)
    f, fh, xi = _case(dims, 2, "uniform", 1e-2)
    bad = fh.copy()
    bad[17] = np.nan
    r = ez.correct(to_dev(f, dims), to_dev(bad, dims), xi, raise_on_error=False)
    assert r["rc"] == -2 and r["status"] == -2
    bad = fh.copy()
    bad[40] = f[40] + np.float32(2 * xi)
    r = ez.correct(to_dev(f, dims), to_dev(bad, dims), xi, raise_on_error=False)
    assert r["rc"] == -3 and r["status"] == -3
    bad = f.copy()
    bad[3] = np.inf
    r = ez.correct(to_dev(bad, dims), to_dev(fh, dims), xi, raise_on_error=False)
    assert r["rc"] == -2
    for x in (0.0, -1.0, float("nan"), float("inf")):
        r = ez.correct(to_dev(f, dims), to_dev(fh, dims), x, raise_on_error=False)
        assert r["rc"] == -1
    one = torch.zeros(1, device="cuda")
    r = ez.correct(one, one, 0.1, raise_on_error=False)
    assert r["rc"] == -1
    # the library still works after rejected calls
    assert_same(gpu_run(f, fh, xi, dims), oracle_run(f, fh, xi, dims), f.size)


def test_classify_and_cp_order():
    import paper_2604_01397_b300 as ez

    rng = np.random.default_rng(7)
    for dims, levels in [((17, 9, 6), 4), ((40, 7, 1), 1000), ((50, 1, 1), 3), ((33, 33, 5), 100000)]:
        n = int(np.prod(dims))
        h = rng.integers(0, levels, n).astype(np.float32)
        desc, ty = ez.classify(to_dev(h, dims))
        desc = desc.cpu().numpy().astype(np.int64)
        up, dn, tyo = oracle.classify(h, dims)
        assert np.array_equal(ty.cpu().numpy(), tyo)
        nx, ny, nz = dims
        offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                if (dx, dy, dz) == (0, 0, 0) or all(c >= 0 for c in (dx, dy, dz)) or all(c <= 0 for c in (dx, dy, dz))]
        delta = np.array([dx + nx * (dy + ny * dz) for dx, dy, dz in offs])
        assert len(delta) == 15 and delta[7] == 0
        idx = np.arange(n)
        assert np.array_equal(idx + delta[desc & 15], up)
        assert np.array_equal(idx + delta[(desc >> 4) & 15], dn)
        o = ez.cp_order(to_dev(h, dims)).cpu().numpy()
        assert np.array_equal(o, oracle.cp_order(h, dims))


def test_batch_matches_single_fields():
    import paper_2604_01397_b300 as ez

    specs = [((10, 9, 8), 3, "quantised", 1e-2), ((40, 1, 1), 7, "uniform", 5e-2),
             ((33, 5, 7), 11, "uniform", 3e-2), ((16, 16, 1), 5, "quantised", 3e-2),
             ((2, 1, 1), 1, "uniform", 1e-1), ((64, 8, 8), 12, "quantised", 1e-2)]
    cases = [_case(*s) for s in specs]
    fs = [to_dev(c[0], s[0]) for c, s in zip(cases, specs)]
    fhs = [to_dev(c[1], s[0]) for c, s in zip(cases, specs)]
    for mode in MODES:
        rs = ez.correct_batch(fs, fhs, [c[2] for c in cases], mode=mode)
        for r, c, s in zip(rs, cases, specs):
            assert_same(r, oracle_run(c[0], c[1], c[2], s[0]), c[0].size)


def test_workspace_reuse_and_host_buffers():
    import paper_2604_01397_b300 as ez

    big = ((48, 40, 30), 31, "uniform", 1e-2)
    small = ((21, 17, 13), 32, "quantised", 2e-2)
    ws = ez.Workspace([big[0]])
    try:
        for spec in (big, small, big):
            f, fh, xi = _case(*spec)
            ref = oracle_run(f, fh, xi, spec[0])
            r = ws.correct([to_dev(f, spec[0])], [to_dev(fh, spec[0])], [xi])[0]
            assert_same(r, ref, f.size)
            # host buffers: copies inside the call
            fc = torch.from_numpy(f.reshape(spec[0][::-1])).pin_memory()
            hc = torch.from_numpy(fh.reshape(spec[0][::-1])).pin_memory()
            g = torch.empty_like(fc).pin_memory()
            eb = torch.empty((f.size, 16), dtype=torch.uint8).pin_memory()
            rh = ws.correct([fc], [hc], [xi], g_out=[g], edit_bufs=[eb], host_buffers=True)[0]
            assert_same(rh, ref, f.size)
    finally:
        ws.close()


def test_launch_schedule_never_changes_results():
    import paper_2604_01397_b300 as ez

    specs = [((40, 36, 30), 5, "uniform", 1e-2), ((33, 5, 7), 11, "uniform", 3e-2), ((64, 8, 8), 12, "quantised", 1e-2)]
    cases = [_case(*sp) for sp in specs]
    fs = [to_dev(c[0], sp[0]) for c, sp in zip(cases, specs)]
    fhs = [to_dev(c[1], sp[0]) for c, sp in zip(cases, specs)]
    xis = [c[2] for c in cases]
    refs = [oracle_run(c[0], c[1], c[2], sp[0]) for c, sp in zip(cases, specs)]
    ws = ez.Workspace([sp[0] for sp in specs])
    try:
        for sched in [(4, 4, 2, 0), (32, 8, 16, 1), (16, 32, 4, 1)]:
            ws.set_tuning(*sched)
            for mode in MODES:
                for r, ref, c in zip(ws.correct(fs, fhs, xis, mode=mode), refs, cases):
                    assert_same(r, ref, c[0].size)
        t = ws.autotune(fs, fhs, xis, repeats=1)
        # a candidate, or the schedule the search started from (the last one set)
        assert t["stencil_blocks_per_sm"] in (6, 12, 24, 36, 48, 16) and t["chunked_schedule"] in (0, 1)
        assert t["best_ms"] > 0 and ws.tuning()["apply_blocks_per_sm"] == t["apply_blocks_per_sm"]
        for r, ref, c in zip(ws.correct(fs, fhs, xis), refs, cases):
            assert_same(r, ref, c[0].size)
        with pytest.raises(ez.ExactzError):
            ws.set_tuning(0, 16, 8, 0)
    finally:
        ws.close()
