"""Parity of the CUDA path with the oracle under the original event
constraints (Sec. 4.2: saddle ordering C2, extremum-graph merge and split
events C3): bit-exact g, edit list, iteration count, status and residual in all
three loop forms, on small random fields, ragged and degenerate grids, heavy
ties, iteration caps, the 64^3 workload and uneven batches; plus the option's
plumbing (workspace reuse across both constraint sets, refusal where the
event lists cannot be allocated)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_same, gpu_run, oracle_run, to_dev

pytestmark = pytest.mark.gpu
MODES = ["plain", "frontier", "graph", "fused"]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01397_b300  # noqa: F401  (fails loudly if the library is missing)


def _case(dims, seed, recipe, rel, n_bumps=8, sigma=(1.5, 3.0)):
    f, fh, xi = synth.make_case("bumps", dims, seed, rel, recipe, n_bumps=n_bumps, sigma=sigma)
    return f.numpy().reshape(-1), fh.numpy().reshape(-1), xi


CASES = [((24, 20, 1), 6, "uniform", 2e-2), ((16, 16, 1), 5, "quantised", 3e-2),
         ((32, 28, 1), 13, "quantised", 5e-2), ((14, 13, 12), 14, "quantised", 3e-2),
         ((18, 16, 14), 17, "uniform", 4e-2), ((10, 9, 8), 3, "quantised", 1e-2),
         ((40, 1, 1), 7, "uniform", 5e-2), ((37, 33, 9), 18, "uniform", 1e-2)]

EDGE = [(33, 5, 7), (65, 3, 2), (1, 7, 9), (2, 1, 1), (1, 1, 100), (31, 31, 1), (32, 4, 4), (97, 13, 11),
        (3, 3, 3), (34, 6, 6)]


def _n_critical(f, dims):
    return int(np.count_nonzero(oracle.classify(f, dims)[2]))


@pytest.mark.parametrize("dims,seed,recipe,rel", CASES)
@pytest.mark.parametrize("mode", MODES)
def test_small_fields(dims, seed, recipe, rel, mode):
    f, fh, xi = _case(dims, seed, recipe, rel)
    r = gpu_run(f, fh, xi, dims, mode, events="original")
    assert_same(r, oracle_run(f, fh, xi, dims, events=True), f.size)
    assert r["n_critical"] == _n_critical(f, dims)


@pytest.mark.parametrize("dims", EDGE)
@pytest.mark.parametrize("recipe", ["quantised", "uniform"])
def test_edge_grids(dims, recipe):
    n = int(np.prod(dims))
    f, fh, xi = _case(dims, 100 + n % 97, recipe, 3e-2, n_bumps=3, sigma=(1.0, 4.0))
    ref = oracle_run(f, fh, xi, dims, events=True)
    for mode in MODES:
        assert_same(gpu_run(f, fh, xi, dims, mode, events="original"), ref, n)


@pytest.mark.parametrize("levels", [2, 5, 50])
def test_heavy_ties(levels):
    dims = (37, 11, 9)
    rng = np.random.default_rng(levels)
    n = int(np.prod(dims))
    f = rng.integers(0, levels, n).astype(np.float32)
    xi = 0.75
    fh = np.clip(f + rng.integers(-1, 2, n).astype(np.float32) * np.float32(0.5),
                 f - np.float32(xi), f + np.float32(xi)).astype(np.float32)
    ref = oracle_run(f, fh, xi, dims, events=True)
    for mode in MODES:
        assert_same(gpu_run(f, fh, xi, dims, mode, events="original"), ref, n)


@pytest.mark.parametrize("mode", MODES)
def test_iteration_cap(mode):
    dims = (14, 13, 12)
    f, fh, xi = _case(dims, 14, "quantised", 3e-2)
    for cap in (0, 1, 2, 5):
        assert_same(gpu_run(f, fh, xi, dims, mode, max_iters=cap, events="original"),
                    oracle_run(f, fh, xi, dims, max_iters=cap, events=True), f.size)


@pytest.mark.parametrize("mode", MODES)
def test_workload_64(mode):
    f, fh, xi = synth.fields.workload_case("bumps64")
    f, fh = f.numpy().reshape(-1), fh.numpy().reshape(-1)
    assert_same(gpu_run(f, fh, xi, (64, 64, 64), mode, events="original"),
                oracle_run(f, fh, xi, (64, 64, 64), events=True), f.size)


def test_constraint_sets_differ_and_workspace_switches():
    import paper_2604_01397_b300 as ez

    dims = (18, 16, 14)
    f, fh, xi = _case(dims, 17, "uniform", 4e-2)
    ref_o = oracle_run(f, fh, xi, dims, events=True)
    ref_r = oracle_run(f, fh, xi, dims)
    assert not np.array_equal(ref_o["g"], ref_r["g"])
    ws = ez.Workspace([dims])
    for events, ref in (("reformulated", ref_r), ("original", ref_o), ("reformulated", ref_r),
                        ("original", ref_o)):
        for mode in MODES:
            r = ws.correct([to_dev(f, dims)], [to_dev(fh, dims)], [xi], mode=mode, events=events)[0]
            torch.cuda.synchronize()
            assert_same(r, ref, f.size)
    st = ws.stats()
    assert st["total_critical"] == int(np.count_nonzero(oracle.classify(f, dims)[2] & (oracle.T_JOIN |
                                                                                        oracle.T_SPLIT)))
    ws.close()


def test_batch_matches_oracle():
    import paper_2604_01397_b300 as ez

    specs = [((10, 9, 8), 3, "quantised", 1e-2), ((33, 17, 9), 22, "quantised", 1e-2), ((200, 1, 1), 23,
             "uniform", 5e-2), ((96, 80, 1), 24, "quantised", 2e-2), ((20, 18, 16), 15, "quantised", 3e-2)]
    fields = [(d,) + _case(d, s, rc, rel) for d, s, rc, rel in specs]
    for mode in MODES:
        rs = ez.correct_batch([to_dev(f, d) for d, f, _, _ in fields], [to_dev(fh, d) for d, _, fh, _ in fields],
                              [xi for *_, xi in fields], dims=[d for d, *_ in fields], mode=mode,
                              events="original")
        torch.cuda.synchronize()
        for (d, f, fh, xi), r in zip(fields, rs):
            assert_same(r, oracle_run(f, fh, xi, d, events=True), f.size)


def test_refused_where_lists_cannot_be_allocated():
    import paper_2604_01397_b300 as ez

    dims = (10, 9, 8)
    f, fh, xi = _case(dims, 3, "quantised", 1e-2)
    g = torch.empty(f.size, device="cuda")
    o = ez.make_opts(mode="frontier", events="original")
    import ctypes
    res = ez._native.Result()
    rc = ez._native.lib().exactz_correct_noalloc(
        ctypes.c_void_p(to_dev(f, dims).data_ptr()), ctypes.c_void_p(to_dev(fh, dims).data_ptr()),
        ez._native.Dims(*dims), ctypes.c_float(xi), ctypes.byref(o), ctypes.c_void_p(g.data_ptr()), None, 0,
        ctypes.byref(res), None)
    assert rc == ez._native.EXACTZ_EINVAL
    with pytest.raises(ez.ExactzError, match="EINVAL"):
        ez.correct(to_dev(f, dims), to_dev(fh, dims), xi, events=7)
