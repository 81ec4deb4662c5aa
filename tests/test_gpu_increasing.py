"""Parity of the CUDA path with the oracle for increasing edits
(opts.direction = EXACTZ_EDITS_INCREASING): the library corrects the point
reflection of -f, -f_hat with its decreasing kernels and maps the result back;
the oracle implements the increasing rules and edits directly.  Bit-exact g,
edit list, iterations, status and residual in all loop forms, with either
event-constraint set, on small and ragged fields, ties, caps, the 64^3
workload, batches and host buffers; the stored form decodes with increments."""
import numpy as np
import pytest
import torch

import synth
from gpu_util import assert_same, gpu_run, oracle_run, to_dev

pytestmark = pytest.mark.gpu
MODES = ["plain", "frontier", "graph"]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01397_b300  # noqa: F401


def _case(dims, seed, recipe, rel, n_bumps=8, sigma=(1.5, 3.0)):
    f, fh, xi = synth.make_case("bumps", dims, seed, rel, recipe, n_bumps=n_bumps, sigma=sigma)
    return f.numpy().reshape(-1), fh.numpy().reshape(-1), xi


CASES = [((24, 20, 1), 6, "uniform", 2e-2), ((14, 13, 12), 14, "quantised", 3e-2), ((18, 16, 14), 17, "uniform", 4e-2),
         ((40, 1, 1), 7, "uniform", 5e-2), ((37, 33, 9), 18, "uniform", 1e-2), ((33, 5, 7), 2, "quantised", 3e-2)]


@pytest.mark.parametrize("dims,seed,recipe,rel", CASES)
@pytest.mark.parametrize("events", ["reformulated", "original"])
def test_small_fields(dims, seed, recipe, rel, events):
    f, fh, xi = _case(dims, seed, recipe, rel)
    ref = oracle_run(f, fh, xi, dims, events=events == "original", increasing=True)
    for mode in MODES:
        assert_same(gpu_run(f, fh, xi, dims, mode, events=events, direction="increasing"), ref, f.size)


@pytest.mark.parametrize("dims", [(2, 1, 1), (1, 7, 9), (31, 31, 1), (32, 4, 4), (97, 13, 11), (3, 3, 3)])
def test_edge_grids(dims):
    n = int(np.prod(dims))
    f, fh, xi = _case(dims, 100 + n % 97, "uniform", 3e-2, n_bumps=3, sigma=(1.0, 4.0))
    ref = oracle_run(f, fh, xi, dims, increasing=True)
    for mode in MODES:
        assert_same(gpu_run(f, fh, xi, dims, mode, direction="increasing"), ref, n)


def test_heavy_ties_and_caps():
    dims = (37, 11, 9)
    rng = np.random.default_rng(3)
    n = int(np.prod(dims))
    f = rng.integers(0, 5, n).astype(np.float32)
    xi = 0.75
    fh = np.clip(f + rng.integers(-1, 2, n).astype(np.float32) * np.float32(0.5), f - np.float32(xi),
                 f + np.float32(xi)).astype(np.float32)
    for cap in (0, 1, 3, 1 << 20):
        ref = oracle_run(f, fh, xi, dims, max_iters=cap, increasing=True)
        for mode in MODES:
            assert_same(gpu_run(f, fh, xi, dims, mode, max_iters=cap, direction="increasing"), ref, n)


def test_workload_64_and_stream():
    import paper_2604_01397_b300 as ez

    f, fh, xi = synth.fields.workload_case("bumps64")
    f, fh = f.numpy().reshape(-1), fh.numpy().reshape(-1)
    dims = (64, 64, 64)
    ref = oracle_run(f, fh, xi, dims, increasing=True)
    r = gpu_run(f, fh, xi, dims, "graph", direction="increasing")
    assert_same(r, ref, f.size)
    st = ez.encode_edits(r["edits"], f.size, 5)
    assert np.array_equal(st["kcodes"].cpu().numpy(), ref["k"])
    g = ez.decode_edits_stream(to_dev(fh, dims).reshape(-1), st["kcodes"], st["lossless"], xi, 5,
                               direction="increasing")
    assert torch.equal(g.view(torch.int32), r["g"].reshape(-1).view(torch.int32))
    dec = oracle_run(f, fh, xi, dims)
    assert not np.array_equal(dec["g"], ref["g"])


def test_batch_and_host_buffers():
    import paper_2604_01397_b300 as ez

    specs = [((10, 9, 8), 3, "quantised", 1e-2), ((33, 17, 9), 22, "quantised", 1e-2),
             ((200, 1, 1), 23, "uniform", 5e-2), ((20, 18, 16), 15, "quantised", 3e-2)]
    fields = [(d,) + _case(d, s, rc, rel) for d, s, rc, rel in specs]
    refs = [oracle_run(f, fh, xi, d, increasing=True) for d, f, fh, xi in fields]
    rs = ez.correct_batch([to_dev(f, d) for d, f, _, _ in fields], [to_dev(fh, d) for d, _, fh, _ in fields],
                          [xi for *_, xi in fields], dims=[d for d, *_ in fields], direction="increasing")
    torch.cuda.synchronize()
    for (d, f, fh, xi), r, ref in zip(fields, rs, refs):
        assert_same(r, ref, f.size)
    d, f, fh, xi = fields[3]
    ws = ez.Workspace([d])
    fc = torch.from_numpy(f.copy()).pin_memory()
    hc = torch.from_numpy(fh.copy()).pin_memory()
    gc = torch.empty_like(fc).pin_memory()
    ec = torch.empty((f.size, 16), dtype=torch.uint8).pin_memory()
    r = ws.correct([fc], [hc], [xi], dims=[d], g_out=[gc], edit_bufs=[ec], host_buffers=True,
                   direction="increasing")[0]
    assert_same(r, refs[3], f.size)
    ws.close()
