"""Parity of the sequence entry point (exactz_ws_correct_sequence: host-resident
fields corrected one after another, the next field copied in and the previous
one copied out while a field is corrected) with the oracle: every field of a
sequence gets the result the oracle gives it alone, with per-field or shared
output buffers, with either event-constraint set and either edit direction;
an invalid field is refused before any copy, and a sequence longer than two
cycles the device slots correctly."""
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


DIMS = (37, 33, 9)  # ragged in x, y and z


def _fields(seeds, rel=2e-2, recipe="uniform"):
    out = []
    for s in seeds:
        f, fh, xi = synth.make_case("bumps", DIMS, s, rel, recipe, n_bumps=8, sigma=(1.5, 3.0))
        out.append((f.numpy().reshape(-1).copy(), fh.numpy().reshape(-1).copy(), xi))
    return out


def _pinned(a):
    return torch.from_numpy(a).pin_memory()


def _bufs(n, count):
    gs = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(count)]
    es = [torch.empty((n, 16), dtype=torch.uint8).pin_memory() for _ in range(count)]
    return gs, es


def _run(ws, fields, gs, es, **kw):
    rs = ws.correct_sequence([_pinned(f) for f, _, _ in fields], [_pinned(h) for _, h, _ in fields],
                             [xi for *_, xi in fields], gs, es, dims=DIMS, **kw)
    torch.cuda.synchronize()
    return rs


@pytest.mark.parametrize("count", [1, 2, 5])
def test_each_field_equals_oracle(count):
    import paper_2604_01397_b300 as ez

    fields = _fields(list(range(31, 31 + count)))
    n = fields[0][0].size
    refs = [oracle_run(f, fh, xi, DIMS) for f, fh, xi in fields]
    gs, es = _bufs(n, count)
    ws = ez.Workspace([DIMS])
    rs = _run(ws, fields, gs, es)
    for r, ref in zip(rs, refs):
        assert_same(r, ref, n)
    # the workspace serves a second sequence (slots and events reused)
    rs = _run(ws, fields[::-1], gs[::-1], es[::-1])
    for r, ref in zip(rs, refs[::-1]):
        assert_same(r, ref, n)
    ws.close()


def test_shared_output_buffers():
    import paper_2604_01397_b300 as ez

    fields = _fields([41, 42, 43, 44], recipe="quantised", rel=3e-2)
    n = fields[0][0].size
    refs = [oracle_run(f, fh, xi, DIMS) for f, fh, xi in fields]
    gs, es = _bufs(n, 1)
    ws = ez.Workspace([DIMS])
    rs = _run(ws, fields, gs * 4, es * 4)
    for r, ref in zip(rs, refs):  # scalars of every field
        for key in ("iterations", "status", "residual", "n_edits", "n_lossless"):
            assert r[key] == ref[key]
    assert_same(rs[3], refs[3], n)  # the shared buffers hold the last field
    ws.close()


@pytest.mark.parametrize("events,direction", [("original", "decreasing"), ("reformulated", "increasing"),
                                              ("original", "increasing")])
def test_options_pass_through(events, direction):
    import paper_2604_01397_b300 as ez

    fields = _fields([51, 52, 53])
    n = fields[0][0].size
    refs = [oracle_run(f, fh, xi, DIMS, events=events == "original", increasing=direction == "increasing")
            for f, fh, xi in fields]
    gs, es = _bufs(n, len(fields))
    ws = ez.Workspace([DIMS])
    rs = _run(ws, fields, gs, es, events=events, direction=direction)
    for r, ref in zip(rs, refs):
        assert_same(r, ref, n)
    ws.close()


def test_no_edit_lists_and_invalid_input():
    import paper_2604_01397_b300 as ez

    fields = _fields([61, 62, 63])
    n = fields[0][0].size
    gs, _ = _bufs(n, 3)
    ws = ez.Workspace([DIMS])
    bad = [fields[0][2], 0.0, fields[2][2]]  # xi = 0 is refused before any copy
    with pytest.raises(ez.ExactzError):
        ws.correct_sequence([_pinned(f) for f, _, _ in fields], [_pinned(h) for _, h, _ in fields], bad, gs,
                            dims=DIMS)
    rs = ws.correct_sequence([_pinned(f) for f, _, _ in fields], [_pinned(h) for _, h, _ in fields],
                             [xi for *_, xi in fields], gs, dims=DIMS)
    torch.cuda.synchronize()
    for (f, fh, xi), r, g in zip(fields, rs, gs):
        ref = oracle_run(f, fh, xi, DIMS)
        assert np.array_equal(g.numpy().view(np.uint32), ref["g"].view(np.uint32))
        assert r["iterations"] == ref["iterations"] and r["n_edits"] == ref["n_edits"] and "edits" not in r
    with pytest.raises(ValueError):  # a field of the wrong size never reaches the library
        ws.correct_sequence([_pinned(fields[0][0][:-1].copy())], [_pinned(fields[0][1])], [fields[0][2]], gs[:1],
                            dims=DIMS)
    ws.close()


def test_fields_larger_than_the_workspace_are_refused():
    import paper_2604_01397_b300 as ez

    fields = _fields([71, 72])
    n = fields[0][0].size
    gs, es = _bufs(n, 2)
    ws = ez.Workspace([(8, 8, 8)])  # planned for 512 vertices
    with pytest.raises(ez.ExactzError) as e:
        ws.correct_sequence([_pinned(f) for f, _, _ in fields], [_pinned(h) for _, h, _ in fields],
                            [xi for *_, xi in fields], gs, es, dims=DIMS)
    assert e.value.rc == -7  # EXACTZ_ESIZE, before any kernel of the first field
    ws.close()


BATCH = [(37, 33, 9), (16, 24, 12), (64, 5, 7)]  # uneven shapes; ragged rows (nx % 4 != 0 and == 0)


@pytest.mark.parametrize("steps", [1, 3])
def test_batch_sequence_each_field_equals_oracle(steps):
    # exactz_ws_correct_batch_sequence: steps of a batch of uneven fields, each
    # field of each step as the oracle gives it alone; more steps than device
    # slots, per-field output buffers in every step
    import paper_2604_01397_b300 as ez

    items = [[None] * len(BATCH) for _ in range(steps)]
    for s in range(steps):
        for j, d in enumerate(BATCH):
            f, fh, xi = synth.make_case("bumps", d, 100 + 10 * s + j, 2e-2, "uniform", n_bumps=6, sigma=(1.5, 3.0))
            items[s][j] = (f.numpy().reshape(-1).copy(), fh.numpy().reshape(-1).copy(), xi)
    ws = ez.Workspace(BATCH)
    gs = [[torch.empty(f.size, dtype=torch.float32).pin_memory() for f, _, _ in row] for row in items]
    es = [[torch.empty((f.size, 16), dtype=torch.uint8).pin_memory() for f, _, _ in row] for row in items]
    rs = ws.correct_batch_sequence([[_pinned(f) for f, _, _ in row] for row in items],
                                   [[_pinned(h) for _, h, _ in row] for row in items],
                                   [[xi for *_, xi in row] for row in items], gs, es, dims=BATCH)
    torch.cuda.synchronize()
    assert len(rs) == steps
    for s in range(steps):
        for j, d in enumerate(BATCH):
            f, fh, xi = items[s][j]
            assert_same(rs[s][j], oracle_run(f, fh, xi, d), f.size)
    # the batch corrected device-resident gives the same (the one-step case)
    dev = [ws.correct([torch.from_numpy(f).cuda() for f, _, _ in items[-1]],
                      [torch.from_numpy(h).cuda() for _, h, _ in items[-1]], [xi for *_, xi in items[-1]],
                      dims=BATCH)]
    for r, rd in zip(rs[-1], dev[0]):
        assert np.array_equal(r["g"].numpy().view(np.uint32), rd["g"].reshape(-1).cpu().numpy().view(np.uint32))
    ws.close()


def test_batch_sequence_refuses_bad_input_before_any_copy():
    import paper_2604_01397_b300 as ez

    ws = ez.Workspace(BATCH)
    row = []
    for j, d in enumerate(BATCH):
        f, fh, xi = synth.make_case("bumps", d, 200 + j, 2e-2, "uniform", n_bumps=6, sigma=(1.5, 3.0))
        row.append((f.numpy().reshape(-1).copy(), fh.numpy().reshape(-1).copy(), xi))
    gs = [[torch.empty(f.size, dtype=torch.float32).pin_memory() for f, _, _ in row]]
    with pytest.raises(ez.ExactzError) as e:  # xi = 0 for one field
        ws.correct_batch_sequence([[_pinned(f) for f, _, _ in row]], [[_pinned(h) for _, h, _ in row]],
                                  [[row[0][2], 0.0, row[2][2]]], gs, dims=BATCH)
    assert e.value.rc == ez._native.EXACTZ_EINVAL
    with pytest.raises(ValueError):  # a step with a field missing never reaches the library
        ws.correct_batch_sequence([[_pinned(f) for f, _, _ in row][:2]], [[_pinned(h) for _, h, _ in row]],
                                  [[xi for *_, xi in row]], gs, dims=BATCH)
    ws.close()
