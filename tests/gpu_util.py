"""Helpers shared by the GPU tests: run the CUDA path on numpy inputs and
compare it with the oracle bit for bit."""
import numpy as np
import torch

import oracle


def to_dev(a, dims):
    nx, ny, nz = dims
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).reshape(nz, ny, nx)).cuda()


def k_from_edits(r, n):
    k = np.zeros(n, np.uint8)
    e = r["edits"]
    k[e["idx"].cpu().numpy()] = e["k"].cpu().numpy()
    return k


def gpu_run(f, fh, xi, dims, mode="graph", N=5, max_iters=1_000_000, events="reformulated",
            direction="decreasing"):
    import paper_2604_01397_b300 as ez

    r = ez.correct(to_dev(f, dims), to_dev(fh, dims), xi, N_steps=N, mode=mode, max_iters=max_iters,
                   events=events, direction=direction)
    torch.cuda.synchronize()
    return r


def assert_same(r, ref, n, N=5, check_edits=True):
    """CUDA result r (api dict) equals oracle result ref (oracle.correct dict)."""
    g = r["g"].reshape(-1).cpu().numpy()
    assert np.array_equal(g.view(np.uint32), ref["g"].view(np.uint32)), \
        f"g differs at {np.count_nonzero(g.view(np.uint32) != ref['g'].view(np.uint32))} vertices"
    for key in ("iterations", "status", "residual", "n_edits", "n_lossless"):
        assert r[key] == ref[key], f"{key}: cuda {r[key]} oracle {ref[key]}"
    if check_edits:
        e = r["edits"]
        idx = e["idx"].cpu().numpy()
        assert np.array_equal(idx, ref["edit_idx"]), "edit indices differ"
        assert np.array_equal(e["k"].cpu().numpy(), ref["edit_k"])
        assert np.array_equal(e["lossless"].cpu().numpy(), ref["edit_lossless"])
        assert np.array_equal(e["value"].cpu().numpy().view(np.uint32), ref["edit_value"].view(np.uint32))


def oracle_run(f, fh, xi, dims, N=5, max_iters=1 << 30, worklist=False, events=False, increasing=False):
    return oracle.correct(f, fh, xi, dims=dims, N=N, max_iters=max_iters, worklist=worklist, events=events,
                          increasing=increasing)
