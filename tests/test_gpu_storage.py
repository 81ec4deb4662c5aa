"""The stored form of a result on the GPU (exactz_encode_edits /
exactz_decode_edits, Sec. 3.3): the edit-count bytes and lossless values equal
the oracle's, decoding reproduces g bit for bit, and malformed input is
refused."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01397_b300  # noqa: F401


CASES = [((24, 20, 16), 6, "uniform", 2e-2), ((32, 28, 1), 13, "quantised", 5e-2), ((37, 11, 9), 4, "uniform", 1e-2),
         ((100, 1, 1), 7, "quantised", 5e-2), ((64, 64, 64), 21, "uniform", 1e-3)]


@pytest.mark.parametrize("dims,seed,recipe,rel", CASES)
@pytest.mark.parametrize("N", [1, 5, 9])
def test_stream_equals_oracle_and_decodes(dims, seed, recipe, rel, N):
    import paper_2604_01397_b300 as ez

    f, fh, xi = synth.make_case("bumps", dims, seed, rel, recipe, n_bumps=max(2, int(np.prod(dims)) // 4096),
                                sigma=(1.5, 4.0))
    f, fh = f.numpy().reshape(-1), fh.numpy().reshape(-1)
    n = f.size
    fd, hd = to_dev(f, dims), to_dev(fh, dims)
    r = ez.correct(fd, hd, xi, N_steps=N)
    s = ez.encode_edits(r["edits"], n, N)
    ref = oracle.correct(f, fh, xi, dims=dims, N=N)
    k_ref, l_ref = oracle.edit_stream(ref, N)
    assert np.array_equal(s["kcodes"].cpu().numpy(), k_ref)
    assert np.array_equal(s["lossless"].cpu().numpy().view(np.uint32), l_ref.view(np.uint32))
    g = ez.decode_edits_stream(hd.reshape(-1), s["kcodes"], s["lossless"], xi, N)
    assert torch.equal(g.view(torch.int32), r["g"].reshape(-1).view(torch.int32))


def _encode_rc(rec, n, N, cap=None):
    import paper_2604_01397_b300 as ez

    kc = torch.empty(n, dtype=torch.uint8, device="cuda")
    lv = torch.empty(max(1, rec.shape[0]), dtype=torch.float32, device="cuda")
    nl = ctypes.c_uint64()
    return ez._native.lib().exactz_encode_edits(
        ctypes.c_void_p(rec.data_ptr()), rec.shape[0], n, N, ctypes.c_void_p(kc.data_ptr()),
        ctypes.c_void_p(lv.data_ptr()), rec.shape[0] if cap is None else cap, ctypes.byref(nl), None), nl.value


def test_malformed_input_is_refused():
    import paper_2604_01397_b300 as ez

    dims = (24, 20, 16)
    f, fh, xi = synth.make_case("bumps", dims, 6, 2e-2, "uniform", n_bumps=8, sigma=(1.5, 3.0))
    n = f.numel()
    r = ez.correct(f.cuda(), fh.cuda(), xi)
    rec = ez.api._edit_records(r["edits"])
    ne = rec.shape[0]
    assert ne > 4 and r["n_lossless"] > 0
    rc, nl = _encode_rc(rec, n, 5)
    assert rc == ez._native.EXACTZ_OK and nl == r["n_lossless"]
    rc, _ = _encode_rc(rec, n, 5, cap=nl - 1)
    assert rc == ez._native.EXACTZ_ECAP
    bad = rec.clone()
    bad[[1, 2]] = bad[[2, 1]]  # not ascending
    assert _encode_rc(bad, n, 5)[0] == ez._native.EXACTZ_EINVAL
    bad = rec.clone()
    bad[-1, 0:8] = torch.tensor([n], dtype=torch.int64).view(torch.uint8).cuda()  # index past the field
    assert _encode_rc(bad, n, 5)[0] == ez._native.EXACTZ_EINVAL
    bad = rec.clone()
    bad[0, 13] = 1 - bad[0, 13]  # lossless flag disagrees with k
    assert _encode_rc(bad, n, 5)[0] == ez._native.EXACTZ_EINVAL
    kc = torch.zeros(n, dtype=torch.uint8, device="cuda")
    kc[3] = 7  # above N + 1
    with pytest.raises(ez.ExactzError, match="EINVAL"):
        ez.decode_edits_stream(fh.cuda().reshape(-1), kc, torch.zeros(1, device="cuda"), xi, 5)
