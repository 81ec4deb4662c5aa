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


def _hand_streams():
    from conftest import read_golden, read_golden_cases

    return read_golden, read_golden_cases("stream_1d.txt")


@pytest.mark.parametrize("name", ["cascade_1d.txt", "lossless_1d.txt", "stuck_1d.txt"])
def test_encoder_writes_the_hand_written_stream(name):
    import paper_2604_01397_b300 as ez

    read_golden, cases = _hand_streams()
    c = read_golden(name)
    dims = tuple(int(x) for x in c["dims"])
    f = np.array([float(x) for x in c["f"]], np.float32)
    fh = np.array([float(x) for x in c["fhat"]], np.float32)
    N = int(c["N"][0])
    r = ez.correct(to_dev(f, dims), to_dev(fh, dims), float(c["xi"][0]), N_steps=N)
    st = ez.encode_edits(r["edits"], f.size, N)
    assert bytes(st["kcodes"].cpu().numpy()) == bytes(int(h, 16) for h in cases[name]["kcodes"])
    want = np.array([int(h, 16) for h in cases[name]["lossless"]], np.uint32)
    assert np.array_equal(st["lossless"].cpu().numpy().view(np.uint32), want)


def test_decoder_reads_a_hand_written_stream():
    import paper_2604_01397_b300 as ez

    _, cases = _hand_streams()
    c = cases["decode_by_hand"]
    fh = torch.tensor([float(x) for x in c["fhat"]], dtype=torch.float32, device="cuda")
    k = torch.tensor([int(h, 16) for h in c["kcodes"]], dtype=torch.uint8, device="cuda")
    lv = torch.from_numpy(np.array([int(h, 16) for h in c["lossless"]], np.uint32).view(np.float32)).cuda()
    g = ez.decode_edits_stream(fh, k, lv, float(c["xi"][0]), int(c["N"][0]))
    assert np.array_equal(g.cpu().numpy(), np.array([float(x) for x in c["g"]], np.float32))
