"""Synthetic scalar fields and error-bounded stand-ins for decompressed data.

Every field is a float32 torch tensor of shape (nz, ny, nx), C-contiguous, so
that the linear vertex index is ``x + nx * (y + ny * z)``.  Values are built
in float64 and rounded once to float32.

Recipes (they stand in for the paper's NYX / Combustion / Turbulence / Vortex
volumes, which are not available here):

* Gaussian bumps: sum over bumps of ``A * exp(-|p - c|^2 / (2 sigma^2))`` with
  centre ``c`` uniform in the box, ``sigma ~ U[lo, hi]`` voxels and
  ``A = +-U[0.5, 1]`` (sign drawn 50/50), evaluated inside a box of radius
  ``ceil(6 sigma)`` around the centre (the tail beyond is below 2e-8 * |A|),
  plus i.i.d. ``N(0, noise_std)`` per vertex.
* Multi-octave: for each (sigma, weight) an independent white-noise volume
  ``N(0, 1)`` is low-pass filtered with a periodic Gaussian of that sigma (in
  the Fourier domain), rescaled to unit standard deviation and weighted.
* ``xi = float32(rel * (max f - min f))`` computed in float64.
* f_hat by 2xi-quantisation ``2 xi * rint(f / 2 xi)`` (round half to even), or
  by ``f + U(-xi, xi)``, both in float64, then rounded to float32 and clamped
  into ``[fl(f - xi), fl(f + xi)]`` with float32 arithmetic, so that the
  pointwise bound ``|f_hat - f| <= xi`` holds after rounding.

Random draws: scalar parameters (centres, sigmas, amplitudes, dims, arrival
times) come from ``numpy.random.default_rng(seed)``; per-vertex noise comes
from a ``torch.Generator`` seeded with the same seed on the generating
device (the multi-octave noise on the CPU: numpy's generator and FFT, whose
results do not depend on the host's thread count), so a field made on a GPU
and one made on the CPU from the same seed differ.  Every comparison
therefore feeds the *same bytes* to both sides; CPU-made fields are the same
on every host with this software (their SHA-256 is checked where stored
digests are compared).
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

import numpy as np
import torch

Dims = Tuple[int, int, int]

# The single-field workloads by name (x fastest).  The batched and serving
# workloads are generated per field / per request by ``batched_specs`` and
# ``serving_requests``.
WORKLOADS: Dict[str, dict] = {
    "bumps64": dict(name="bumps64", kind="bumps", dims=(64, 64, 64), n_bumps=32,
            sigma=(2.0, 8.0), seed=0, rel=1e-3, fhat="quantised"),
    "bumps512": dict(name="bumps512", kind="bumps", dims=(512, 512, 512), n_bumps=4096,
            sigma=(2.0, 16.0), seed=1, rel=1e-4, fhat="uniform"),
    "octave1024": dict(name="octave1024", kind="octave", dims=(1024, 1024, 1024),
            seed=2, rel=1e-4, rels=(1e-2, 1e-3, 1e-4), fhat="quantised"),
}


def _gen(device, seed: int) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def gaussian_bumps(dims: Dims, n_bumps: int, sigma_range: Sequence[float],
                   seed: int, noise_std: float = 0.01,
                   device="cpu") -> torch.Tensor:
    """Sum of isotropic Gaussian bumps plus i.i.d. Gaussian noise (float32)."""
    nx, ny, nz = (int(d) for d in dims)
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(n_bumps, 3)) * np.array([nx, ny, nz], float)
    sigmas = rng.uniform(sigma_range[0], sigma_range[1], size=n_bumps)
    amps = rng.uniform(0.5, 1.0, size=n_bumps)
    signs = np.where(rng.random(n_bumps) < 0.5, -1.0, 1.0)
    amps = amps * signs
    f = torch.zeros((nz, ny, nx), dtype=torch.float64, device=device)
    for b in range(n_bumps):
        s = float(sigmas[b])
        r = int(math.ceil(6.0 * s))
        lo, hi = [], []
        for a, n in enumerate((nx, ny, nz)):
            c = centres[b, a]
            lo.append(max(0, int(math.floor(c)) - r))
            hi.append(min(n, int(math.floor(c)) + r + 1))
        if any(h <= l for l, h in zip(lo, hi)):
            continue
        prof = []
        for a in range(3):
            t = torch.arange(lo[a], hi[a], dtype=torch.float64, device=device)
            prof.append(torch.exp(-((t - centres[b, a]) ** 2) / (2.0 * s * s)))
        ex, ey, ez = prof
        f[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += float(amps[b]) * (
            ez[:, None, None] * ey[None, :, None] * ex[None, None, :])
    if noise_std > 0:
        noise = torch.randn((nz, ny, nx), dtype=torch.float64, device=device,
                            generator=_gen(device, seed))
        f += noise_std * noise
    return f.to(torch.float32)


def multi_octave(dims: Dims, seed: int, sigmas=(2.0, 8.0, 32.0),
                 weights=(1.0, 0.5, 0.25), device="cpu") -> torch.Tensor:
    """Weighted sum of periodic-Gaussian-filtered white-noise octaves (float32).

    On the CPU the noise comes from ``numpy.random.default_rng(seed)`` and the
    filtering from numpy's FFT (single-threaded, no run-time CPU dispatch), so
    the same seed gives the same bytes on every host with this software; on a
    GPU the noise and the FFTs are torch's on that device (other bytes)."""
    nx, ny, nz = (int(d) for d in dims)
    if torch.device(device).type == "cpu":
        return _multi_octave_numpy((nx, ny, nz), seed, sigmas, weights)
    gen = _gen(device, seed)
    kz = torch.fft.fftfreq(nz, dtype=torch.float64, device=device)
    ky = torch.fft.fftfreq(ny, dtype=torch.float64, device=device)
    kx = torch.fft.rfftfreq(nx, dtype=torch.float64, device=device)
    total = torch.zeros((nz, ny, nx), dtype=torch.float64, device=device)
    for s, w in zip(sigmas, weights):
        noise = torch.randn((nz, ny, nx), dtype=torch.float64, device=device, generator=gen)
        spec = torch.fft.rfftn(noise)
        del noise
        c = -2.0 * math.pi ** 2 * float(s) ** 2
        spec *= torch.exp(c * kz * kz)[:, None, None]
        spec *= torch.exp(c * ky * ky)[None, :, None]
        spec *= torch.exp(c * kx * kx)[None, None, :]
        sm = torch.fft.irfftn(spec, s=(nz, ny, nx))
        del spec
        sd = float(sm.std())
        sm *= float(w) / sd if sd > 0 else float(w)
        total += sm
        del sm
    return total.to(torch.float32)


def _multi_octave_numpy(dims: Dims, seed: int, sigmas, weights) -> torch.Tensor:
    """The CPU form of ``multi_octave`` (numpy RNG and FFT)."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    kz = np.fft.fftfreq(nz)
    ky = np.fft.fftfreq(ny)
    kx = np.fft.rfftfreq(nx)
    total = np.zeros((nz, ny, nx), dtype=np.float64)
    for s, w in zip(sigmas, weights):
        noise = rng.standard_normal((nz, ny, nx))
        spec = np.fft.rfftn(noise, axes=(0, 1, 2))
        del noise
        c = -2.0 * math.pi ** 2 * float(s) ** 2
        spec *= np.exp(c * kz * kz)[:, None, None]
        spec *= np.exp(c * ky * ky)[None, :, None]
        spec *= np.exp(c * kx * kx)[None, None, :]
        sm = np.fft.irfftn(spec, s=(nz, ny, nx), axes=(0, 1, 2))
        del spec
        sd = float(sm.std())
        sm *= float(w) / sd if sd > 0 else float(w)
        total += sm
        del sm
    return torch.from_numpy(total.astype(np.float32))


def xi_from_relative(f: torch.Tensor, rel: float) -> float:
    """Absolute bound xi = float32(rel * (max f - min f)), product in float64."""
    rng = float(f.max().item()) - float(f.min().item())
    return float(np.float32(rel * rng))


def clamp_into_bound(f: torch.Tensor, fhat: torch.Tensor, xi: float) -> torch.Tensor:
    """Clamp f_hat into [fl(f - xi), fl(f + xi)] using float32 arithmetic."""
    x = torch.tensor(xi, dtype=torch.float32, device=f.device)
    lo = f - x
    hi = f + x
    return torch.minimum(torch.maximum(fhat, lo), hi)


def fhat_quantised(f: torch.Tensor, xi: float) -> torch.Tensor:
    """2xi-quantisation in float64 (round half to even), then float32 + clamp."""
    q = 2.0 * float(xi)
    fh = (q * torch.round(f.to(torch.float64) / q)).to(torch.float32)
    return clamp_into_bound(f, fh, xi)


def fhat_uniform(f: torch.Tensor, xi: float, seed: int) -> torch.Tensor:
    """f + U(-xi, xi) i.i.d. per vertex in float64, then float32 + clamp."""
    u = torch.rand(f.shape, dtype=torch.float64, device=f.device,
                   generator=_gen(f.device, seed ^ 0x5EED5))
    fh = (f.to(torch.float64) + float(xi) * (2.0 * u - 1.0)).to(torch.float32)
    return clamp_into_bound(f, fh, xi)


def make_case(kind: str, dims: Dims, seed: int, rel: float, fhat: str,
              n_bumps: int | None = None, sigma=(2.0, 8.0), noise_std=0.01,
              device="cpu"):
    """Build (f, f_hat, xi) for one field."""
    dims = tuple(int(d) for d in dims)
    if kind == "bumps":
        if n_bumps is None:
            n_bumps = max(1, math.ceil(dims[0] * dims[1] * dims[2] / 4096))
        f = gaussian_bumps(dims, n_bumps, sigma, seed, noise_std, device)
    elif kind == "octave":
        f = multi_octave(dims, seed, device=device)
    else:
        raise ValueError(f"unknown field kind {kind!r}")
    xi = xi_from_relative(f, rel)
    if fhat == "quantised":
        fh = fhat_quantised(f, xi)
    elif fhat == "uniform":
        fh = fhat_uniform(f, xi, seed)
    else:
        raise ValueError(f"unknown f_hat recipe {fhat!r}")
    return f, fh, xi


def _make_case_worker(spec: dict):
    torch.set_num_threads(1)
    f, fh, xi = make_case(spec["kind"], spec["dims"], spec["seed"], spec["rel"], spec["fhat"],
                          n_bumps=spec.get("n_bumps"), sigma=spec.get("sigma", (2.0, 8.0)), device="cpu")
    return f.numpy(), fh.numpy(), xi


def make_cases_cpu(specs: Sequence[dict], workers: int = 0):
    """(f, f_hat, xi) for many specs, made on the CPU with one torch thread per
    field in a pool of ``workers`` spawned processes (0: one per host core).
    The bytes equal those of ``make_case(..., device="cpu")`` one by one."""
    import concurrent.futures
    import multiprocessing
    import os

    workers = workers or os.cpu_count() or 1
    ctx = multiprocessing.get_context("spawn")  # safe after CUDA has been initialised
    with concurrent.futures.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        out = list(ex.map(_make_case_worker, specs, chunksize=1))
    return [(torch.from_numpy(f), torch.from_numpy(fh), xi) for f, fh, xi in out]


def workload_case(name: str, device="cpu", rel: float | None = None):
    """(f, f_hat, xi) of the named workload (optionally overriding rel)."""
    c = WORKLOADS[name]
    return make_case(c["kind"], c["dims"], c["seed"], c["rel"] if rel is None else rel,
                     c["fhat"], n_bumps=c.get("n_bumps"), sigma=c.get("sigma", (2.0, 8.0)),
                     device=device)


def batched_specs(count: int = 256, seed_base: int = 1000,
                  lo: int = 32, hi: int = 256) -> List[dict]:
    """Per-field specs of the many-fields workload: each axis uniform in
    [lo, hi], bumps = ceil(volume / 4096), sigma ~ U[2, 8], xi alternating
    1e-3 / 1e-4 of the range, f_hat = f + U(-xi, xi)."""
    out = []
    for j in range(count):
        seed = seed_base + j
        rng = np.random.default_rng(seed)
        dims = tuple(int(v) for v in rng.integers(lo, hi + 1, size=3))
        vol = dims[0] * dims[1] * dims[2]
        out.append(dict(kind="bumps", dims=dims, seed=seed,
                        n_bumps=max(1, math.ceil(vol / 4096)), sigma=(2.0, 8.0),
                        rel=1e-3 if j % 2 == 0 else 1e-4, fhat="uniform"))
    return out


def serving_requests(rate: float, duration: float, stream_seed: int = 999_999,
                     seed_base: int = 1_000_000,
                     sizes=(64, 128, 256, 512), probs=(0.4, 0.3, 0.2, 0.1)) -> List[dict]:
    """Poisson request stream: arrival times (s) and per-request field specs."""
    rng = np.random.default_rng(stream_seed)
    t = 0.0
    out = []
    r = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        seed = seed_base + r
        rr = np.random.default_rng(seed)
        side = int(rr.choice(sizes, p=probs))
        kind = "bumps" if rr.random() < 0.5 else "octave"
        rel = 1e-3 if rr.random() < 0.5 else 1e-4
        dims = (side, side, side)
        out.append(dict(t=t, kind=kind, dims=dims, seed=seed, rel=rel, fhat="quantised",
                        n_bumps=max(1, math.ceil(side ** 3 / 4096)), sigma=(2.0, 8.0)))
        r += 1
    return out
