#!/usr/bin/env python
"""Benchmark of the B300 EXaCTz correction: corrected GB/s to fixpoint.

Default workload (N = 1): one 512^3 float32 field of 4096 Gaussian bumps
(sigma ~ U[2, 16]) + N(0, 0.01) noise, seed 1, xi = 1e-4 * range,
f_hat = f + U(-xi, xi), corrected to its fixpoint with the CUDA-graph loop.
A step is one whole correction (set-up stencil, CP compaction and sort, all
passes, residual check, edit list) with inputs resident in HBM; the value is
4 * n bytes of float32 input per step time (each input field is 512 MiB, so
every step streams more than the 126 MB L2).

Also reported on the same JSON line: the same metric end to end through the C
ABI with host buffers (copies inside the timed region), the roofline of the
dominant kernel from CUDA events recorded around it on its own stream during
the timed steps, the plain and host-driven frontier loops, the oracle on a
bounded crop of the same workload on the host cores, and the SM clocks
sampled during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload bumps512|bumps64|octave1024|batched] [--size S]

With N > 1 (torchrun) every rank corrects its own replica of the workload
(no data-path collective; a barrier and a max-reduction of the step time only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "corrected GB/s on 1 B300 to fixpoint, batched vs plain; % HBM peak; p99 ms"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6400.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="bumps512")
    p.add_argument("--size", type=int, default=0, help="override the cube side (profiling runs)")
    p.add_argument("--mode", default="graph", choices=["graph", "frontier", "plain"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-extras", action="store_true")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--fields", type=int, default=256, help="field count of the batched workload")
    p.add_argument("--no-autotune", action="store_true", help="keep the default launch schedule")
    return p.parse_args()


# ---------------------------------------------------------------- workloads
def workload_spec(name: str, size: int = 0):
    from synth.fields import CONFIGS

    if name == "bumps512":
        c = dict(CONFIGS[2])
    elif name == "bumps64":
        c = dict(CONFIGS[1])
    elif name == "octave1024":
        c = dict(CONFIGS[3])
    else:
        raise SystemExit(f"unknown workload {name}")
    if size:
        vol = float(np.prod(c["dims"]))
        c["dims"] = (size, size, size)
        if c["kind"] == "bumps":  # same bump density
            c["n_bumps"] = max(1, round(c["n_bumps"] * size ** 3 / vol))
        c["name"] = f"{name}@{size}"
    return c


def describe(c) -> str:
    nx, ny, nz = c["dims"]
    if c["kind"] == "bumps":
        gen = (f"{c['n_bumps']} Gaussian bumps sigma~U[{c['sigma'][0]:g},{c['sigma'][1]:g}] amplitude +-U[0.5,1]"
               f" + N(0,0.01) noise")
    else:
        gen = "3 octaves of periodic-Gaussian-filtered white noise (sigma 2/8/32, weights 1/0.5/0.25)"
    fh = "f_hat = f + U(-xi,xi)" if c["fhat"] == "uniform" else "f_hat = 2xi*rint(f/2xi)"
    return f"{nx}x{ny}x{nz} float32, {gen}, seed {c['seed']}, xi = {c['rel']:g}*range, {fh}"


def make_fields(c, device):
    import synth

    return synth.make_case(c["kind"], c["dims"], c["seed"], c["rel"], c["fhat"], n_bumps=c.get("n_bumps"),
                           sigma=c.get("sigma", (2.0, 8.0)), device=device)


# ---------------------------------------------------------------- clocks
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class Clocks:
    def __init__(self, device_index: int, enabled: bool = True):
        self.proc = None
        self.idx = device_index
        if enabled:
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", f"--query-gpu={CLOCK_Q}", "--format=csv,noheader,nounits", "-i",
                     str(device_index), "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                    text=True)
            except OSError:
                self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def peaks():
    try:
        p = json.load(open(PEAKS_FILE))
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for fn in ("exz_kernels.cu", "exz_common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2604_01397_b300", "csrc", fn), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was
    taken on the current kernel source (null otherwise)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.md")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for line in open(path):
        m = re.match(r"\|\s*(\S+)\s*\|\s*(\S+)\s*\|\s*(\S+)\s*\|\s*([0-9.eE+]+)\s*\|", line)
        if m and m.group(1) == kernel and m.group(2) == workload and m.group(3) == src:
            return float(m.group(4))
    return None


def oracle_sample(f, fh, xi, side: int):
    """Run the oracle (plain mode, as it stands) on the side^3 corner crop."""
    import oracle

    fc = np.ascontiguousarray(f[:side, :side, :side])
    hc = np.ascontiguousarray(fh[:side, :side, :side])
    t0 = time.perf_counter()
    r = oracle.correct(fc.reshape(-1), hc.reshape(-1), xi, dims=(side, side, side))
    return time.perf_counter() - t0, r


def omp_threads() -> int:
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def choose_side(f, fh, xi, budget_s: float, lo=32, hi=256):
    """Pick a crop side whose oracle run takes about budget_s (calibrated on a small crop)."""
    t, _ = oracle_sample(f, fh, xi, lo)
    per = t / lo ** 3
    side = int((budget_s / max(per, 1e-12)) ** (1 / 3))
    return max(lo, min(hi, side, min(f.shape)))


# ---------------------------------------------------------------- reference arm
def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch

    c = workload_spec(a.workload, a.size)
    f, fh, xi = make_fields(c, "cpu")
    f, fh = f.numpy(), fh.numpy()
    budget = max(2.0, min(30.0, 150.0 / max(1, a.steps + a.warmup)))
    side = choose_side(f, fh, xi, budget)
    for _ in range(a.warmup):
        oracle_sample(f, fh, xi, side)
    times = []
    for _ in range(a.steps):
        t, r = oracle_sample(f, fh, xi, side)
        times.append(t)
    ms = 1e3 * statistics.mean(times)
    val = 4.0 * side ** 3 / (ms / 1e3) / 1e9
    cores = omp_threads()
    sample = (f"{side}^3 corner crop of the {c['name']} workload ({side ** 3} vertices), plain oracle "
              f"(full sweep each pass), to fixpoint: {r['iterations']} passes, {r['n_edits']} edits")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": describe(c), "sample": sample},
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def run_ours(a):
    import torch

    import paper_2604_01397_b300 as ez

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else torch.cuda.current_device())
    torch.cuda.set_device(dev)
    c = workload_spec(a.workload, a.size)
    f, fh, xi = make_fields(c, dev)
    torch.cuda.synchronize()
    n = f.numel()
    dims = c["dims"]
    ws = ez.Workspace([dims])
    g = torch.empty_like(f)
    cap = n if n <= (1 << 26) else n // 4
    ebuf = torch.empty((cap, 16), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(mode=a.mode, profile=True):
        return ws.correct([f], [fh], [xi], mode=mode, g_out=[g], edit_bufs=[ebuf], profile=profile)[0]

    tuning = ws.autotune([f], [fh], [xi], repeats=2) if not a.no_autotune else ws.tuning()

    for _ in range(max(3, a.warmup)):
        r = step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(dev.index if dev.index is not None else 0, enabled=not a.no_clocks)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    setup_ms, launches, stage_tot = [], 0, {}
    ev0.record(stream)
    for _ in range(a.steps):
        r = step()
        st = ws.stats()
        setup_ms.append(st["stage_ms"]["setup"])
        launches += st["kernel_launches"]
        for k, v in st["stage_ms"].items():
            stage_tot[k] = stage_tot.get(k, 0.0) + v
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / a.steps
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    value = world * 4.0 * n / (ms / 1e3) / 1e9
    if rank != 0:
        ws.close()
        if dist:
            dist.destroy_process_group()
        return
    st = ws.stats()
    stages = {k: v / a.steps for k, v in stage_tot.items()}

    # roofline of the dominant single kernel: the set-up stencil (one launch per step)
    peak, peak_kind = peaks()
    setup_avg = statistics.mean(setup_ms)
    n_tiles = math.ceil(dims[0] / 32) * math.ceil(dims[1] / 4) * math.ceil(dims[2] / 4)
    # algorithmic bytes per launch: read f and f_hat (4 + 4), write g, the
    # descriptor and k (4 + 4 + 1) and the critical-point bitmap (1/8) per vertex
    alg_bytes = n * (4 + 4 + 4 + 4 + 1) + n / 8.0
    achieved = alg_bytes / (setup_avg / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": "k_stencil<SETUP>", "achieved": achieved, "peak": peak,
            "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
            "traffic": ncu_traffic("k_stencil<SETUP>", c["name"]),
            "algorithmic_bytes": alg_bytes, "launch_ms": setup_avg, "tiles": n_tiles}

    extras = {"sum_requests": st["sum_requests"], "sum_tiles": st["sum_tiles"], "sum_pairs": st["sum_pairs"],
              "iterations": r["iterations"], "status": r["status_name"], "n_edits": r["n_edits"],
              "n_lossless": r["n_lossless"], "n_critical": r["n_critical"], "passes": st["passes"],
              "stage_ms": stages, "mvertices_per_s": n / (ms / 1e3) / 1e6,
              "workspace_gib": ws.nbytes / 2 ** 30}
    if not a.no_extras:
        for mode in ("plain", "frontier"):
            if mode == a.mode:
                continue
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            step(mode, False)
            e0.record(stream)
            rm = step(mode, False)
            e1.record(stream)
            torch.cuda.synchronize()
            extras[f"{mode}_ms"] = e0.elapsed_time(e1)
            extras[f"{mode}_gbs"] = 4.0 * n / (extras[f"{mode}_ms"] / 1e3) / 1e9
            extras[f"{mode}_same_result"] = bool(torch.equal(g.view(torch.int32), r["g"].view(torch.int32))) and \
                rm["iterations"] == r["iterations"]
        extras[f"{a.mode}_ms"] = ms
        if "plain_ms" in extras:
            extras["speedup_vs_plain"] = extras["plain_ms"] / ms

    e2e = None
    if not a.no_e2e:
        fc = f.cpu().pin_memory()
        hc = fh.cpu().pin_memory()
        gc = torch.empty_like(fc).pin_memory()
        ec = torch.empty((cap, 16), dtype=torch.uint8).pin_memory()
        ws.correct([fc], [hc], [xi], g_out=[gc], edit_bufs=[ec], host_buffers=True, mode=a.mode)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            rh = ws.correct([fc], [hc], [xi], g_out=[gc], edit_bufs=[ec], host_buffers=True, mode=a.mode)[0]
        torch.cuda.synchronize()
        ems = 1e3 * (time.perf_counter() - t0) / a.steps
        e2e = {"value": 4.0 * n / (ems / 1e3) / 1e9, "unit": "GB/s", "ms_per_step": ems,
               "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 4 * n + 16 * min(rh["n_edits"], cap) + 48,
               "same_result": bool(torch.equal(gc.view(torch.int32), g.cpu().view(torch.int32)))}

    cpu = None
    if not a.no_cpu and world == 1:
        fn, hn = f.cpu().numpy(), fh.cpu().numpy()
        side = choose_side(fn, hn, xi, 15.0)
        t, ro = oracle_sample(fn, hn, xi, side)
        cpu = {"value": 4.0 * side ** 3 / t / 1e9, "unit": "GB/s", "cores": omp_threads(), "kind": "oracle",
               "sample": f"{side}^3 corner crop of this workload, plain oracle to fixpoint "
                         f"({ro['iterations']} passes, {t:.1f} s)"}

    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": a.steps,
            "warmup": max(3, a.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": describe(c), "mode": a.mode, "l2": "inputs larger than L2 (4n bytes per field)",
                       "parallelism": f"replicas x{world}", "tuning": tuning},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches * 1,
            "clocks": clk, "extras": extras}
    print(json.dumps(line), flush=True)
    ws.close()
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------- many fields
def run_batched(a):
    """256 uneven fields corrected in one run (one launch per stage per pass over
    all fields, CUDA-graph loop) against the same fields one call at a time."""
    import torch

    import paper_2604_01397_b300 as ez
    import synth

    specs = synth.batched_specs(count=a.fields)
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    fs, fhs, xis = [], [], []
    for sp in specs:
        f, fh, xi = synth.make_case(sp["kind"], sp["dims"], sp["seed"], sp["rel"], sp["fhat"],
                                    n_bumps=sp["n_bumps"], sigma=sp["sigma"], device=dev)
        fs.append(f)
        fhs.append(fh)
        xis.append(xi)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    dims = [sp["dims"] for sp in specs]
    n_total = sum(f.numel() for f in fs)
    ws = ez.Workspace(dims)
    gs = [torch.empty_like(f) for f in fs]
    caps = [min(f.numel(), 1 << 22) for f in fs]
    ebufs = [torch.empty((c, 16), dtype=torch.uint8, device=dev) for c in caps]
    stream = torch.cuda.current_stream()

    def batched(mode="graph"):
        return ws.correct(fs, fhs, xis, mode=mode, g_out=gs, edit_bufs=ebufs)

    tuning = ws.autotune(fs, fhs, xis, repeats=1) if not a.no_autotune else ws.tuning()

    for _ in range(max(3, a.warmup)):
        rs = batched()
    torch.cuda.synchronize()
    clocks = Clocks(dev.index, enabled=not a.no_clocks)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    e0.record(stream)
    for _ in range(a.steps):
        rs = batched()
        launches += ws.stats()["kernel_launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / a.steps
    st = ws.stats()

    # the same fields one call at a time, each with its own workspace (made beforehand)
    per = [ez.Workspace([d]) for d in dims]
    g1 = [torch.empty_like(f) for f in fs]
    loop_ms = {}
    same = True
    for mode in ("graph", "plain"):
        for i in range(len(fs)):  # warm-up: graphs captured, caches primed
            per[i].correct([fs[i]], [fhs[i]], [xis[i]], mode=mode, g_out=[g1[i]], edit_bufs=[ebufs[i]])
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(len(fs)):
            r1 = per[i].correct([fs[i]], [fhs[i]], [xis[i]], mode=mode, g_out=[g1[i]], edit_bufs=[ebufs[i]])[0]
            same &= r1["iterations"] == rs[i]["iterations"] and r1["status"] == rs[i]["status"]
        e1.record(stream)
        torch.cuda.synchronize()
        loop_ms[mode] = e0.elapsed_time(e1)
        same &= all(torch.equal(g1[i].view(torch.int32), gs[i].view(torch.int32)) for i in range(len(fs)))
    for w in per:
        w.close()
    value = 4.0 * n_total / (ms / 1e3) / 1e9
    iters = [r["iterations"] for r in rs]
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": 1, "steps": a.steps,
            "warmup": max(3, a.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{len(fs)} fields, axes U{{32..256}}, Gaussian bumps (volume/4096, sigma~U[2,8]) "
                                   f"+ N(0,0.01), seeds 1000+j, xi 1e-3/1e-4 alternating, f_hat = f + U(-xi,xi)",
                       "vertices": n_total, "mode": "graph, all fields in one run", "parallelism": "replicas x1",
                       "tuning": tuning},
            "gpu_launches": launches, "clocks": clk,
            "extras": {"per_field_graph_ms": loop_ms["graph"], "per_field_plain_ms": loop_ms["plain"],
                       "speedup_vs_per_field_graph": loop_ms["graph"] / ms,
                       "speedup_vs_per_field_plain": loop_ms["plain"] / ms,
                       "per_field_plain_gbs": 4.0 * n_total / (loop_ms["plain"] / 1e3) / 1e9,
                       "same_results": bool(same), "passes": st["passes"], "max_iterations": max(iters),
                       "mean_iterations": statistics.mean(iters), "generation_s": gen_s,
                       "workspace_gib": ws.nbytes / 2 ** 30}}
    print(json.dumps(line), flush=True)
    ws.close()


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batched":
        run_batched(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
