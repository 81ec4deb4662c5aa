#!/usr/bin/env python
"""Write the oracle's digests of full-size corrections to tests/golden/fullsize.json.

Every value stored here comes from the oracle (``oracle.correct``, Algorithm 1
with the EG constraints of Sec. 4.2 and the event constraints of Sec. 4.3, or
the original ones of Sec. 4.2) on inputs made by ``synth`` on the CPU; nothing
is read from the CUDA library.  The GPU tests regenerate the same inputs on
the CPU (their SHA-256 is stored and checked first), run the CUDA path and
compare its g, edit list and counters with these digests.

Cases (the workloads the benchmark times, at full size):
  octave1024/rel<r>  1024^3 three-octave noise, seed 2, f_hat by
                     2xi-quantisation, xi = r * range, r in {1e-2, 1e-3, 1e-4};
                     oracle worklist mode (bit-identical to the plain mode),
                     OpenMP on the host cores
  batched256/<j>     field j of the 256-field batch (axes U{32..256}, bumps,
                     seed 1000 + j, f_hat = f + U(-xi, xi)); worklist mode
  bumps512/original  512^3 bumps (seed 1) under the original event
                     constraints; the oracle's event mode (full sweeps)

  python tests/golden/make_fullsize.py octave1024/rel1e-4 [more cases ...]
  python tests/golden/make_fullsize.py batched256
Each case runs in its own process (a 1024^3 case holds about 54 GB of host
memory); results are merged into the JSON file.
"""
from __future__ import annotations

import json
import os
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "fullsize.json")
N_STEPS = 5


def _merge(entries: dict):
    data = {"cases": {}}
    if os.path.exists(OUT):
        data = json.load(open(OUT))
    data["note"] = ("Oracle digests of full-size corrections (written by tests/golden/make_fullsize.py, which "
                    "calls only oracle/ and synth/).  Edit lists are hashed as 16-byte records "
                    "(tests/golden/fullsize_digest.py); g and the inputs as their float32 bytes in index order.")
    data["cases"].update(entries)
    data["cases"] = dict(sorted(data["cases"].items()))
    tmp = OUT + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1)
        fh.write("\n")
    os.replace(tmp, OUT)


def _one(name: str, spec: dict, events: bool) -> dict:
    import torch

    import oracle
    import synth
    from tests.golden.fullsize_digest import sha_array, sha_edits_from_kg, xi_bits

    t0 = time.time()
    nthreads = torch.get_num_threads()
    torch.set_num_threads(1)  # the inputs do not depend on it; it also sets the OpenMP threads of the oracle
    f, fh, xi = synth.make_case(spec["kind"], spec["dims"], spec["seed"], spec["rel"], spec["fhat"],
                                n_bumps=spec.get("n_bumps"), sigma=spec.get("sigma", (2.0, 8.0)), device="cpu")
    torch.set_num_threads(nthreads)
    f = f.numpy().reshape(-1)
    fh = fh.numpy().reshape(-1)
    t1 = time.time()
    r = oracle.correct(f, fh, xi, dims=spec["dims"], N=N_STEPS, worklist=not events, events=events,
                       edit_list=False)
    t2 = time.time()
    return {"kind": spec["kind"], "dims": list(spec["dims"]), "seed": spec["seed"], "rel": spec["rel"],
            "fhat": spec["fhat"], "n_bumps": spec.get("n_bumps"), "sigma": list(spec.get("sigma", (2.0, 8.0))),
            "events": "original" if events else "reformulated", "N": N_STEPS,
            "xi_bits": xi_bits(xi), "f_sha256": sha_array(f), "fhat_sha256": sha_array(fh),
            "g_sha256": sha_array(r["g"]), "edits_sha256": sha_edits_from_kg(r["k"], r["g"], N_STEPS),
            "iterations": r["iterations"], "status": r["status"], "status_name": oracle.STATUS_NAMES[r["status"]],
            "residual": r["residual"], "n_edits": r["n_edits"], "n_lossless": r["n_lossless"],
            "oracle_mode": "events (full sweeps)" if events else "worklist",
            "oracle_s": round(t2 - t1, 1), "generate_s": round(t1 - t0, 1)}


def run_case(name: str) -> dict:
    import synth
    from synth.fields import WORKLOADS

    if name.startswith("octave1024/rel"):
        c = dict(WORKLOADS["octave1024"])
        c["rel"] = float(name.split("/rel")[1])
        return {name: _one(name, c, False)}
    if name == "bumps512/original":
        return {name: _one(name, dict(WORKLOADS["bumps512"]), True)}
    if name == "batched256":
        out = {}
        for j, sp in enumerate(synth.batched_specs(count=256)):
            key = f"batched256/{j:03d}"
            out[key] = _one(key, sp, False)
            print(key, out[key]["iterations"], out[key]["status_name"], out[key]["oracle_s"], flush=True)
        return out
    raise SystemExit(f"unknown case {name}")


def main(argv):
    if len(argv) >= 2 and argv[0] == "--child":
        sys.path.insert(0, ROOT)
        res = run_case(argv[1])
        _merge(res)
        for k, v in res.items():
            if not k.startswith("batched256/"):
                print(k, json.dumps(v), flush=True)
        return
    for name in argv:
        subprocess.run([sys.executable, os.path.abspath(__file__), "--child", name], check=True, cwd=ROOT)


if __name__ == "__main__":
    main(sys.argv[1:])
