"""Measure p(n), the time per flop of the sign iteration's matrix products at submatrix dimension n,
for the performance-aware combination of submatrices (Section III-B-1, Eq. 10).

For every n of the grid a batch of uncoupled dense blocks of dimension n (``synth.dense_blocks``:
every index set has exactly n entries) goes through nolsm_build_submatrices and then
nolsm_sign_batch at mu = -0.25 Ha, inside the blocks' spectral gap.  After one warm-up evaluation,
p(n) = device time of the products phase (CUDA events) / the products' flops counted as the paper
counts them (2 n^3 per product at the true n, so the padding to whole tiles is part of p), summed
over `reps` evaluations.  The batch holds about as many flops per iteration as 4,096 blocks of 480
(at least 4 blocks, at most 16,384 and 1e8 stored entries), in the precision and schedule the
library uses by default.

With ``--what step`` the numerator is instead the device time of every stage of one full step
of the batch (build, one sign evaluation, density, band energy), still divided by 2 n^3 per block
and product: Eq. 10's comparison of predicted run times applied to the whole step rather than to
the matrix function alone (not in the paper; the paper's setting spends its time in the matrix
function, a step whose mu search needs one sign evaluation spends it in the build).

    python -m paper_2205_12182_gb300.measure_pn [--out paper_2205_12182_gb300/weights/pn_gb300.json]
                                               [--what products|step] [--step 64] [--max 4096] [--reps 3]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

MU_GAP = -0.25


def batch_size(n: int, max_entries: float = 1e8) -> int:
    b = int(round(4096 * (480.0 / n) ** 3))
    b = min(b, 16384, int(max_entries) // (n * n))
    return max(b, 4)


def measure(nolsm, n: int, reps: int = 3, seed: int = 0, precision=None, max_entries: float = 1e8,
            what: str = "products"):
    from synth import dense_blocks
    nb = batch_size(n, max_entries)
    system = dense_blocks(n, nb, seed, n_unique=min(nb, 4))
    kw = {} if precision is None else {"precision": precision}
    lib = nolsm.Nolsm(**kw).build(system)
    lib.sign_batch(MU_GAP)                          # warm-up
    if what == "step":
        lib.density()
        lib.band_energy()
    lib.phase_times(reset=True)
    flops, iters = 0.0, 0.0
    for _ in range(reps):
        if what == "step":
            lib.build(system)
        st = lib.sign_batch(MU_GAP)
        if what == "step":
            lib.density()
            lib.band_energy()
        flops += st["flops_paper"]
        iters += st["iters_avg"]
    phases = lib.phase_times(reset=True)
    ms = phases["products"] if what == "products" else sum(phases.values())
    lib.close()
    del system
    return {"n": n, "blocks": nb, "ms": ms / reps, "flops": flops / reps, "iters_avg": iters / reps,
            "time_per_flop": ms * 1e-3 / flops, "tflops": flops / (ms * 1e-3) / 1e12}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "weights", "pn_gb300.json"))
    ap.add_argument("--step", type=int, default=64)
    ap.add_argument("--min", type=int, default=64)
    ap.add_argument("--max", type=int, default=4096)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--what", choices=["products", "step"], default="products")
    a = ap.parse_args()
    import torch
    from paper_2205_12182_gb300.build import build
    build()
    from paper_2205_12182_gb300 import nolsm
    torch.cuda.set_device(0)
    t0 = time.time()
    rows = []
    for n in range(a.min, a.max + 1, a.step):
        r = measure(nolsm, n, a.reps, what=a.what)
        rows.append(r)
        print(f"n={n:5d} blocks={r['blocks']:6d} iters={r['iters_avg']:5.2f} {a.what} {r['ms']:8.3f} ms "
              f"{r['tflops']:7.1f} TFLOP/s ({time.time() - t0:.0f} s)", flush=True)
    out = {"what": ("time per flop (s) of the Newton-Schulz products at true dimension n, 2 n^3 per product"
                    if a.what == "products" else
                    "device time (s) of one full step (build, one sign evaluation, density, band energy) per "
                    "flop of the step's products at true dimension n, 2 n^3 per product"),
           "device": torch.cuda.get_device_name(0), "precision": "library default (mixed FP16)",
           "command": "python -m paper_2205_12182_gb300.measure_pn " + " ".join(sys.argv[1:]),
           "n": [r["n"] for r in rows], "time_per_flop": [r["time_per_flop"] for r in rows],
           "tflops": [round(r["tflops"], 2) for r in rows], "blocks": [r["blocks"] for r in rows],
           "iters_avg": [round(r["iters_avg"], 3) for r in rows]}
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    with open(a.out, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {a.out} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
