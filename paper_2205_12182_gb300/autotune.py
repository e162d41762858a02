"""Autotuner of the product schedule: time the Newton-Schulz products of the mixed path at each padded
dimension under every schedule the library implements and keep, per n_pad, the fastest one.

For every n_pad of the grid a batch of uncoupled dense blocks of dimension n_pad - 8
(``synth.dense_blocks``: every index set has exactly that many entries; the batch holds about as
many flops per iteration as 4,096 blocks of 480, as for the p(n) table of Eq. 10) is built once and
evaluated at mu = -0.25 Ha, inside the blocks' spectral gap, under

* NOLSM_SCHEDULE_PERSISTENT (one launch per evaluation, one block per 2-CTA cluster),
* NOLSM_SCHEDULE_PERSISTENT_INTERLEAVED (two blocks per cluster),
* NOLSM_SCHEDULE_PER_PRODUCT (one launch per product, host-driven iteration),

after one warm-up evaluation each; the products' device time (the stage timer) over `reps`
evaluations decides.  The table (weights/schedule_gb300.json) is what nolsm_set_schedule_table
takes: NOLSM_SCHEDULE_AUTO then runs, in every sign evaluation, the blocks whose n_pad prefers a
persistent schedule in one persistent launch and the others in per-product launches.

    python -m paper_2205_12182_gb300.autotune [--out paper_2205_12182_gb300/weights/schedule_gb300.json]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2205_12182_gb300.measure_pn import MU_GAP, batch_size  # noqa: E402

GRID = (128, 256, 384, 512, 640, 768, 896, 1024, 1280, 1536, 1792, 2048, 2560, 3072, 3584, 4096)


def time_schedules(nolsm, n_pad: int, reps: int = 3, seed: int = 0):
    """Products ms per sign evaluation of each schedule on one batch at n = n_pad - 8."""
    from synth import dense_blocks
    n = n_pad - 8
    nb = batch_size(n)
    system = dense_blocks(n, nb, seed, n_unique=min(nb, 4))
    out = {}
    names = (("persistent", nolsm.SCHEDULE_PERSISTENT), ("interleaved", nolsm.SCHEDULE_PERSISTENT_INTERLEAVED),
             ("per_product", nolsm.SCHEDULE_PER_PRODUCT))
    lib = None
    for name, sched in names:
        lib = nolsm.Nolsm(schedule=sched).build(system)
        lib.sign_batch(MU_GAP)                     # warm-up
        lib.phase_times(reset=True)
        iters = 0.0
        for _ in range(reps):
            iters += lib.sign_batch(MU_GAP)["iters_avg"]
        out[name] = lib.phase_times(reset=True)["products"] / reps
        lib.close()
    del system
    return nb, out, iters / reps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "weights", "schedule_gb300.json"))
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args()
    import torch
    from paper_2205_12182_gb300.build import build
    build()
    from paper_2205_12182_gb300 import nolsm
    torch.cuda.set_device(0)
    t0 = time.time()
    kinds = {"persistent": nolsm.SCHEDULE_PERSISTENT, "interleaved": nolsm.SCHEDULE_PERSISTENT_INTERLEAVED,
             "per_product": nolsm.SCHEDULE_PER_PRODUCT}
    rows = []
    for n_pad in GRID:
        nb, ms, iters = time_schedules(nolsm, n_pad, a.reps)
        best = min(ms, key=ms.get)
        rows.append((n_pad, nb, ms, best, iters))
        print(f"n_pad={n_pad:5d} blocks={nb:5d} iters={iters:5.2f} " +
              " ".join(f"{k}={v:8.3f} ms" for k, v in ms.items()) + f"  -> {best} ({time.time() - t0:.0f} s)",
              flush=True)
    out = {"what": "products ms per sign evaluation of each schedule on dense blocks of n = n_pad - 8 at mu in "
                   "their gap; schedule = nolsm_schedule of the fastest",
           "device": torch.cuda.get_device_name(0), "precision": "library default (mixed FP16)",
           "command": "python -m paper_2205_12182_gb300.autotune " + " ".join(sys.argv[1:]),
           "n_pad": [r[0] for r in rows], "schedule": [kinds[r[3]] for r in rows],
           "schedule_name": [r[3] for r in rows], "blocks": [r[1] for r in rows],
           "iters_avg": [round(r[4], 3) for r in rows],
           "ms": {k: [round(r[2][k], 4) for r in rows] for k in kinds}}
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    with open(a.out, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {a.out} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
