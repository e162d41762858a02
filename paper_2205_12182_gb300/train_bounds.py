"""Train the spectral-bound predictor on submatrix spectra that the method itself computes.

For every training system -- seeded water boxes with the 8 A neighbourhood and protein-like
globules (the 10-200-atom blocks of 30,000-atom systems, n_b 160-2,700), all held apart from the
benchmark seeds -- the library builds the submatrices in FP32, and for a set of chemical potentials
it evaluates the sign and then runs Lanczos:

* on A0 (64 steps): lambda_min, lambda_max -- the targets of outputs 0 and 1;
* on |A0 - mu| = X (A0 - mu) with X the FP32 sign iterate (64 steps): the distance from mu to the
  nearest eigenvalue -- log10 of it is the target of output 2;

and the 32 block features at mu are the inputs.  Training runs the library's own kernels
(nolsm_mlp_gradient, nolsm_mlp_adam).  The weights go to a raw float32 file plus JSON metadata.

    python -m paper_2205_12182_gb300.train_bounds [--out paper_2205_12182_gb300/weights/bounds_mlp]
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

TRAIN_SEEDS_4096 = (100, 101, 102, 103, 104)
TRAIN_SEEDS_1000 = tuple(range(110, 120))
TRAIN_SEEDS_GLOBULE = tuple(range(100, 112))
HELDOUT = ((16, 11), (16, 200), (12, 201))
HELDOUT_GLOBULE = (200, 201, 202)
MU_OFFSETS = (-0.05, -0.02, -0.01, 0.0, 0.01, 0.02, 0.05)


def system_samples(nolsm, system, n_random_mu=2, seed=0, steps=64):
    """(features, targets) for every block at several mu around the gap and inside the bands."""
    import torch
    lib = nolsm.Nolsm(precision=nolsm.PREC_FP32, chol_precision=nolsm.CHOL_FP32).build(system)
    mu0, _, _ = lib.set_mu(system.n_electrons, tol_n=1e-3)
    lz = lib.lanczos(steps, op=0)
    lo, hi = lib.bounds()
    rng = np.random.default_rng(seed)
    mus = [mu0 + d for d in MU_OFFSETS] + list(rng.uniform(lz[:, 0].min().item(), lz[:, 1].max().item(), n_random_mu))
    mus.append(0.5 * (lo.min() + hi.max()))        # the first midpoint of the default bisection
    xs, ys = [], []
    for mu in mus:
        lib.sign_batch(mu)
        dist = lib.lanczos(steps, op=1)[:, 0].clamp_min(1e-8)
        xs.append(lib.features(mu))
        ys.append(torch.stack([lz[:, 0], lz[:, 1], torch.log10(dist)], dim=1))
    lib.close()
    return torch.cat(xs), torch.cat(ys), mu0


def train(nolsm, x, y, epochs=40, batch=512, lr=2e-3, seed=0, log=print):
    import torch
    xm, xsd = x.mean(0).cpu().numpy(), x.std(0).cpu().numpy()
    ym, ysd = y.mean(0).cpu().numpy(), y.std(0).cpu().numpy()
    xsd = np.where(xsd < 1e-6, 1.0, xsd)
    ysd = np.where(ysd < 1e-6, 1.0, ysd)
    norm = np.concatenate([xm, xsd, ym, ysd]).astype(np.float32)
    # initial weights: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)), zero biases, in the library's order
    rng = np.random.default_rng(seed)
    parts = []
    for fi, fo in ((32, 128), (128, 128), (128, 3)):
        lim = 1.0 / np.sqrt(fi)
        parts += [rng.uniform(-lim, lim, size=fo * fi), np.zeros(fo)]
    bp = nolsm.BoundPredictor(np.concatenate(parts).astype(np.float32), norm)
    n = x.shape[0]
    hist = []
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).to(x.device)
        xe, ye = x[perm].contiguous(), y[perm].contiguous()
        tot = 0.0
        step_lr = lr * (0.5 * (1 + np.cos(np.pi * ep / epochs)) * 0.95 + 0.05)
        for s in range(0, n, batch):
            xb, yb = xe[s:s + batch], ye[s:s + batch]
            tot += bp.gradient(xb, yb) * xb.shape[0]
            bp.adam(lr=step_lr)
        hist.append(tot / n)
        if ep % 10 == 0 or ep == epochs - 1:
            log(f"epoch {ep:3d} loss {tot / n:.5f}")
    return bp, hist


def iteration_study(nolsm, bp, system, mu):
    """Average NS iterations and accuracy proxies at mu for Gershgorin bounds (the library's default
    lower bound 0.02, and the uninformed 1e-3), Lanczos and learned bounds."""
    out = {}
    for name, kw in (("gershgorin", {}), ("gershgorin_lower_bound_1e-3", {"lower_bound": 1e-3}),
                     ("lanczos", {"bounds": nolsm.BOUNDS_LANCZOS}), ("learned", {"bounds": nolsm.BOUNDS_LEARNED})):
        lib = nolsm.Nolsm(precision=nolsm.PREC_MIXED_FP16, **kw).build(system)
        if name == "learned":
            lib.set_predictor(bp)
        st = lib.sign_batch(mu)
        out[name] = {"iters_avg": st["iters_avg"], "iters_max": st["iters_max"], "n_electrons": st["n_electrons"],
                     "restarted": st["n_restarted"], "ms": st["ms"]}
        lib.close()
    return out


def _globule(seed):
    from synth import protein_globule
    return protein_globule(seed, name=f"globule30000-s{seed}")


def globules(seeds):
    """Globule systems generated in parallel on the host cores (a spawn pool: numpy work only)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(len(seeds), os.cpu_count() or 1)) as pool:
        return pool.map(_globule, list(seeds))


def main():
    import torch
    from paper_2205_12182_gb300.build import build
    build()
    from synth import water_box

    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "weights", "bounds_mlp"))
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--quick", action="store_true", help="two small training systems (smoke run)")
    a = ap.parse_args()
    t0 = time.time()
    g_train = globules(TRAIN_SEEDS_GLOBULE[:1] if a.quick else TRAIN_SEEDS_GLOBULE)
    g_held = [] if a.quick else globules(HELDOUT_GLOBULE)
    print(f"globules generated ({time.time() - t0:.1f} s)", flush=True)
    from paper_2205_12182_gb300 import nolsm
    torch.cuda.set_device(0)
    xs, ys = [], []
    specs = [(10, s) for s in TRAIN_SEEDS_1000[:2]] if a.quick else \
        [(16, s) for s in TRAIN_SEEDS_4096] + [(10, s) for s in TRAIN_SEEDS_1000]
    for side, seed in specs:
        sysm = water_box(side, seed, neighbourhood=8.0)
        x, y, _ = system_samples(nolsm, sysm, seed=seed)
        xs.append(x)
        ys.append(y)
        print(f"system side={side} seed={seed}: {x.shape[0]} samples ({time.time() - t0:.1f} s)", flush=True)
    for g in g_train:
        x, y, _ = system_samples(nolsm, g, seed=len(xs))
        xs.append(x)
        ys.append(y)
        print(f"system {g.name}: {x.shape[0]} samples ({time.time() - t0:.1f} s)", flush=True)
    x, y = torch.cat(xs), torch.cat(ys)
    bp, hist = train(nolsm, x, y, epochs=a.epochs)
    report = {"train_samples": int(x.shape[0]),
              "train_systems": [list(s) for s in specs] + [g.name for g in g_train], "loss": hist[-1],
              "heldout": []}
    for side, seed in ([] if a.quick else HELDOUT):
        sysm = water_box(side, seed, neighbourhood=8.0)
        xh, yh, mu0 = system_samples(nolsm, sysm, n_random_mu=0, seed=seed)
        pred = bp.predict(xh)
        err = (pred - yh).abs().mean(0).cpu().numpy()
        study = iteration_study(nolsm, bp, sysm, mu0)
        report["heldout"].append({"side": side, "seed": seed, "mu": mu0,
                                  "mae": {"lambda_min": float(err[0]), "lambda_max": float(err[1]),
                                          "log10_dist": float(err[2])}, "iterations": study})
        print(json.dumps(report["heldout"][-1]), flush=True)
    for g in g_held:
        xh, yh, mu0 = system_samples(nolsm, g, n_random_mu=0, seed=0)
        err = (bp.predict(xh) - yh).abs().mean(0).cpu().numpy()
        study = iteration_study(nolsm, bp, g, mu0)
        report["heldout"].append({"system": g.name, "mu": mu0,
                                  "mae": {"lambda_min": float(err[0]), "lambda_max": float(err[1]),
                                          "log10_dist": float(err[2])}, "iterations": study})
        print(json.dumps(report["heldout"][-1]), flush=True)
    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    bp.save(a.out, meta={"trained_on": report["train_systems"], "train_samples": report["train_samples"],
                         "final_loss": report["loss"]})
    with open(a.out + "_report.json", "w") as f:
        json.dump(report, f, indent=1)
    print(f"saved {a.out}.json / .bin in {time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()
