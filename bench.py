"""Benchmark: one full NOLSM density solve per step on the 4,096-molecule water system.

A step is the whole hot path on one batch of synthetic input already resident in HBM:
nolsm_build_submatrices (gather, Cholesky, inverse, congruence, bounds) + nolsm_set_mu
(bisection; every step a batched Newton-Schulz sign over all blocks) + nolsm_density (scatter)
+ nolsm_band_energy.  The metric is atoms per second of converged solves; the line also gives
the sign-product TFLOP/s (the paper's 2 n^3 per product and as executed), the roofline of the
dominant kernel, the end-to-end figure through host buffers, and the FP64 CPU oracle's rate.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank solves its own seeded box and the ranks share
one chemical potential: the electron count N(mu) is summed over ranks (NCCL all-reduce of one
float64) at every bisection step -- weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = {"workload": "water-4096", "molecules": 4096, "atoms": 12288, "basis": 24576, "box_A": 49.6,
            "blocks": 4096, "index_rule": "pattern + 8 A neighbourhood", "seed": 11}
METRIC = "atoms/s & sign-GEMM TFLOP/s (% FP16 peak) at max|dD|<=1e-3 vs FP32 plain"
TOL_N = 1e-3
WEIGHTS = os.path.join(ROOT, "paper_2205_12182_gb300", "weights", "bounds_mlp.json")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d["bf16_tflops_sustained"], "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------ our arm

def solve(lib, system, mu_fn, d_out, memory):
    """One full step: build, bisection, density, band energy."""
    from paper_2205_12182_gb300 import nolsm
    lib.build(system, memory=memory)
    mu, n, steps = mu_fn(lib, system)
    lib.density(d_out, memory=nolsm.MEM_HOST if memory == "host" else nolsm.MEM_DEVICE)
    e = lib.band_energy()
    return mu, n, steps, e


def run_ours(args):
    import torch
    from paper_2205_12182_gb300 import nolsm
    from paper_2205_12182_gb300.distributed import set_mu_distributed
    from synth import make_config, water_box

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    lpt = world > 1 and args.partition == "lpt"
    seed = WORKLOAD["seed"] + (0 if lpt else rank)
    if args.side != 16:
        system = water_box(args.side, seed=seed, neighbourhood=8.0)
        WORKLOAD.update(workload=f"water-{args.side ** 3}", molecules=args.side ** 3, atoms=3 * args.side ** 3,
                        basis=6 * args.side ** 3, box_A=3.1 * args.side, blocks=args.side ** 3)
    else:
        system = make_config(2, seed=seed)
    n_e_global = system.n_electrons * (1 if lpt else world)
    if lpt:
        # one system, its blocks dealt to the ranks by LPT on their predicted cost (strong scaling)
        from paper_2205_12182_gb300.distributed import block_cost_estimate, lpt_partition
        system = system.subset_blocks(lpt_partition(block_cost_estimate(system), world)[rank])

    def mu_fn(lib, s):
        if world == 1:
            return lib.set_mu(s.n_electrons, tol_n=TOL_N)
        return set_mu_distributed(lib, n_e_global, tol_n=TOL_N, group=None)

    predictor = nolsm.BoundPredictor.load(WEIGHTS)
    lib = nolsm.Nolsm(precision=nolsm.PREC_MIXED_FP16, bounds=nolsm.BOUNDS_LEARNED)
    lib.set_predictor(predictor)
    d_dev = torch.empty(system.nnz, dtype=torch.float64, device=dev)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        solve(lib, system, mu_fn, d_dev, "device")
    barrier()
    lib.counters(reset=True)
    lib.phase_times(reset=True)
    phase = {"steps": []}
    with ClockSampler(local) as clk:
        barrier()
        t0 = time.perf_counter()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            mu, n, steps, e = solve(lib, system, mu_fn, d_dev, "device")
            phase["steps"].append(steps)
        ev1.record()
        barrier()
        wall = time.perf_counter() - t0
    dev_ms = ev0.elapsed_time(ev1)
    _CLOCK_MAX["mhz"] = clk.summary().get("sm_max_mhz")
    cnt = lib.counters(reset=True)
    stage_ms = {k: v / args.steps for k, v in lib.phase_times(reset=True).items()}
    t_step = max(wall, dev_ms / 1000.0) / args.steps
    if dist is not None:
        tt = torch.tensor([t_step], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step = float(tt.item())

    # end to end: host-resident CSR in (copied by the library), D back to pinned host memory
    d_host = torch.empty(system.nnz, dtype=torch.float64).pin_memory()
    solve(lib, system, mu_fn, d_host, "host")
    barrier()
    t1 = time.perf_counter()
    for _ in range(args.steps):
        solve(lib, system, mu_fn, d_host, "host")
    barrier()
    t_e2e = (time.perf_counter() - t1) / args.steps
    if dist is not None:
        tt = torch.tensor([t_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_e2e = float(tt.item())
    h2d = system.row_ptr.astype(np.int64).nbytes + system.col.astype(np.int32).nbytes + 2 * system.nnz * 8
    d2h = system.nnz * 8 + 8 * 3

    # D of this run on sampled blocks, compared with the oracle in the cpu_baseline leg (not timed)
    checks = {}
    if rank == 0 and not args.no_parity:
        checks["headline"] = (system, d_host.numpy().copy(), mu, 8)

    atoms = WORKLOAD["atoms"] * (1 if lpt else world)
    pk = peaks()
    gemm_tflops = cnt["gemm_flops"] / (cnt["gemm_ms"] * 1e-3) / 1e12 if cnt["gemm_ms"] > 0 else None
    frac = gemm_tflops / pk["bf16_tflops_sustained"] if gemm_tflops else None
    st = lib.sign_batch(mu)   # statistics of one evaluation at the converged mu (not timed)
    n_b = np.array([nolsm.nolsm_block_info(lib.ctx, b)[0] for b in range(system.n_blocks)], np.float64)
    # useful flops of the symmetric products: n_b^2 (n_b + 1) per product at the true n_b (one
    # triangle and the diagonal of X X^T), 2 i_b + 1 products per block; every timed step ran the
    # same evaluations at the same mu, so the timed region's useful flops are its executed flops
    # times this evaluation's useful / executed ratio
    prod_b = 2.0 * lib.iters().astype(np.float64) + 1.0
    useful_eval = float(np.sum(prod_b * n_b * n_b * (n_b + 1.0)))
    useful_ratio = useful_eval / st["flops_executed"]
    roofs = rooflines(stage_ms, cnt, args.steps, n_b, pk, clk_max_mhz(), torch.cuda.get_device_properties(dev),
                      products_per_launch=float(prod_b.sum()), useful_ratio=useful_ratio)
    dominant = max(roofs, key=lambda r: r["ms_per_step"])
    line = {
        "metric": METRIC,
        "value": atoms / t_step,
        "unit": "atoms/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_step * 1e3,
        "higher_is_better": True,
        "scaling": "strong" if lpt else "weak",
        "vs_baseline": None,
        "dtype": "f16",
        "data": "synthetic (seeded water boxes; no dataset)",
        "config": dict(WORKLOAD, mu_tol_rel=TOL_N, bounds="learned (predictor weights committed, trained on other seeds)",
                       precision="FP16 operands / FP32 accumulate; S factor in double-float (48-bit)",
                       l2="working set > 10 GB >> 129 MB L2 (no flush needed)",
                       parallelism=(f"dp{world} (one system, blocks dealt to the ranks by LPT, shared mu)" if lpt
                                    else f"dp{world} (one box per rank, shared mu)")),
        "sign_gemm": {
            "tflops_executed": gemm_tflops,
            "tflops_paper_convention": (cnt["gemm_flops"] * st["flops_paper"] / st["flops_executed"])
            / (cnt["gemm_ms"] * 1e-3) / 1e12 if cnt["gemm_ms"] > 0 else None,
            "pct_fp16_peak_measured": 100 * frac if frac else None,
            "gemm_ms_per_step": cnt["gemm_ms"] / args.steps,
            "tflops_useful": gemm_tflops * useful_ratio if gemm_tflops else None,
            "pct_fp16_peak_measured_useful": 100 * frac * useful_ratio if frac else None,
            "useful_flops": "n_b^2 (n_b + 1) per symmetric product at the true n_b",
            "ms_per_mu_iteration": st["ms"],   # one sign evaluation at the converged mu (the paper's T_NOLSM unit)
            "ns_iters_avg": st["iters_avg"],
            "mu_steps": phase["steps"][-1],
        },
        "mu_search": {"first_point": "Aufbau estimate (nolsm_set_mu)", "tol_n_rel": TOL_N,
                      "evaluations_per_step": phase["steps"][-1],
                      "n_electrons": n, "n_target": float(n_e_global),
                      "count_error_rel": abs(n - n_e_global) / n_e_global,
                      "ms_per_mu_iteration": st["ms"]},
        "roofline": dominant,
        "rooflines": roofs,
        "stage_ms_per_step": stage_ms,
        "e2e": {"value": atoms / t_e2e, "unit": "atoms/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(cnt["launches"]),
        "clocks": clk.summary(),
        "parity": None,
        "result": {"mu": mu, "n_electrons": n, "band_energy": e},
    }
    if not args.no_variants:
        line["variants"] = variants(nolsm, system, mu_fn, d_dev, predictor, barrier, world)
    want = rank == 0 and not args.no_parity
    if not args.no_combination and world == 1:
        line["combination"] = combination(nolsm, predictor, system, checks if want else None)
    if not args.no_large and world == 1:
        line["largest_blocks"] = large_blocks(nolsm, predictor, pk, checks if want else None)
    if not args.no_md and world == 1:
        line["md_steps"] = md_steps(nolsm, predictor, system, checks if want else None, keep_steps=args.keep_steps)
    if not args.no_globule and world == 1:
        from synth import atom_blocks, make_config
        g = make_config(3)
        # learned bounds (the predictor saw globules of other seeds), and Gershgorin bounds with the
        # default lower bound 0.02 beside them
        line["globule"] = combination(nolsm, predictor, g, checks if want else None, tag="globule", combine=False)
        line["globule"]["workload"] = (f"protein-like globule, {g.n_atoms} atoms ({g.n_basis} basis functions), "
                                       f"{g.n_blocks} blocks of 10-200 atoms, 8 A neighbourhood; learned bounds")
        gg = combination(nolsm, predictor, g, None, tag="globule_gershgorin", combine=False, bounds=0.02)
        line["globule"]["gershgorin_lower_bound_0.02"] = gg["none"]["measured"]
        line["globule_schedules"] = globule_schedules(nolsm, g)
        ga = atom_blocks(g)
        line["combination_globule"] = combination(nolsm, predictor, ga, checks if want else None,
                                                  tag="combination_globule", bounds=0.02)
        line["combination_globule"]["workload"] = (f"the same globule, one block per atom ({ga.n_blocks} blocks) "
                                                   "before combination, 8 A neighbourhood")
    if not args.no_million and world == 1:
        line["million_molecules"] = million_molecules(nolsm, predictor, pk, checks if want else None)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the cpu_baseline leg: the oracle timed on the host cores, then the parity spot checks
        line["cpu_baseline"] = cpu_baseline(system, seconds=args.cpu_seconds)
        for key, res in parity_checks(checks).items():
            if key == "headline":
                line["parity"] = res
            elif key in ("largest_blocks", "million_molecules"):
                line[key]["parity"] = res
            else:
                section, name = key.split(".", 1)
                line[section][name]["parity"] = res
    lib.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def variants(nolsm, system, mu_fn, d_dev, predictor, barrier, world, steps=2):
    """atoms/s of the same full step with other precision / bound choices (1 warm-up, `steps` timed)."""
    out = {}
    cases = {
        "fp32_plain": dict(precision=nolsm.PREC_FP32, scaled=0),
        "mixed_fp16_gershgorin": dict(precision=nolsm.PREC_MIXED_FP16),
        "mixed_fp16_learned_fp32_cholesky": dict(precision=nolsm.PREC_MIXED_FP16, bounds=nolsm.BOUNDS_LEARNED,
                                                 chol_precision=nolsm.CHOL_FP32),
        "mixed_fp16_learned_fp64_cholesky": dict(precision=nolsm.PREC_MIXED_FP16, bounds=nolsm.BOUNDS_LEARNED,
                                                 chol_precision=nolsm.CHOL_FP64),
        "mixed_fp16_learned_per_product_launches": dict(precision=nolsm.PREC_MIXED_FP16, bounds=nolsm.BOUNDS_LEARNED,
                                                        schedule=nolsm.SCHEDULE_PER_PRODUCT),
    }
    for name, kw in cases.items():
        lib = nolsm.Nolsm(**kw)
        if kw.get("bounds") == nolsm.BOUNDS_LEARNED:
            lib.set_predictor(predictor)
        solve(lib, system, mu_fn, d_dev, "device")
        barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            mu, n, st, e = solve(lib, system, mu_fn, d_dev, "device")
        barrier()
        dt = (time.perf_counter() - t0) / steps
        s = lib.sign_batch(mu)
        out[name] = {"value": WORKLOAD["atoms"] * world / dt, "unit": "atoms/s", "ms_per_step": dt * 1e3,
                     "mu_steps": st, "ns_iters_avg": s["iters_avg"]}
        lib.close()
    if world == 1:
        # plain bisection: the headline's path with the first point at the bracket midpoint (no Aufbau
        # estimate), stopping at |N - N_e| <= 1e-6 N_e or a bracket below 1e-10 Ha (nolsm_set_mu's rules)
        lib = nolsm.Nolsm(precision=nolsm.PREC_MIXED_FP16, bounds=nolsm.BOUNDS_LEARNED,
                          mu_first=nolsm.MU_FIRST_MIDPOINT)
        lib.set_predictor(predictor)
        bis = lambda lib_, s_: lib_.set_mu(s_.n_electrons, tol_n=1e-6)   # noqa: E731
        solve(lib, system, bis, d_dev, "device")
        barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            mu, n, st, e = solve(lib, system, bis, d_dev, "device")
        barrier()
        dt = (time.perf_counter() - t0) / steps
        out["bisection_from_bracket_tol1e-6"] = {
            "value": WORKLOAD["atoms"] / dt, "unit": "atoms/s", "ms_per_step": dt * 1e3, "mu_steps": st,
            "ms_per_mu_iteration": dt * 1e3 / st if st else None, "mu": mu, "n_electrons": n,
            "count_error_rel": abs(n - system.n_electrons) / system.n_electrons,
            "first_point": "bracket midpoint [min Gershgorin lo, max Gershgorin hi]",
            "stop": "|N - N_e| <= 1e-6 N_e, or bracket < 1e-10 Ha, or 60 evaluations"}
        lib.close()
    return out


def large_blocks(nolsm, predictor, pk, checks=None, steps=2, evals=3):
    """The block shape of the 1,000,000-molecule configuration -- 32-molecule clusters with an 8 A
    halo, n_b ~ 1,870 (n_pad 1,920) -- on a 13,824-molecule box (432 blocks): atoms/s of the full
    step (1 warm-up, `steps` timed) and the sign products' TFLOP/s over `evals` sign evaluations at
    the converged mu (device events around every product launch)."""
    import torch
    from synth import make_config
    s = make_config(5)
    lib = nolsm.Nolsm(precision=nolsm.PREC_MIXED_FP16, bounds=nolsm.BOUNDS_LEARNED)
    lib.set_predictor(predictor)
    d_dev = torch.empty(s.nnz, dtype=torch.float64, device="cuda")
    mu_fn = lambda lib_, s_: lib_.set_mu(s_.n_electrons, tol_n=TOL_N)   # noqa: E731
    solve(lib, s, mu_fn, d_dev, "device")
    torch.cuda.synchronize()
    lib.phase_times(reset=True)
    t0 = time.perf_counter()
    for _ in range(steps):
        mu, n, mu_steps, e = solve(lib, s, mu_fn, d_dev, "device")
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    stage_ms = {k: v / steps for k, v in lib.phase_times(reset=True).items()}
    lib.counters(reset=True)
    for _ in range(evals):
        st = lib.sign_batch(mu)
    cnt = lib.counters(reset=True)
    tf = cnt["gemm_flops"] / (cnt["gemm_ms"] * 1e-3) / 1e12
    n_b = np.array([nolsm.nolsm_block_info(lib.ctx, b)[0] for b in range(s.n_blocks)], np.float64)
    useful = float(np.sum((2.0 * lib.iters() + 1.0) * n_b * n_b * (n_b + 1.0)))
    tf_useful = tf * useful / st["flops_executed"]
    out = {"workload": "water-13824, 32-molecule clusters + 8 A halo", "blocks": s.n_blocks, "atoms": s.n_atoms,
           "n_b": "1,860-1,872 (n_pad 1,920)", "value": s.n_atoms / dt, "unit": "atoms/s", "ms_per_step": dt * 1e3,
           "mu_steps": mu_steps, "stage_ms_per_step": stage_ms,
           "sign_gemm": {"tflops_executed": tf,
                         "tflops_paper_convention": tf * st["flops_paper"] / st["flops_executed"],
                         "pct_fp16_peak_measured": 100 * tf / pk["bf16_tflops_sustained"],
                         "tflops_useful": tf_useful,
                         "pct_fp16_peak_measured_useful": 100 * tf_useful / pk["bf16_tflops_sustained"],
                         "ms_per_sign_evaluation": cnt["gemm_ms"] / evals, "ns_iters_avg": st["iters_avg"],
                         "schedule": "per-product launches, tiles dealt round-robin"}}
    if checks is not None:
        checks["largest_blocks"] = (s, lib.density().cpu().numpy(), mu, 2)
    lib.close()
    return out


def million_molecules(nolsm, predictor, pk, checks=None, parity_blocks=256, sample_blocks=1024):
    """The 1,000,000-molecule configuration at full size: 6,000,000 basis functions, 31,250 blocks of
    32-molecule clusters with an 8 A halo (n_b ~ 1,870), generated on the device (synth.device) and
    solved by nolsm_solve_chunked with the learned bounds: the CSR of H0, S and D resident, the blocks
    streamed through the pools in chunks sized to the free memory, mu to 1e-3 relative, the band
    energy from the assembled D.  One warm-up solve of the first 2,000 blocks sizes the pools; the
    full solve is timed once (CUDA events inside the call and the host clock around it).  Beside
    it: the plain FP32 path and the mixed path on the first `sample_blocks` blocks, and the oracle on
    `parity_blocks` sampled blocks at the returned mu."""
    import torch
    from synth.device import DeviceSystem, water_clusters_device
    t0 = time.perf_counter()
    ds = water_clusters_device(100, seed=31)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    torch.cuda.empty_cache()

    def head(k):
        return DeviceSystem(ds.name, ds.box, ds.n_mol, ds.row_ptr, ds.col, ds.h, ds.s, ds.blk_ptr[:k + 1],
                            ds.blk_cols, ds.extra_ptr[:k + 1], ds.extra_idx, ds.n_electrons * k / ds.n_blocks)

    d = torch.zeros(ds.nnz, dtype=torch.float64, device="cuda")
    lib = nolsm.Nolsm(precision=nolsm.PREC_MIXED_FP16, bounds=nolsm.BOUNDS_LEARNED)
    lib.set_predictor(predictor)
    lib.solve_chunked(head(2000), d, tol_n=1e-3, max_passes=1)
    lib.counters(reset=True)
    lib.phase_times(reset=True)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        t1 = time.perf_counter()
        st = lib.solve_chunked(ds, d, tol_n=1e-3, block_traces=True)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t1
    cnt = lib.counters(reset=True)
    stage = {k: round(v, 1) for k, v in lib.phase_times(reset=True).items()}
    lib.close()
    t_solve = max(wall, st["ms_total"] * 1e-3)
    ex = cnt["gemm_flops"] / (cnt["gemm_ms"] * 1e-3) / 1e12 if cnt["gemm_ms"] > 0 else None
    useful = ex * st["flops_useful"] / st["flops_executed"] if ex else None
    out = {"workload": "water-1000000: 32-molecule clusters + 8 A halo, 6,000,000 basis functions, 31,250 blocks",
           "atoms": ds.n_atoms, "basis": ds.n_basis, "nnz": ds.nnz, "blocks": ds.n_blocks,
           "generation_s_not_timed": round(gen_s, 1),
           "value": ds.n_atoms / t_solve, "unit": "atoms/s", "seconds_per_solve": t_solve,
           "device_ms": st["ms_total"], "passes": st["passes"], "chunks": st["chunks"],
           "max_chunk_blocks": st["max_chunk_blocks"], "ms_per_mu_iteration": st["ms_last_pass"],
           "mu": st["mu"], "n_electrons": st["n_electrons"], "n_target": ds.n_electrons,
           "count_error_rel": abs(st["n_electrons"] - ds.n_electrons) / ds.n_electrons,
           "band_energy": st["band_energy"], "band_energy_from_traces": st["band_energy_traces"],
           "ns_iters_avg": st["iters_avg"], "stage_ms": stage, "clocks": clk.summary(),
           "sign_gemm": {"tflops_executed": ex, "tflops_useful": useful,
                         "tflops_paper_convention": ex * st["flops_paper"] / st["flops_executed"] if ex else None,
                         "pct_fp16_peak_measured_useful": 100 * useful / pk["bf16_tflops_sustained"] if ex else None,
                         "pct_fp16_peak_measured_executed": 100 * ex / pk["bf16_tflops_sustained"] if ex else None,
                         "pct_fp16_peak_measured_burst_useful": 100 * useful / pk["bf16_tflops"] if ex else None,
                         "gemm_ms": cnt["gemm_ms"], "gemm_launches": cnt["gemm_launches"],
                         "useful_flops": "n_b^2 (n_b + 1) per symmetric product at the true n_b"}}
    if checks is not None and parity_blocks:
        # sampled blocks at the returned mu: their restricted systems and the D this solve left
        # behind at their own-column entries (the oracle runs in the parity leg)
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from oracle_pool import own_positions, restrict_groups, trace_bounds_device
        sample = np.sort(np.random.default_rng(31).choice(ds.n_blocks, parity_blocks, replace=False))
        groups = restrict_groups(ds, sample)
        dd = d[torch.from_numpy(own_positions(groups)).cuda()].cpu().numpy()
        bn, be = trace_bounds_device(ds, sample, 1e-3)
        checks["million_molecules"] = ("restricted", groups, dd, st["mu"], st["block_n"][sample],
                                       st["block_e"][sample], bn, be)
    # the plain FP32 path against the mixed path on the same bounded sample of blocks
    sub = head(sample_blocks)
    cmp = {}
    for name, kw in (("mixed_fp16_learned", dict(precision=nolsm.PREC_MIXED_FP16, bounds=nolsm.BOUNDS_LEARNED)),
                     ("fp32_plain", dict(precision=nolsm.PREC_FP32, scaled=0))):
        lb = nolsm.Nolsm(**kw)
        if kw.get("bounds") == nolsm.BOUNDS_LEARNED:
            lb.set_predictor(predictor)
        lb.solve_chunked(head(64), d, tol_n=1e-3, max_passes=1)   # warm-up
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        s2 = lb.solve_chunked(sub, d, tol_n=1e-3, max_passes=1)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t2
        atoms = 3 * 32 * sample_blocks
        cmp[name] = {"value": atoms / dt, "unit": "atoms/s", "seconds": dt, "ns_iters_avg": s2["iters_avg"],
                     "mu": s2["mu"]}
        lb.close()
    cmp["sample"] = f"the first {sample_blocks} of {ds.n_blocks} blocks (one pass each, mu from the first chunk)"
    cmp["speedup_mixed_over_fp32"] = cmp["mixed_fp16_learned"]["value"] / cmp["fp32_plain"]["value"]
    out["fp32_plain_comparison"] = cmp
    del d, ds
    torch.cuda.empty_cache()
    return out


def combination(nolsm, predictor, system, checks=None, steps=2, evals=3, tag="combination", combine=True,
                bounds="learned"):
    """Submatrix combination (Section III-B-1, Table II) on the benchmark system: no combination,
    Eq. 9 and Eq. 10 with the committed p(n) table.  Per criterion: the planning time on the host,
    the submatrix statistics of Table II (count, smallest, largest, average dimension, flops of one
    product of every submatrix, estimated TFLOP/s and speedup from p(n)), and the same full step
    measured on the GPU with the combined blocks (1 warm-up, `steps` timed) with the products'
    device time over `evals` sign evaluations at the converged mu."""
    import torch
    def table(path):
        try:
            return nolsm.load_pn_table(path)
        except OSError:
            return None
    pn, pn_step = table(nolsm.PN_TABLE), table(nolsm.PN_STEP_TABLE)
    crits = [("none", None, None)]
    if combine:
        crits.append(("eq9_cubic", nolsm.COMBINE_CUBIC, None))
        if pn is not None:
            crits.append(("eq10_performance", nolsm.COMBINE_PERFORMANCE, pn))
        if pn_step is not None:       # Eq. 10's rule with the whole step's measured time per flop
            crits.append(("eq10_full_step_time", nolsm.COMBINE_PERFORMANCE, pn_step))
    d_dev = torch.empty(system.nnz, dtype=torch.float64, device="cuda")
    mu_fn = lambda lib_, s_: lib_.set_mu(s_.n_electrons, tol_n=TOL_N)   # noqa: E731

    def t_est(dims):
        """Predicted products time of one multiplication of every submatrix: sum 2 n^3 p(n) (s)."""
        d = dims.astype(np.float64)
        return float((2 * d ** 3 * np.interp(d, pn[0], pn[1])).sum()) if pn is not None else None

    out = {"p_table": None if pn is None else {"n": [int(pn[0][0]), int(pn[0][-1])], "points": len(pn[0]),
                                               "source": "paper_2205_12182_gb300/weights/pn_gb300.json",
                                               "estimates": "Table II columns use this table for every row"}}
    base_est = None
    for name, crit, tab in crits:
        t0 = time.perf_counter()
        s, r = (system, None) if crit is None else nolsm.combine_blocks(system, crit, tab)
        plan_s = time.perf_counter() - t0
        if bounds == "learned":
            lib = nolsm.Nolsm(precision=nolsm.PREC_MIXED_FP16, bounds=nolsm.BOUNDS_LEARNED)
            lib.set_predictor(predictor)
        else:   # Gershgorin scale with a fixed lower bound on |eig(X_0)|
            lib = nolsm.Nolsm(precision=nolsm.PREC_MIXED_FP16, lower_bound=float(bounds))
        solve(lib, s, mu_fn, d_dev, "device")
        torch.cuda.synchronize()
        lib.phase_times(reset=True)
        dims = np.array([nolsm.nolsm_block_info(lib.ctx, b)[0] for b in range(s.n_blocks)], np.int64)
        if r is not None:
            assert np.array_equal(dims, r["dim"]), "combined dimensions disagree with the built index sets"
        flops = float((2 * dims.astype(np.float64) ** 3).sum())
        est = t_est(dims)
        if base_est is None:
            base_est = est
        t1 = time.perf_counter()
        for _ in range(steps):
            mu, n, mu_steps, e = solve(lib, s, mu_fn, d_dev, "device")
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t1) / steps
        stage = {k: round(v / steps, 3) for k, v in lib.phase_times(reset=True).items()}
        fp = 0.0
        for _ in range(evals):
            st = lib.sign_batch(mu)
            fp += st["flops_paper"]
        prod_ms = lib.phase_times(reset=True)["products"] / evals
        row = {"submatrices": int(len(dims)), "smallest": int(dims.min()), "largest": int(dims.max()),
               "average_dim": float(dims.mean()), "gflop_per_multiplication": flops / 1e9,
               "histogram_128": {int(k * 128): int(c) for k, c in enumerate(np.bincount(dims // 128)) if c},
               "estimated_tflops": flops / est / 1e12 if est else None,
               "estimated_speedup": base_est / est if est else None,
               "plan_seconds": plan_s,
               "measured": {"value": system.n_atoms / dt, "unit": "atoms/s", "ms_per_step": dt * 1e3,
                            "mu_steps": mu_steps, "ns_iters_avg": st["iters_avg"],
                            "products_ms_per_sign_evaluation": prod_ms,
                            "products_ms_per_average_iteration": prod_ms / st["iters_avg"],
                            "stage_ms_per_step": stage,
                            "products_tflops_paper_convention": fp / evals / (prod_ms * 1e-3) / 1e12}}
        if checks is not None:
            checks[tag + "." + name] = (s, lib.density().cpu().numpy(), mu, 2)
        out[name] = row
        lib.close()
    base = out["none"]["measured"]
    for name, _, _ in crits[1:]:
        m = out[name]["measured"]
        m["speedup_full_step"] = base["ms_per_step"] / m["ms_per_step"]
        m["speedup_products"] = base["products_ms_per_sign_evaluation"] / m["products_ms_per_sign_evaluation"]
    return out


def globule_schedules(nolsm, g, evals=3):
    """The ragged globule's products (n_b 163-2,678) under each product schedule: the built-in AUTO
    rule, AUTO with the autotuner's measured table and times (the predicted fastest of the single
    schedules and the split), the table's per-bin choice alone (a split evaluation: the bins that
    prefer the persistent kernel in one persistent launch, the rest in per-product launches), and
    every single schedule.  Products ms per sign evaluation (stage timer) at the converged mu,
    Gershgorin bounds with lower bound 0.02."""
    import torch
    try:
        table = nolsm.load_schedule_table()
    except OSError:
        table = None
    cases = [("auto_builtin", nolsm.SCHEDULE_AUTO, None), ("persistent", nolsm.SCHEDULE_PERSISTENT, None),
             ("per_product", nolsm.SCHEDULE_PER_PRODUCT, None),
             ("interleaved", nolsm.SCHEDULE_PERSISTENT_INTERLEAVED, None)]
    if table is not None:
        cases.insert(1, ("auto_measured_table", nolsm.SCHEDULE_AUTO, table))
        # the table's per-bin choice without its times: always the split evaluation
        cases.insert(2, ("split_by_table_bins", nolsm.SCHEDULE_AUTO, table[:2]))
    out = {"workload": f"protein-like globule, {g.n_atoms} atoms, {g.n_blocks} blocks", "evaluations": evals,
           "table": None if table is None else "paper_2205_12182_gb300/weights/schedule_gb300.json"}
    mu = None
    for name, sched, tab in cases:
        lib = nolsm.Nolsm(precision=nolsm.PREC_MIXED_FP16, lower_bound=0.02, schedule=sched)
        if tab is not None:
            lib.set_schedule_table(tab)
        lib.build(g)
        if mu is None:
            mu = lib.set_mu(g.n_electrons, tol_n=TOL_N)[0]
        lib.sign_batch(mu)
        torch.cuda.synchronize()
        lib.phase_times(reset=True)
        for _ in range(evals):
            st = lib.sign_batch(mu)
        ms = lib.phase_times(reset=True)["products"] / evals
        sc, nq = lib.last_schedule()
        out[name] = {"products_ms_per_sign_evaluation": ms, "ns_iters_avg": st["iters_avg"],
                     "schedule_run": {-2: "split"}.get(sc, ["persistent", "per_product", "auto", "interleaved"][sc]),
                     "persistent_blocks": nq,
                     "products_tflops_paper_convention": st["flops_paper"] / (ms * 1e-3) / 1e12}
        lib.close()
    return out


def md_steps(nolsm, predictor, system, checks=None, steps=4, keep_steps=16):
    """MD-like steps on the benchmark system: two geometries (the second with every atom moved by
    N(0, 0.02^2) A per axis) alternate, so each step's kept bounds come from the other geometry.
    A timed step: build, mu search, density and band energy, and for the kept-bounds run also the
    Lanczos runs that keep the bounds for the next step (nolsm_keep_bounds, `keep_steps` steps).  Bounds:
    learned (the headline's) against kept from the previous geometry with the mu search bracketed
    by +-0.02 Ha around the previous mu."""
    import torch
    from synth import displaced
    geo = [system, displaced(system, 0.02, seed=1234)]
    d_dev = torch.empty(max(g.nnz for g in geo), dtype=torch.float64, device="cuda")
    out = {"workload": "water-4096 and a displaced copy (0.02 A per axis), alternating", "steps": steps,
           "lanczos_steps_kept": keep_steps}
    for name in ("learned", "kept"):
        if name == "learned":
            lib = nolsm.Nolsm(precision=nolsm.PREC_MIXED_FP16, bounds=nolsm.BOUNDS_LEARNED)
            lib.set_predictor(predictor)
        else:
            lib = nolsm.Nolsm(precision=nolsm.PREC_MIXED_FP16, bounds=nolsm.BOUNDS_GIVEN)
        mu_prev = None

        def one(k):
            nonlocal mu_prev
            g = geo[k % 2]
            lib.build(g)
            if name == "kept" and mu_prev is not None:
                mu, n, ms = lib.set_mu(g.n_electrons, mu_lo=mu_prev - 0.02, mu_hi=mu_prev + 0.02, tol_n=TOL_N)
            else:
                mu, n, ms = lib.set_mu(g.n_electrons, tol_n=TOL_N)
            lib.density(d_dev[:g.nnz])
            lib.band_energy()
            if name == "kept":
                lib.keep_bounds(keep_steps)
            mu_prev = mu
            return mu, ms

        one(0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mus = []
        for k in range(1, steps + 1):
            mu, ms = one(k)
            mus.append(ms)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / steps
        st = lib.sign_batch(mu)
        out[name] = {"value": system.n_atoms / dt, "unit": "atoms/s", "ms_per_step": dt * 1e3,
                     "mu_steps": mus, "ns_iters_avg_last_geometry": st["iters_avg"],
                     "restarted": st["n_restarted"]}
        if checks is not None and name == "kept":
            g = geo[steps % 2]
            checks["md_steps." + name] = (g, lib.density().cpu().numpy(), mu, 2)
        lib.close()
    return out


_CLOCK_MAX = {"mhz": None}


def clk_max_mhz():
    return _CLOCK_MAX["mhz"]


def source_hash(relpath, begin, function):
    """sha256 (16 hex digits) of a source region: from the first line containing `begin` to the closing
    brace (a lone '}' line) of the __global__ function `function`."""
    import hashlib
    lines = open(os.path.join(ROOT, relpath)).read().split("\n")
    i0 = next(i for i, ln in enumerate(lines) if begin in ln)
    i1 = next(i for i, ln in enumerate(lines) if "__global__" in ln and function + "(" in ln)
    i2 = next(i for i in range(i1, len(lines)) if lines[i] == "}")
    return hashlib.sha256("\n".join(lines[i0:i2 + 1]).encode()).hexdigest()[:16]


def traffic_per_launch(kernel, units):
    """DRAM bytes of one launch from the committed ncu summary profiles/<kernel>_traffic.json
    (bytes per unit x units of this launch), or None when the kernel's source changed since."""
    p = os.path.join(ROOT, "profiles", kernel + "_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        src = d["source"]
        if source_hash(src["file"], src["begin"], src["function"]) != d["source_sha256_16"]:
            return None
        return d["dram_bytes_per_unit"] * units
    except (ValueError, OSError, KeyError, StopIteration):
        return None


OZ_SLICES = 6                                   # 8-bit slices per double-float value (csrc/internal.h)
TRSM_OPS_PER_ENTRY = 2 * (10 * OZ_SLICES + 6) + 8 * OZ_SLICES


def oz_update_tiles(n_b, panel=64, tm=128, tn=32):
    """128 x 32 tiles of the tensor-core trailing updates of the blocked double-float Cholesky (the
    library's work items: per panel, 32-column chunks of the trailing columns, and their 128-row
    tiles that reach the diagonal)."""
    tiles = 0
    for n in n_b.astype(int):
        for t0 in range(panel, n, panel):
            for n0 in range(t0, n, tn):
                d = n0 - t0 - (tm - 1)
                m_first = t0 + (max(d, 0) + tm - 1) // tm * tm
                tiles += len(range(m_first, n, tm))
    return tiles


def rooflines(stage_ms, cnt, steps, n_b, pk, sm_max_mhz, props, products_per_launch, useful_ratio=1.0):
    """The kernels that dominate a step, each against its own bound, from the stage times measured in
    the timed region (CUDA events on the library's stream around each stage's launches).
    * ns_pair_kernel (stage 'products'): tensor cores, useful FP16 FLOP (n_b^2 (n_b + 1) per symmetric
      product at the true n_b) over its time; the executed fraction (padded n_pad, whole diagonal
      tiles) beside it;
    * chol_update_kernel ('factor_update'): tensor cores, the executed BF16 FLOP of the slice-pair
      products (OZ_SLICES (OZ_SLICES + 1) / 2 = 21 pairs x 2 x 128 x 32 x 64 per tile);
    * chol_trsm_tc_kernel ('factor_trsm'): the FP32 pipe, which splits every entry of A21 into six
      slices, adds the six level sums of the result in double-float and splits the result again
      (66 + 48 + 66 = 180 FP32 operations per entry of L21: 10 per slice and 6 more per splitting,
      8 per level; 64 entries per trailing row per panel; the slice products themselves are a small
      tensor-core load); peak: 128 FP32 operations per SM and clock;
    * the triangular inverse ('inverse', mixed paths: 128 x 128 diagonal blocks from the factor's
      64 x 64 inverses on the FP32 pipe, the off-diagonal blocks as three-pass TF32 tensor-core
      products): n_b^3 / 3 FP32-accurate flops per
      block against the three-pass TF32 rate (TF32 at half the BF16 dense rate, three passes)."""
    mhz = sm_max_mhz or 2070.0
    sms = props.multi_processor_count
    alu_peak = sms * 128 * mhz * 1e6 / 1e12   # FP32 operations (not FMA-doubled)
    tf32x3_peak = pk["bf16_tflops_sustained"] / 2.0 / 3.0
    out = []
    prod_ms = stage_ms.get("products", 0.0)
    if prod_ms > 0 and cnt["gemm_flops"] > 0:
        exe = cnt["gemm_flops"] / steps / (prod_ms * 1e-3) / 1e12
        ach = exe * useful_ratio
        out.append({"kernel": "ns_pair_kernel (tcgen05 FP16 Newton-Schulz products, whole iteration per launch)",
                    "bound": "tensor", "achieved": ach, "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                    "frac": ach / pk["bf16_tflops_sustained"],
                    "flops": "useful: n_b^2 (n_b + 1) per symmetric product at the true n_b",
                    "achieved_executed": exe, "frac_executed": exe / pk["bf16_tflops_sustained"],
                    "peak_source": pk["source"] + " bf16 sustained (FP16 dense rate = BF16 dense rate)",
                    "ms_per_step": prod_ms,
                    "traffic": traffic_per_launch("ns_pair_kernel", products_per_launch)})
    upd_ms = stage_ms.get("factor_update", 0.0)
    if upd_ms > 0:
        tiles = oz_update_tiles(n_b)
        flop = tiles * (OZ_SLICES * (OZ_SLICES + 1) // 2) * 2.0 * 128 * 32 * 64
        ach = flop / (upd_ms * 1e-3) / 1e12
        out.append({"kernel": "chol_update_kernel (Cholesky trailing updates from exact BF16 slices, tcgen05; "
                              "7 launches per step, traffic summed)",
                    "bound": "tensor", "achieved": ach, "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                    "frac": ach / pk["bf16_tflops_sustained"],
                    "peak_source": pk["source"] + " bf16 sustained", "ms_per_step": upd_ms,
                    "traffic": traffic_per_launch("chol_update_kernel", tiles)})
    trsm_ms = stage_ms.get("factor_trsm", 0.0)
    if trsm_ms > 0:
        rows = sum(max(int(n) - t0, 0) for n in n_b for t0 in range(64, int(n), 64))
        ops = rows * 64 * float(TRSM_OPS_PER_ENTRY)
        ach = ops / (trsm_ms * 1e-3) / 1e12
        out.append({"kernel": "chol_trsm_tc_kernel (rows below each 64 x 64 diagonal block: exact slices, "
                              "tcgen05 slice products, double-float recombination)",
                    "bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "T FP32 operations/s",
                    "frac": ach / alu_peak,
                    "work": f"{TRSM_OPS_PER_ENTRY} FP32 operations per entry of L21 (slicing A21, adding the "
                            f"{OZ_SLICES} levels, slicing L21)",
                    "peak_source": f"derived: {sms} SMs x 128 FP32 operations/clk x {mhz:.0f} MHz",
                    "ms_per_step": trsm_ms, "traffic": traffic_per_launch("chol_trsm_tc_kernel", rows)})
    inv_ms = stage_ms.get("inverse", 0.0)
    if inv_ms > 0:
        flop = float(np.sum(n_b ** 3) / 3.0)
        ach = flop / (inv_ms * 1e-3) / 1e12
        out.append({"kernel": "L^-1 (trinv128_kernel on the 128 x 128 diagonal blocks from the factor's 64 x 64 "
                              "inverses, cong_tc_kernel three-pass TF32 products off the diagonal)",
                    "bound": "tensor", "achieved": ach, "peak": tf32x3_peak, "unit": "TFLOP/s (FP32-accurate)",
                    "frac": ach / tf32x3_peak,
                    "peak_source": pk["source"] + " bf16 sustained / 2 (TF32 dense rate) / 3 (three passes)",
                    "ms_per_step": inv_ms, "traffic": None})
    return out


def parity_sample(system, d, mu, n_blocks=8):
    from oracle.nolsm import NolsmOracle
    rng = np.random.default_rng(1)
    sample = rng.choice(system.n_blocks, n_blocks, replace=False)
    o = NolsmOracle.from_system(system, blocks=sample).prepare()
    ref = o.density(mu)
    own = np.isin(system.col, np.concatenate([system.block_cols(int(b)) for b in sample]))
    return {"blocks": int(n_blocks), "max_abs_dD": float(np.abs(d[own] - ref[own]).max())}


def parity_restricted(groups, dd, mu, block_n, block_e, bn, be):
    """The oracle on restricted groups of sampled blocks of a device-resident system."""
    from oracle_pool import oracle_restricted
    t0 = time.perf_counter()
    o_n, o_e, pos, o_d = oracle_restricted(groups, mu)
    return {"blocks": int(len(block_n)), "max_abs_dD": float(np.abs(dd - o_d).max()),
            "max_block_n_err_over_bound": float(np.max(np.abs(block_n - o_n) / bn)),
            "max_block_e_err_over_bound": float(np.max(np.abs(block_e - o_e) / be)),
            "sampled_count_rel_err": float(abs(block_n.sum() - o_n.sum()) / o_n.sum()),
            "oracle_seconds": round(time.perf_counter() - t0, 1)}


def parity_checks(checks):
    """The oracle on sampled blocks of every recorded run (system, D, mu, blocks), at the run's mu."""
    return {key: parity_restricted(*args[1:]) if args[0] == "restricted" else parity_sample(*args)
            for key, args in checks.items()}


# ------------------------------------------------------------------------------------ oracle

def oracle_sample_time(system, n_sample, seed=0):
    """Time the FP64 oracle on n_sample blocks: per-block spectra, 20 electron counts, density."""
    from oracle.nolsm import NolsmOracle
    rng = np.random.default_rng(seed)
    sample = np.sort(rng.choice(system.n_blocks, n_sample, replace=False))
    t0 = time.perf_counter()
    o = NolsmOracle.from_system(system, blocks=sample).prepare()
    for mu in np.linspace(-0.6, -0.4, 20):
        o.electron_count(mu)
    o.density(-0.45)
    return time.perf_counter() - t0, sample


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def cpu_baseline(system, seconds=15.0):
    t_small, _ = oracle_sample_time(system, 4)
    per_block = max(t_small / 4, 1e-4)
    n_sample = int(min(system.n_blocks, max(8, seconds / per_block)))
    t, _ = oracle_sample_time(system, n_sample, seed=1)
    t_full = t * system.n_blocks / n_sample
    return {"value": WORKLOAD["atoms"] / t_full, "unit": "atoms/s", "cores": cores(), "kind": "oracle",
            "sample": f"{n_sample} of {system.n_blocks} blocks (numpy/LAPACK FP64 eigh route), {t:.1f} s, "
                      f"extrapolated linearly to all blocks"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from synth import make_config
    system = make_config(2, seed=WORKLOAD["seed"])
    # each step: a bounded sample of the workload timed on the host cores, scaled to atoms/s
    times = []
    n_sample = 16
    for _ in range(args.warmup):
        oracle_sample_time(system, 2)
    for k in range(args.steps):
        t, _ = oracle_sample_time(system, n_sample, seed=100 + k)
        times.append(t * system.n_blocks / n_sample)
    t_step = float(np.mean(times))
    value = WORKLOAD["atoms"] / t_step
    line = {"metric": METRIC, "value": value, "unit": "atoms/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded water boxes; no dataset)",
            "config": dict(WORKLOAD), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "atoms/s", "cores": cores(), "kind": "oracle",
                             "sample": f"{n_sample} of {system.n_blocks} blocks per step, extrapolated"},
            "e2e": {"value": value, "unit": "atoms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the large-block (32-molecule cluster) section")
    ap.add_argument("--no-combination", action="store_true", help="skip the submatrix-combination section")
    ap.add_argument("--no-globule", action="store_true", help="skip the protein-like globule section")
    ap.add_argument("--no-md", action="store_true", help="skip the MD-like steps with kept bounds")
    ap.add_argument("--no-million", action="store_true",
                    help="skip the 1,000,000-molecule configuration (chunked solve)")
    ap.add_argument("--keep-steps", type=int, default=16, help="Lanczos steps of the kept bounds (MD-like steps)")
    ap.add_argument("--partition", choices=["boxes", "lpt"], default="boxes",
                    help="N > 1: one seeded box per rank (weak scaling) or one box with its blocks dealt to the "
                         "ranks by LPT on the predicted cost (strong scaling)")
    ap.add_argument("--side", type=int, default=16,
                    help="molecules per box edge (16: the 4,096-molecule workload; smaller boxes for profiling)")
    args = ap.parse_args()
    if args.impl == "ours":
        from paper_2205_12182_gb300.build import build
        build()      # idempotent: compiles libnolsm.so only when it is missing or stale
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
