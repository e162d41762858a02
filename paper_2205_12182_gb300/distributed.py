"""Chemical-potential bisection shared by several ranks (one GPU each).

The blocks are independent (the solution phase needs no communication, Section I), so ranks
own disjoint sets of blocks; the only exchange is the electron count.  Every bisection step
each rank evaluates its blocks at the common mu (nolsm_sign_batch) and the partial counts are
summed over ranks (one float64 all-reduce) before the bracket update, so all ranks take the
same decisions and end at the same mu.  The first point and the stopping rule are those of
nolsm_set_mu: the Aufbau estimate from the own-column diagonal of A0 over all ranks (gathered
once per build), then bisection.
"""
from __future__ import annotations

import math

import numpy as np


def _device(group):
    import torch
    import torch.distributed as dist
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")


def allreduce_sum(values, group=None):
    """Sum a small list of floats over ranks (torch.distributed, any backend)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64, device=_device(group))
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return [float(x) for x in t.cpu()]


def allreduce_minmax(lo, hi, group=None):
    import torch
    import torch.distributed as dist
    dev = _device(group)
    a = torch.tensor([lo], dtype=torch.float64, device=dev)
    b = torch.tensor([hi], dtype=torch.float64, device=dev)
    dist.all_reduce(a, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(b, op=dist.ReduceOp.MAX, group=group)
    return float(a.item()), float(b.item())


def allgather_floats(values, group=None) -> np.ndarray:
    """Concatenation over ranks (rank order) of every rank's float32 array (sizes may differ)."""
    import torch
    import torch.distributed as dist
    dev = _device(group)
    world = dist.get_world_size(group)
    local = torch.as_tensor(np.ascontiguousarray(values, np.float32), device=dev)
    n = torch.tensor([local.numel()], dtype=torch.int64, device=dev)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(x.item()) for x in sizes]
    m = max(sizes)
    padded = torch.zeros(m, dtype=torch.float32, device=dev)
    padded[:local.numel()] = local
    parts = [torch.empty(m, dtype=torch.float32, device=dev) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    return np.concatenate([p[:k].cpu().numpy() for p, k in zip(parts, sizes)])


def aufbau_point(own_diag, n_electrons, spin_factor=2.0):
    """nolsm_set_mu's first point: with k = floor(N_e / spin) occupied orbitals, the midpoint of
    the k-th and (k+1)-th smallest own-column diagonal entries of A0 (None when k is out of range).
    The entries are float32, and the midpoint is taken in float64 as the library does."""
    d = np.asarray(own_diag, np.float32)
    k = int(math.floor(n_electrons / spin_factor))
    if k < 1 or k >= d.size:
        return None
    part = np.partition(d, k)
    above = float(part[k])
    below = float(part[:k].max())
    return 0.5 * (below + above)


def bisect_shared(evaluate, reduce, n_electrons, lo, hi, tol_n=1e-3, max_steps=60, mu0=None):
    """Bisection on the global count: evaluate(mu) -> local count, reduce([x]) -> [sum over ranks].
    mu0, when inside (lo, hi), replaces the midpoint as the first point."""
    lo0, hi0 = lo, hi
    mu = mu0 if (mu0 is not None and lo < mu0 < hi) else 0.5 * (lo + hi)
    steps = 0
    while True:
        n_mu = reduce([evaluate(mu)])[0]
        steps += 1
        if abs(n_mu - n_electrons) <= tol_n * n_electrons:
            break
        if steps >= max_steps or hi - lo < 1e-10:
            break
        if n_mu < n_electrons:
            lo = mu
        else:
            hi = mu
        mu = 0.5 * (lo + hi)
    if abs(n_mu - n_electrons) > tol_n * n_electrons and (mu - lo0 < 1e-9 or hi0 - mu < 1e-9):
        raise RuntimeError("EBRACKET: N(mu) does not bracket the electron count")
    return mu, n_mu, steps


def set_mu_distributed(lib, n_electrons_global, tol_n=1e-3, max_steps=60, group=None, aufbau=True):
    """nolsm_set_mu over all ranks of `group`; lib is this rank's built Nolsm context.  The first
    point is the Aufbau estimate over every rank's own columns (aufbau=False: the midpoint)."""
    lo_b, hi_b = lib.bounds()
    lo, hi = allreduce_minmax(float(lo_b.min()), float(hi_b.max()), group)
    mu0 = None
    if aufbau:
        mu0 = aufbau_point(allgather_floats(lib.own_diagonal(), group), n_electrons_global,
                           lib.options.spin_factor)
    return bisect_shared(lambda mu: lib.sign_batch(mu)["n_electrons"], lambda v: allreduce_sum(v, group),
                         n_electrons_global, lo, hi, tol_n, max_steps, mu0=mu0)


def lpt_partition(costs, n_ranks):
    """Blocks to ranks by longest processing time first: blocks in decreasing cost (ties by index),
    each to the rank with the smallest load so far (ties to the lower rank).  Returns one ascending
    array of block indices per rank."""
    import heapq
    costs = np.asarray(costs, np.float64)
    order = sorted(range(len(costs)), key=lambda b: (-costs[b], b))
    heap = [(0.0, r) for r in range(n_ranks)]
    parts = [[] for _ in range(n_ranks)]
    for b in order:
        load, r = heapq.heappop(heap)
        parts[r].append(b)
        heapq.heappush(heap, (load + float(costs[b]), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def block_cost_estimate(system):
    """Predicted cost of every block for the partition: (own columns + extra indices)^3, an upper
    bound of n_b^3 that needs no index sets (the products cost 2 n_b^3 per product)."""
    bp = np.asarray(system.blk_ptr, np.int64)
    n = np.diff(bp).astype(np.float64)
    if system.extra_ptr is not None:
        n = n + np.diff(np.asarray(system.extra_ptr, np.int64))
    return n ** 3
