"""Chemical-potential bisection shared by several ranks (one GPU each).

The blocks are independent (the solution phase needs no communication, Section I), so ranks
own disjoint sets of blocks; the only exchange is the electron count.  Every bisection step
each rank evaluates its blocks at the common mu (nolsm_sign_batch) and the partial counts are
summed over ranks (one float64 all-reduce) before the bracket update, so all ranks take the
same decisions and end at the same mu.  The stopping rule is that of nolsm_set_mu.
"""
from __future__ import annotations


def allreduce_sum(values, group=None):
    """Sum a small list of floats over ranks (torch.distributed, any backend)."""
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    t = torch.tensor(list(values), dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return [float(x) for x in t.cpu()]


def allreduce_minmax(lo, hi, group=None):
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    a = torch.tensor([lo], dtype=torch.float64, device=dev)
    b = torch.tensor([hi], dtype=torch.float64, device=dev)
    dist.all_reduce(a, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(b, op=dist.ReduceOp.MAX, group=group)
    return float(a.item()), float(b.item())


def bisect_shared(evaluate, reduce, n_electrons, lo, hi, tol_n=1e-3, max_steps=60):
    """Bisection on the global count: evaluate(mu) -> local count, reduce([x]) -> [sum over ranks]."""
    lo0, hi0 = lo, hi
    mu = 0.5 * (lo + hi)
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


def set_mu_distributed(lib, n_electrons_global, tol_n=1e-3, max_steps=60, group=None):
    """nolsm_set_mu over all ranks of `group`; lib is this rank's built Nolsm context."""
    lo_b, hi_b = lib.bounds()
    lo, hi = allreduce_minmax(float(lo_b.min()), float(hi_b.max()), group)
    return bisect_shared(lambda mu: lib.sign_batch(mu)["n_electrons"], lambda v: allreduce_sum(v, group),
                         n_electrons_global, lo, hi, tol_n, max_steps)
