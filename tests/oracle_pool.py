"""Test helper: the FP64 oracle over many blocks in parallel (a spawn pool of single-threaded
workers), for parity checks of whole systems.

Per block b at one chemical potential mu it returns the block's terms of the electron count and the
band energy, n_b = spin * sum_{j in C_b} (S_b D_b)_jj and e_b = spin * sum_{j in C_b} (H_b D_b)_jj
(Eq. 4, Section V-A), and the values of D_b[:, C_b] at their positions in the stored pattern.  The
pool is started with `spawn` (never forked after the parent has touched the GPU).
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_SYSTEM = None


def _init(system, threads_env):
    global _SYSTEM
    os.environ.update(threads_env)
    _SYSTEM = system


def _work(args):
    blocks, mu = args
    from oracle.nolsm import NolsmOracle, theta
    o = NolsmOracle.from_system(_SYSTEM, blocks=blocks).prepare()
    sf = o.spin_factor
    n_b = np.array([sf * float(np.dot(w, theta(mu - e))) for w, e in zip(o.wn, o.eps)])
    e_b = np.array([sf * float(np.dot(w, theta(mu - e))) for w, e in zip(o.we, o.eps)])
    d = o.density(mu)
    own = np.concatenate([o.cols_of(int(b)) for b in blocks])
    pos = np.flatnonzero(np.isin(o.col, own))
    return blocks, n_b, e_b, pos, d[pos]


def workers() -> int:
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return max(1, min(n, 32))


def oracle_blocks(system, blocks, mu, n_workers=None, chunk=None):
    """(n_b, e_b per listed block, positions of their own-column entries, oracle D there)."""
    blocks = np.asarray(blocks, np.int64)
    nw = n_workers or workers()
    chunk = chunk or max(1, int(np.ceil(len(blocks) / (4 * nw))))
    tasks = [(blocks[i:i + chunk], float(mu)) for i in range(0, len(blocks), chunk)]
    env = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}
    saved = {k: os.environ.get(k) for k in env}
    os.environ.update(env)          # inherited by the spawned workers before they import numpy
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(nw, initializer=_init, initargs=(system, env)) as pool:
            res = pool.map(_work, tasks)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    index = {int(b): i for i, b in enumerate(blocks)}
    n_b = np.empty(len(blocks))
    e_b = np.empty(len(blocks))
    pos, val = [], []
    for bl, nb, eb, p, v in res:
        for k, b in enumerate(bl):
            n_b[index[int(b)]] = nb[k]
            e_b[index[int(b)]] = eb[k]
        pos.append(p)
        val.append(v)
    return n_b, e_b, np.concatenate(pos), np.concatenate(val)


def trace_bounds(system, blocks, d_tol, spin=2.0):
    """Bounds on |dn_b| and |de_b| implied by max|dD| <= d_tol on the own columns of each block:
    |sum_{j in C_b} sum_i S_ji dD_ij| <= d_tol * sum_{j in C_b} sum_i |S_ji| (the same with H0)."""
    col_abs_s = np.zeros(system.n_basis)
    col_abs_h = np.zeros(system.n_basis)
    np.add.at(col_abs_s, system.col, np.abs(system.s))
    np.add.at(col_abs_h, system.col, np.abs(system.h))
    bs = np.array([col_abs_s[system.block_cols(int(b))].sum() for b in blocks])
    bh = np.array([col_abs_h[system.block_cols(int(b))].sum() for b in blocks])
    return spin * d_tol * bs, spin * d_tol * bh
