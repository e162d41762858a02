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


class Restricted:
    """Host arrays of a system cut down to the rows and columns of a set U that holds every index
    set of the chosen blocks (their own columns, the pattern rows of those columns and their extra
    lists), renumbered in ascending order.  Every entry H_ij, S_ij with i, j in U is kept, so the
    chosen blocks' index sets, submatrices and columns of D are those of the full system.
    `full_pos[e]` is the position in the full CSR of entry e of the restricted one."""

    def __init__(self, row_ptr, col, h, s, blk_ptr, blk_cols, extra_ptr, extra_idx, n_electrons, full_pos, rows):
        self.row_ptr, self.col, self.h, self.s = row_ptr, col, h, s
        self.blk_ptr, self.blk_cols, self.extra_ptr, self.extra_idx = blk_ptr, blk_cols, extra_ptr, extra_idx
        self.n_electrons = n_electrons
        self.full_pos = full_pos
        self.rows = rows

    @property
    def n_basis(self):
        return len(self.row_ptr) - 1

    @property
    def nnz(self):
        return len(self.col)

    @property
    def n_blocks(self):
        return len(self.blk_ptr) - 1

    def block_cols(self, b):
        return self.blk_cols[self.blk_ptr[b]:self.blk_ptr[b + 1]]


def restrict_device_system(ds, blocks):
    """Restricted host copy (see `Restricted`) of a device-resident system for the given blocks."""
    import torch
    blocks = np.asarray(blocks, np.int64)
    dev = ds.row_ptr.device
    own = [np.asarray(ds.block_cols(int(b)), np.int64) for b in blocks]
    ext = [np.asarray(ds.block_extra(int(b)), np.int64) if ds.extra_ptr is not None else np.zeros(0, np.int64)
           for b in blocks]
    own_t = torch.from_numpy(np.concatenate(own)).to(dev)

    def rows_entries(r):
        """Positions of every stored entry of rows r (device int64)."""
        st = ds.row_ptr[r]
        ln = ds.row_ptr[r + 1] - st
        base = torch.repeat_interleave(st - torch.cumsum(ln, 0) + ln, ln)
        return base + torch.arange(int(ln.sum().item()), device=dev), torch.repeat_interleave(
            torch.arange(len(r), device=dev), ln)

    pos, _ = rows_entries(own_t)
    u = torch.unique(torch.cat([own_t, torch.from_numpy(np.concatenate(ext)).to(dev), ds.col[pos].long()]))
    new = torch.full((ds.n_basis,), -1, dtype=torch.int64, device=dev)
    new[u] = torch.arange(len(u), device=dev)
    pos, row_of = rows_entries(u)
    c = new[ds.col[pos].long()]
    keep = c >= 0
    pos, row_of, c = pos[keep], row_of[keep], c[keep]
    row_ptr = torch.zeros(len(u) + 1, dtype=torch.int64, device=dev)
    row_ptr[1:] = torch.cumsum(torch.bincount(row_of, minlength=len(u)), 0)
    bp = np.zeros(len(blocks) + 1, np.int32)
    bp[1:] = np.cumsum([len(x) for x in own])
    ep = np.zeros(len(blocks) + 1, np.int32)
    ep[1:] = np.cumsum([len(x) for x in ext])
    mp = new.cpu().numpy()
    return Restricted(row_ptr.cpu().numpy(), c.to(torch.int32).cpu().numpy(), ds.h[pos].cpu().numpy(),
                      ds.s[pos].cpu().numpy(), bp, mp[np.concatenate(own)].astype(np.int32), ep,
                      mp[np.concatenate(ext)].astype(np.int32), 0.0, pos.cpu().numpy(), u.cpu().numpy())


def _work_restricted(args):
    r, mu = args
    global _SYSTEM
    _SYSTEM = r
    blocks, n_b, e_b, pos, d = _work((np.arange(r.n_blocks), mu))
    return n_b, e_b, r.full_pos[pos], d


def restrict_groups(ds, blocks, group=4):
    """The blocks cut into groups of `group`, each as its restricted host system."""
    blocks = np.asarray(blocks, np.int64)
    return [restrict_device_system(ds, blocks[i:i + group]) for i in range(0, len(blocks), group)]


def own_positions(groups):
    """Full-CSR positions of the own-column entries of every group's blocks, in the order in which
    oracle_restricted returns its values."""
    return np.concatenate([r.full_pos[np.flatnonzero(np.isin(r.col, r.blk_cols))] for r in groups])


def oracle_restricted(groups, mu, n_workers=None):
    """oracle_blocks over restricted groups, one group per task: the per-block terms (in group
    order) and, for their own-column entries, the positions in the full CSR and the oracle's D."""
    tasks = [(r, float(mu)) for r in groups]
    nw = n_workers or workers()
    env = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}
    saved = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        with mp.get_context("spawn").Pool(nw, initializer=_init, initargs=(None, env)) as pool:
            res = pool.map(_work_restricted, tasks, chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return (np.concatenate([x[0] for x in res]), np.concatenate([x[1] for x in res]),
            np.concatenate([x[2] for x in res]), np.concatenate([x[3] for x in res]))


def oracle_device_blocks(ds, blocks, mu, group=4, n_workers=None):
    """oracle_blocks for a device-resident system (restricted groups of `group` blocks)."""
    return oracle_restricted(restrict_groups(ds, blocks, group), mu, n_workers)


def trace_bounds_device(ds, blocks, d_tol, spin=2.0):
    """trace_bounds for a device-resident system (column sums of |S| and |H0| on the device)."""
    import torch
    col = ds.col.long()
    cs = torch.zeros(ds.n_basis, dtype=torch.float64, device=col.device).index_add_(0, col, ds.s.abs())
    ch = torch.zeros(ds.n_basis, dtype=torch.float64, device=col.device).index_add_(0, col, ds.h.abs())
    cs, ch = cs.cpu().numpy(), ch.cpu().numpy()
    bs = np.array([cs[ds.block_cols(int(b))].sum() for b in blocks])
    bh = np.array([ch[ds.block_cols(int(b))].sum() for b in blocks])
    return spin * d_tol * bs, spin * d_tol * bh
