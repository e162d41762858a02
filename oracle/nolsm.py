"""Plain FP64 CPU oracle of the NOLSM density step.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this module.  The
library's product path never calls it, and it shares no code with the CUDA path.

What it computes (the paper's Section II, "Overview of the Problem"):

* Eq. 5: D = 1/2 (I - sign(S^-1 H0 - mu I)) S^-1, at zero electronic temperature.
* The submatrix method, three steps per column block (Section II, Fig. 1):
  (1) keep the rows/columns where an own column has a stored entry, on the
  combined pattern of H0 and S (the non-orthogonal variant); (2) evaluate the
  matrix function on the dense submatrices, Eq. 8; (3) write the own columns
  back into a matrix with the input's sparsity pattern.
* Eq. 4: E_elec = Tr(D H0).
* The chemical potential is the one that makes the system charge neutral
  (Section V-A, "Simulation Details"); this oracle finds it by bisection.

How it computes the sign: the matrix sign of S_b^-1 H_b - mu I is evaluated
exactly through symmetric eigendecompositions, never by an iteration.  With
S_b = V diag(s) V^T, S_b^-1/2 = V diag(s^-1/2) V^T and M = S_b^-1/2 H_b S_b^-1/2
= U diag(eps) U^T, one has S_b^-1 H_b = S_b^-1/2 M S_b^1/2, hence
sign(S_b^-1 H_b - mu) = S_b^-1/2 U sign(eps - mu) U^T S_b^1/2 and, with
Q = S_b^-1/2 U,  D_b = Q diag(theta(mu - eps)) Q^T  where theta = (1 - sign)/2
evaluated at eps - mu, i.e. 1 below mu, 0 above, 1/2 exactly at mu.

Readings where the paper is silent (stated here in full):
* closed shell: the electron count targets Tr(D S) = N_e / 2 per spin, and the
  reported band energy is spin_factor * Tr(D H0) with spin_factor = 2;
* index set: the pattern rule of step (1), optionally unioned with a given list
  of extra indices (the neighbourhood rule's geometric part);
* scatter: only entries (i, c) stored in the global pattern are kept, no
  symmetrisation;
* bisection: stop when |N(mu) - N_occ| <= tol_rel * N_occ, or the bracket is
  below 1e-10 Ha, or after 60 steps.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import jacobi


def theta(x: np.ndarray) -> np.ndarray:
    """Occupation (1 - sign(-x)) / 2 of an eigenvalue a distance x below mu: 1, 1/2 at 0, 0."""
    return np.where(x > 0, 1.0, np.where(x < 0, 0.0, 0.5))


def csr_matrix(row_ptr, col, val, n) -> sp.csr_matrix:
    return sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col), np.asarray(row_ptr)), shape=(n, n))


def index_set(pattern_csc: sp.csc_matrix, cols_b: np.ndarray, extra: np.ndarray | None = None) -> np.ndarray:
    """Step (1) of the submatrix method on the combined pattern (Section II; Eq. 8).

    The rows that hold a stored entry in any of the block's own columns, plus the
    optional extra indices; sorted ascending.
    """
    parts = [pattern_csc.indices[pattern_csc.indptr[c]:pattern_csc.indptr[c + 1]] for c in cols_b]
    parts.append(np.asarray(cols_b))
    if extra is not None:
        parts.append(np.asarray(extra))
    return np.unique(np.concatenate(parts).astype(np.int64))


def eigh(a: np.ndarray, backend: str = "lapack"):
    if backend == "lapack":
        return np.linalg.eigh(a)
    if backend == "jacobi":
        return jacobi.eigh(a)
    raise ValueError(backend)


def block_spectrum(hb: np.ndarray, sb: np.ndarray, backend: str = "lapack"):
    """(eps, Q) with S_b^-1 H_b = Q diag(eps) Q^-1 and Q^T S_b Q = I, via two eigh calls."""
    s, v = eigh(sb, backend)
    if s.min() <= 0.0:
        raise np.linalg.LinAlgError("overlap submatrix is not positive definite")
    sm12 = (v * s ** -0.5) @ v.T
    m = sm12 @ hb @ sm12
    m = 0.5 * (m + m.T)      # exact in exact arithmetic; removes rounding asymmetry only
    eps, u = eigh(m, backend)
    return eps, sm12 @ u


def sign_eq8(hb: np.ndarray, sb: np.ndarray, mu: float) -> np.ndarray:
    """sign(S_b^-1 H_b - mu I) by a general (non-symmetric) eigendecomposition (Eq. 8).

    A second, independent route to the same matrix, for small blocks.
    """
    a = np.linalg.solve(sb, hb)
    lam, vec = np.linalg.eig(a)
    lam = lam.real
    vec = vec.real
    return vec @ np.diag(np.sign(lam - mu)) @ np.linalg.inv(vec)


def density_eq8(hb: np.ndarray, sb: np.ndarray, mu: float) -> np.ndarray:
    """T(D) = 1/2 (I - sign(T(S)^-1 T(H0) - mu I)) T(S)^-1, written out (Eq. 5 / Eq. 8)."""
    n = hb.shape[0]
    return 0.5 * (np.eye(n) - sign_eq8(hb, sb, mu)) @ np.linalg.inv(sb)


def newton_schulz(a: np.ndarray, iters: int) -> np.ndarray:
    """Eq. 6 as written: X_0 = A, X_{k+1} = 1/2 X_k (3 I - X_k^2)."""
    x = np.array(a, dtype=np.float64)
    eye = np.eye(a.shape[0])
    for _ in range(iters):
        x = 0.5 * x @ (3.0 * eye - x @ x)
    return x


class NolsmOracle:
    """NOLSM density, electron count, chemical potential and band energy in FP64.

    Inputs are plain arrays: the CSR pattern (row_ptr, col) shared by H0 and S, their
    values, the column blocks (blk_ptr, blk_cols) and optional extra index lists.
    ``blocks`` restricts the work to a subset of blocks (a bounded sample): N(mu)
    and the energy are then partial sums over those blocks only.
    """

    def __init__(self, row_ptr, col, h, s, blk_ptr, blk_cols, n_electrons,
                 extra_ptr=None, extra_idx=None, spin_factor: float = 2.0,
                 blocks=None, backend: str = "lapack"):
        self.n = int(len(row_ptr) - 1)
        self.row_ptr = np.asarray(row_ptr, np.int64)
        self.col = np.asarray(col, np.int64)
        self.hval = np.asarray(h, np.float64)
        self.sval = np.asarray(s, np.float64)
        self.H = csr_matrix(self.row_ptr, self.col, self.hval, self.n)
        self.S = csr_matrix(self.row_ptr, self.col, self.sval, self.n)
        self.pattern = csr_matrix(self.row_ptr, self.col, np.ones(len(self.col)), self.n).tocsc()
        self.blk_ptr = np.asarray(blk_ptr, np.int64)
        self.blk_cols = np.asarray(blk_cols, np.int64)
        self.extra_ptr = None if extra_ptr is None else np.asarray(extra_ptr, np.int64)
        self.extra_idx = None if extra_idx is None else np.asarray(extra_idx, np.int64)
        self.n_electrons = float(n_electrons)
        self.spin_factor = float(spin_factor)
        self.n_occ = self.n_electrons / self.spin_factor
        nb = len(self.blk_ptr) - 1
        self.blocks = np.arange(nb) if blocks is None else np.asarray(blocks, np.int64)
        self.backend = backend
        self._prepared = False

    @classmethod
    def from_system(cls, system, **kw):
        return cls(system.row_ptr, system.col, system.h, system.s, system.blk_ptr, system.blk_cols,
                   system.n_electrons, system.extra_ptr, system.extra_idx, **kw)

    # -- step (1): index sets and dense submatrices
    def cols_of(self, b: int) -> np.ndarray:
        return self.blk_cols[self.blk_ptr[b]:self.blk_ptr[b + 1]]

    def extra_of(self, b: int):
        if self.extra_ptr is None:
            return None
        return self.extra_idx[self.extra_ptr[b]:self.extra_ptr[b + 1]]

    def index_set(self, b: int) -> np.ndarray:
        return index_set(self.pattern, self.cols_of(b), self.extra_of(b))

    def submatrices(self, b: int):
        idx = self.index_set(b)
        hb = self.H[idx][:, idx].toarray()
        sb = self.S[idx][:, idx].toarray()
        return idx, hb, sb

    # -- step (2): the spectral data each block's matrix function needs
    def prepare(self):
        """Per block: I_b, own positions, eigenpairs and the weights of N(mu) and Tr(DH)."""
        self.idx, self.own, self.eps, self.Q, self.wn, self.we = [], [], [], [], [], []
        for b in self.blocks:
            idx, hb, sb = self.submatrices(int(b))
            own = np.searchsorted(idx, self.cols_of(int(b)))
            eps, q = block_spectrum(hb, sb, self.backend)
            # (S_b D_b)_jj = sum_k (S_b Q)_jk theta_k Q_jk ; (H_b D_b)_jj likewise
            sq = sb @ q
            hq = hb @ q
            self.idx.append(idx)
            self.own.append(own)
            self.eps.append(eps)
            self.Q.append(q)
            self.wn.append(np.sum(sq[own] * q[own], axis=0))
            self.we.append(np.sum(hq[own] * q[own], axis=0))
        self._prepared = True
        return self

    def _need(self):
        if not self._prepared:
            self.prepare()

    def electron_count(self, mu: float) -> float:
        """N(mu) = sum_b sum_{j in C_b} (S_b D_b)_jj = Tr(D S) of the assembled D, per spin."""
        self._need()
        return float(sum(np.dot(w, theta(mu - e)) for w, e in zip(self.wn, self.eps)))

    def band_energy_of_mu(self, mu: float) -> float:
        """spin_factor * Tr(D H0) from the block spectra (equals band_energy(density(mu)))."""
        self._need()
        return self.spin_factor * float(sum(np.dot(w, theta(mu - e)) for w, e in zip(self.we, self.eps)))

    def block_density_cols(self, k: int, mu: float) -> np.ndarray:
        """D_b[:, C_b] (n_b x |C_b|) of the k-th prepared block at mu."""
        self._need()
        t = theta(mu - self.eps[k])
        q = self.Q[k]
        return (q * t) @ q[self.own[k]].T

    def spectral_bounds(self):
        self._need()
        return min(e[0] for e in self.eps), max(e[-1] for e in self.eps)

    def bisect(self, lo: float | None = None, hi: float | None = None, tol_rel: float = 1e-6,
               max_steps: int = 60, n_target: float | None = None):
        """mu with N(mu) = N_occ by bisection; returns (mu, N(mu), steps)."""
        self._need()
        target = self.n_occ if n_target is None else float(n_target)
        if lo is None or hi is None:
            emin, emax = self.spectral_bounds()
            lo, hi = emin - 1e-3, emax + 1e-3
        if not (self.electron_count(lo) <= target <= self.electron_count(hi)):
            raise ValueError("N(mu) does not bracket the electron count")
        mu = 0.5 * (lo + hi)
        n_mu = self.electron_count(mu)
        steps = 1
        while steps < max_steps and abs(n_mu - target) > tol_rel * target and hi - lo >= 1e-10:
            if n_mu < target:
                lo = mu
            else:
                hi = mu
            mu = 0.5 * (lo + hi)
            n_mu = self.electron_count(mu)
            steps += 1
        return mu, n_mu, steps

    # -- step (3): write own columns back into the global pattern
    def density(self, mu: float) -> np.ndarray:
        """Values of D on the stored pattern (nnz), own columns of each block only."""
        self._need()
        out = np.zeros(len(self.col))
        csc_pos = self._csc_positions()
        for k, b in enumerate(self.blocks):
            dcols = self.block_density_cols(k, mu)
            idx = self.idx[k]
            for jj, c in enumerate(self.cols_of(int(b))):
                rows, pos = csc_pos[c]
                p = np.searchsorted(idx, rows)
                out[pos] = dcols[p, jj]
        return out

    def _csc_positions(self):
        if not hasattr(self, "_cscpos"):
            order = np.lexsort((np.repeat(np.arange(self.n), np.diff(self.row_ptr)), self.col))
            rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))[order]
            cols = self.col[order]
            starts = np.searchsorted(cols, np.arange(self.n + 1))
            self._cscpos = {c: (rows[starts[c]:starts[c + 1]], order[starts[c]:starts[c + 1]])
                            for c in range(self.n)}
        return self._cscpos

    def band_energy(self, d_val: np.ndarray) -> float:
        """Eq. 4 with the spin factor: spin_factor * Tr(D H0) = spin_factor * sum_ij D_ij H0_ji."""
        d = csr_matrix(self.row_ptr, self.col, d_val, self.n)
        return self.spin_factor * float(d.multiply(self.H.T).sum())

    def trace_ds(self, d_val: np.ndarray) -> float:
        d = csr_matrix(self.row_ptr, self.col, d_val, self.n)
        return float(d.multiply(self.S.T).sum())


def full_density(h: np.ndarray, s: np.ndarray, n_occ: int) -> tuple[np.ndarray, float]:
    """Exact D of the whole system: the n_occ lowest generalized eigenvectors (mu in the gap)."""
    import scipy.linalg as sla
    eps, c = sla.eigh(h, s)
    d = c[:, :n_occ] @ c[:, :n_occ].T
    mu = 0.5 * (eps[n_occ - 1] + eps[n_occ])
    return d, mu
