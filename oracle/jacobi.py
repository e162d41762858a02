"""Cyclic Jacobi eigen-solver for small symmetric matrices (test infrastructure).

Textbook cyclic-by-row Jacobi (Golub & Van Loan, Matrix Computations, Section 8.5):
sweep over all off-diagonal pairs (p, q), zero each with a plane rotation chosen
from the symmetric 2x2 Schur decomposition, until the off-diagonal Frobenius norm
is below tol * ||A||_F.  It exists only to cross-check the oracle's one library
dependency (LAPACK eigh) on n <= 64.
"""
from __future__ import annotations

import numpy as np


def _sym_schur2(app: float, aqq: float, apq: float):
    """(c, s) such that the rotation zeroes the (p, q) entry."""
    if abs(apq) <= 1e-150 * (abs(app) + abs(aqq)) or apq == 0.0:
        return 1.0, 0.0     # already diagonal to working precision (also avoids overflow in tau)
    tau = (aqq - app) / (2.0 * apq)
    if tau >= 0:
        t = 1.0 / (tau + np.sqrt(1.0 + tau * tau))
    else:
        t = -1.0 / (-tau + np.sqrt(1.0 + tau * tau))
    c = 1.0 / np.sqrt(1.0 + t * t)
    return c, t * c


def eigh(a: np.ndarray, tol: float = 1e-15, max_sweeps: int = 100):
    """Eigenvalues ascending and orthonormal eigenvectors (columns), like numpy.linalg.eigh."""
    a = np.array(a, dtype=np.float64)
    n = a.shape[0]
    v = np.eye(n)
    norm = np.linalg.norm(a)
    for _ in range(max_sweeps):
        off = np.sqrt(max(np.sum(a * a) - np.sum(np.diag(a) ** 2), 0.0))
        if off <= tol * norm:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                c, s = _sym_schur2(a[p, p], a[q, q], a[p, q])
                if s == 0.0:
                    continue
                # A <- J^T A J with J the rotation in the (p, q) plane
                ap = a[:, p].copy()
                aq = a[:, q].copy()
                a[:, p] = c * ap - s * aq
                a[:, q] = s * ap + c * aq
                ap = a[p, :].copy()
                aq = a[q, :].copy()
                a[p, :] = c * ap - s * aq
                a[q, :] = s * ap + c * aq
                vp = v[:, p].copy()
                vq = v[:, q].copy()
                v[:, p] = c * vp - s * vq
                v[:, q] = s * vp + c * vq
    w = np.diag(a).copy()
    order = np.argsort(w)
    return w[order], v[:, order]
