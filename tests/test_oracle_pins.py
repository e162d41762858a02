"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test fixes the oracle to a closed form, an exact identity of the method, an
invariant of the exact density matrix, or an independent numerical route.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import jacobi
from oracle.nolsm import (NolsmOracle, density_eq8, full_density, index_set, newton_schulz,
                          sign_eq8, theta, csr_matrix)
from synth import dimer_system, isolated_waters, water_box

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense(system):
    n = system.n_basis
    h = csr_matrix(system.row_ptr, system.col, system.h, n).toarray()
    s = csr_matrix(system.row_ptr, system.col, system.s, n).toarray()
    return h, s


# --------------------------------------------------------------- closed form: the 2x2 dimer

@pytest.mark.parametrize("a,b,s", [(-1.0, -0.3, 0.2), (-0.5, -0.1, 0.0), (0.3, -0.25, 0.45), (-0.7, 0.2, -0.3)])
def test_dimer_closed_form(a, b, s):
    """H=[[a,b],[b,a]], S=[[1,s],[s,1]]: generalized eigenvalues (a+-b)/(1+-s); one occupied orbital.

    The bonding vector (1,1)/sqrt(2(1+s)) gives D = [[1,1],[1,1]] / (2(1+s)) when (a+b)/(1+s) is the
    lower level, else the antibonding (1,-1)/sqrt(2(1-s)) gives [[1,-1],[-1,1]] / (2(1-s)).
    """
    o = NolsmOracle.from_system(dimer_system(a, b, s))
    e_plus, e_minus = (a + b) / (1 + s), (a - b) / (1 - s)
    lo, hi = sorted([e_plus, e_minus])
    mu = 0.5 * (lo + hi)
    d = o.density(mu)
    if e_plus < e_minus:
        expect = np.array([1, 1, 1, 1]) / (2 * (1 + s))
    else:
        expect = np.array([1, -1, -1, 1]) / (2 * (1 - s))
    np.testing.assert_allclose(d, expect, atol=1e-14)
    assert o.electron_count(mu) == pytest.approx(1.0, abs=1e-14)
    assert o.band_energy(d) == pytest.approx(2 * lo, abs=1e-14)
    mu_b, n_b, _ = o.bisect(lo - 1.0, hi + 1.0, tol_rel=1e-12)
    assert lo < mu_b < hi and n_b == pytest.approx(1.0, abs=1e-12)


# --------------------------------------------------------------- exact identities of the method

def test_full_index_set_equals_exact_density(config1):
    """With every I_b = all indices, Eq. 8 per block is Eq. 5: NOLSM D = exact D (Section II)."""
    sysm = config1
    n = sysm.n_basis
    h, s = dense(sysm)
    n_occ = int(sysm.n_electrons / 2)
    d_exact, mu = full_density(h, s, n_occ)
    nb = 8
    blk_ptr = np.arange(nb + 1, dtype=np.int32) * 6
    blk_cols = np.arange(6 * nb, dtype=np.int32)
    extra_ptr = np.arange(nb + 1, dtype=np.int32) * n
    extra_idx = np.tile(np.arange(n, dtype=np.int32), nb)
    o = NolsmOracle(sysm.row_ptr, sysm.col, sysm.h, sysm.s, blk_ptr, blk_cols, sysm.n_electrons,
                    extra_ptr, extra_idx)
    o.prepare()
    for k in range(nb):
        assert len(o.idx[k]) == n
        cols = o.cols_of(k)
        np.testing.assert_allclose(o.block_density_cols(k, mu), d_exact[:, cols], atol=1e-11)


def test_isolated_molecules_are_exact():
    """Molecules farther apart than the cutoff: H0 and S block diagonal, so NOLSM is exact."""
    sysm = isolated_waters(8, seed=3)
    h, s = dense(sysm)
    n_occ = int(sysm.n_electrons / 2)
    d_exact, mu = full_density(h, s, n_occ)
    o = NolsmOracle.from_system(sysm).prepare()
    assert all(len(i) == 6 for i in o.idx)
    d = o.density(mu)
    # D is kept on the stored pattern only (zero intra-atom off-diagonals are not stored)
    rows = np.repeat(np.arange(sysm.n_basis), np.diff(sysm.row_ptr))
    np.testing.assert_allclose(d, d_exact[rows, sysm.col], atol=1e-12)
    assert o.electron_count(mu) == pytest.approx(n_occ, abs=1e-10)
    mu_b, n_b, steps = o.bisect(tol_rel=1e-9)
    assert n_b == pytest.approx(n_occ, rel=1e-9)


def test_full_matrix_invariants(config1):
    """Exact D (one block = all columns): sign^2 = I, DSD = D, Tr(DS) = N_occ, D = D^T, eig(DS) in {0,1}."""
    sysm = config1
    n = sysm.n_basis
    h, s = dense(sysm)
    o = NolsmOracle(sysm.row_ptr, sysm.col, sysm.h, sysm.s, [0, n], np.arange(n), sysm.n_electrons,
                    [0, n], np.arange(n)).prepare()
    n_occ = int(sysm.n_electrons / 2)
    mu = 0.5 * (o.eps[0][n_occ - 1] + o.eps[0][n_occ])
    d = o.block_density_cols(0, mu)
    np.testing.assert_allclose(d, d.T, atol=1e-12)
    np.testing.assert_allclose(d @ s @ d, d, atol=1e-10)
    assert np.trace(d @ s) == pytest.approx(n_occ, abs=1e-9)
    ev = np.sort(np.linalg.eigvals(d @ s).real)
    np.testing.assert_allclose(ev[: n - n_occ], 0.0, atol=1e-9)
    np.testing.assert_allclose(ev[n - n_occ:], 1.0, atol=1e-9)
    sg = sign_eq8(h, s, mu)
    np.testing.assert_allclose(sg @ sg, np.eye(n), atol=1e-8)
    np.testing.assert_allclose(0.5 * (np.eye(n) - sg) @ np.linalg.inv(s), d, atol=1e-8)


def test_orthogonal_case_is_eigenprojector():
    """S = I reduces Eq. 8 to the orthogonal submatrix method: D_b = spectral projector of H_b."""
    sysm = water_box(4, seed=7)
    s_identity = np.where(sysm.col == np.repeat(np.arange(sysm.n_basis), np.diff(sysm.row_ptr)), 1.0, 0.0)
    o = NolsmOracle(sysm.row_ptr, sysm.col, sysm.h, s_identity, sysm.blk_ptr, sysm.blk_cols,
                    sysm.n_electrons, blocks=[0, 5, 17]).prepare()
    mu = -0.45
    for k in range(3):
        _, hb, _ = o.submatrices(int(o.blocks[k]))
        w, v = np.linalg.eigh(hb)
        proj = (v * theta(mu - w)) @ v.T
        np.testing.assert_allclose(o.block_density_cols(k, mu), proj[:, o.own[k]], atol=1e-12)


def test_eq8_general_eig_route_matches(config1):
    """The reweighted eigh form equals Eq. 8 written out with a non-symmetric eigensolver."""
    o = NolsmOracle.from_system(config1, blocks=[0, 9, 33]).prepare()
    mu = -0.45
    for k in range(3):
        _, hb, sb = o.submatrices(int(o.blocks[k]))
        d_lit = density_eq8(hb, sb, mu)
        np.testing.assert_allclose(o.block_density_cols(k, mu), d_lit[:, o.own[k]], atol=1e-9)


# --------------------------------------------------------------- the iteration of Eq. 6

def test_scalar_newton_schulz_map():
    """For diagonal A, X_k stays diagonal and follows x -> x (3 - x^2) / 2 exactly."""
    x = np.array([0.05, -0.3, 0.9, -1.2, 1.7, 1e-3])
    xk = x.copy()
    for k in range(1, 8):
        xk = 0.5 * xk * (3 - xk * xk)
        np.testing.assert_allclose(np.diag(newton_schulz(np.diag(x), k)), xk, rtol=0, atol=1e-15)
    # below sqrt(3) every non-zero x converges to its sign; zero is a fixed point
    xs = np.array([1e-2, -0.5, 1.0, 1.5, -1.7, 0.0])
    np.testing.assert_allclose(np.diag(newton_schulz(np.diag(xs), 40)), np.sign(xs), atol=1e-12)


def test_newton_schulz_gives_matrix_sign():
    rng = np.random.default_rng(5)
    q, _ = np.linalg.qr(rng.normal(size=(40, 40)))
    lam = np.concatenate([rng.uniform(0.05, 1.0, 20), -rng.uniform(0.05, 1.0, 20)])
    a = (q * lam) @ q.T
    np.testing.assert_allclose(newton_schulz(a, 40), (q * np.sign(lam)) @ q.T, atol=1e-12)


# --------------------------------------------------------------- the oracle's one library dependency

@pytest.mark.parametrize("n", [1, 2, 5, 33, 64])
def test_jacobi_matches_lapack(n):
    rng = np.random.default_rng(n)
    a = rng.normal(size=(n, n))
    a = a + a.T
    if n >= 5:
        a[:2, :] = 0.0
        a[:, :2] = 0.0          # a double zero eigenvalue
    w, v = jacobi.eigh(a)
    np.testing.assert_allclose(w, np.linalg.eigvalsh(a), atol=1e-12 * max(1, np.abs(a).max()))
    np.testing.assert_allclose(v.T @ v, np.eye(n), atol=1e-12)
    np.testing.assert_allclose(v.T @ a @ v, np.diag(w), atol=1e-11 * max(1, np.abs(a).max()))


def test_oracle_jacobi_backend_matches_lapack():
    sysm = isolated_waters(8, seed=4)
    a = NolsmOracle.from_system(sysm).prepare()
    b = NolsmOracle.from_system(sysm, backend="jacobi").prepare()
    mu, _, _ = a.bisect(tol_rel=1e-9)
    np.testing.assert_allclose(a.density(mu), b.density(mu), atol=1e-12)
    s2 = water_box(4, seed=1)
    a = NolsmOracle.from_system(s2, blocks=[3]).prepare()
    b = NolsmOracle.from_system(s2, blocks=[3], backend="jacobi").prepare()
    np.testing.assert_allclose(a.block_density_cols(0, -0.45), b.block_density_cols(0, -0.45), atol=1e-10)


# --------------------------------------------------------------- step (1), step (3) and the traces

def test_index_set_brute_force(config1):
    sysm = config1
    n = sysm.n_basis
    pat = csr_matrix(sysm.row_ptr, sysm.col, np.ones(sysm.nnz), n).toarray() != 0
    o = NolsmOracle.from_system(sysm)
    for b in [0, 1, 40, 63]:
        cols = sysm.block_cols(b)
        brute = np.array([r for r in range(n) if any(pat[r, c] for c in cols)])
        np.testing.assert_array_equal(o.index_set(b), brute)
    extra = np.array([5, 100, 383])
    got = index_set(o.pattern, sysm.block_cols(2), extra)
    brute = sorted(set(r for r in range(n) if pat[r, sysm.block_cols(2)].any()) | set(extra.tolist()))
    np.testing.assert_array_equal(got, brute)


def test_traces_two_ways(config1):
    """N(mu), Tr(D S) of the scattered D, and the band energy agree between the two formulas."""
    o = NolsmOracle.from_system(config1).prepare()
    for mu in (-0.6, -0.45, -0.44):
        d = o.density(mu)
        assert o.trace_ds(d) == pytest.approx(o.electron_count(mu), abs=1e-10)
        assert o.band_energy(d) == pytest.approx(o.band_energy_of_mu(mu), abs=1e-10)
    # scatter keeps only stored positions of own columns: every stored entry is written
    d = o.density(-0.45)
    assert np.count_nonzero(d) > 0.99 * len(d)


def test_theta_convention():
    np.testing.assert_array_equal(theta(np.array([-1e-300, 0.0, 2.0])), [0.0, 0.5, 1.0])


# --------------------------------------------------------------- golden: Table II arithmetic

def test_table2_time_is_flops_over_performance():
    """Table II: estimated speedup = (FLOPs / performance) of no-combination over each criterion.

    Pins the reading of Eq. 10 in which p(n) enters as time per flop (1 / performance).
    """
    g = json.load(open(os.path.join(GOLDEN, "table2_combination.json")))
    f, p = g["pflop_per_multiplication"], g["estimated_tflops_per_a100"]
    t = [fi / pi for fi, pi in zip(f, p)]
    assert t[0] / t[1] == pytest.approx(g["estimated_speedup"][1], abs=0.05)
    assert t[0] / t[2] == pytest.approx(g["estimated_speedup"][2], abs=0.05)


# --------------------------------------------------------------- the approximation against the full matrix

def test_neighbourhood_submatrices_approximate_the_full_density():
    """343 waters with the 8 A neighbourhood: the submatrix densities (Eq. 8) against the exact density
    of the whole matrix (dense generalized eigendecomposition), both at the exact mu (midway between
    the exact HOMO and LUMO, so both occupy the same states): within 1e-3 on every stored entry.  The
    same blocks combined into one block covering the system give the exact density."""
    s = water_box(7, 5, neighbourhood=8.0)
    h, sm = dense(s)
    w, v = sla.eigh(h, sm)
    k = int(s.n_electrons // 2)
    mu = 0.5 * (w[k - 1] + w[k])
    rows = np.repeat(np.arange(s.n_basis), np.diff(s.row_ptr))
    exact = ((v * (w < mu)) @ v.T)[rows, s.col]
    o = NolsmOracle.from_system(s).prepare()
    assert np.abs(o.density(mu) - exact).max() <= 1e-3
    one = s.subset_blocks(np.arange(s.n_blocks))
    one.blk_ptr = np.array([0, s.blk_cols.size], np.int32)
    one.extra_ptr = np.array([0, s.extra_idx.size], np.int32)
    np.testing.assert_allclose(NolsmOracle.from_system(one).prepare().density(mu), exact, atol=1e-10)
