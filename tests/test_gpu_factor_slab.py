"""The S factorisation modes and both own-column slab kernels against independent references.

* the Cholesky factor of T_b(S) in every mode against LAPACK's FP64 factor (numpy.linalg.cholesky);
* the double-float factor and the FP64 one give the same FP32 factor, L^-1 and A0;
* A0 (tensor-core congruence with three TF32 passes on the mixed path, SIMT FP32 on the FP32 path)
  against L^-1 T_b(H0) L^-T in FP64 from the library's own L^-1 and the block's H;
* blocks too large for the shared-memory-resident slab kernel (n_pad 640 in the FP32 path, 896 in
  the mixed path) run through the one-CTA slab kernel and keep the parity bar; blocks of n_pad 512
  in the FP32 path run through the resident kernel with compensated sums.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.nolsm import NolsmOracle  # noqa: E402
from synth import make_config, water_box  # noqa: E402


@pytest.fixture(scope="module")
def nl():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2205_12182_gb300 import nolsm
    return nolsm


@pytest.fixture(scope="module")
def sys1():
    return make_config(1)


@pytest.fixture(scope="module")
def orc1(sys1):
    return NolsmOracle.from_system(sys1)


@pytest.mark.parametrize("chol", [0, 1, 2, 3, 4])
def test_factor_matches_lapack(nl, sys1, orc1, chol):
    lib = nl.Nolsm(precision=nl.PREC_FP32, chol_precision=chol).build(sys1)
    for b in [0, 5, 31, 63]:
        _, _, sb = orc1.submatrices(b)
        ref = np.linalg.cholesky(sb)
        got = lib.block_matrix(b, 5).astype(np.float64)
        assert got.shape == ref.shape
        if chol == nl.CHOL_FP32:
            np.testing.assert_allclose(got, ref, rtol=0, atol=2e-5)
            continue
        # an FP64-accurate factor rounds to LAPACK's FP32 rounding, up to rounding-boundary cases.
        # The tensor-core updates slice every entry on its row's scale sqrt(S_rr), so their error
        # (~1e-13) is normwise: entries far below the scale (the decaying tail of L, down to 1e-20)
        # carry it as many of their own ulps, and the entrywise check covers |L| >= 1e-4 there.
        ref32 = ref.astype(np.float32)
        diff = np.abs(got - ref32.astype(np.float64))
        ulp = np.spacing(np.abs(ref32)).astype(np.float64)
        sel = np.abs(ref) >= 1e-4 if chol == nl.CHOL_DF64 else np.ones(ref.shape, bool)
        assert np.all(diff[sel] <= ulp[sel]), (b, float((diff[sel] / np.maximum(ulp[sel], 1e-45)).max()))
        assert np.count_nonzero(diff[sel]) <= 1e-3 * diff.size


@pytest.mark.parametrize("chol", ["df64_tensor", "df64_simt", "fp64"])
def test_factor_fp64_accuracy(nl, sys1, orc1, chol):
    """The factor as computed (before any FP32 rounding) against LAPACK's FP64 factor, relative to
    the row scales sqrt(S_rr S_cc) (O(1) here): the double-float modes carry a 48-bit significand
    (n_b ~ 200 terms: a few 1e-14), the tensor-core updates 48 bits of every slice product."""
    mode = {"df64_tensor": nl.CHOL_DF64, "df64_simt": nl.CHOL_DF64_SIMT, "fp64": nl.CHOL_FP64}[chol]
    bound = 1e-15 if chol == "fp64" else 1.5e-13
    lib = nl.Nolsm(precision=nl.PREC_FP32, chol_precision=mode).build(sys1)
    for b in [0, 5, 31, 63]:
        _, _, sb = orc1.submatrices(b)
        ref = np.linalg.cholesky(sb)
        scale = np.sqrt(np.outer(np.diag(sb), np.diag(sb)))
        err = np.abs(lib.block_factor(b) - ref) / scale
        assert err.max() <= bound, (b, float(err.max()))


def test_blocked_factor_on_large_blocks(nl):
    """n_b ~ 1,900 (30 panels of the blocked factorisation, 29 tensor-core trailing updates):
    the tensor-core factor against LAPACK and against the all-SIMT double-float factor."""
    from synth import water_clusters
    s = water_clusters(12, seed=41, cluster=(3, 3, 4))
    o = NolsmOracle.from_system(s, blocks=np.array([0, 29]))
    t = nl.Nolsm(precision=nl.PREC_MIXED_FP16, chol_precision=nl.CHOL_DF64).build(s)
    u = nl.Nolsm(precision=nl.PREC_MIXED_FP16, chol_precision=nl.CHOL_DF64_SIMT).build(s)
    for b in [0, 29]:
        _, _, sb = o.submatrices(b)
        ref = np.linalg.cholesky(sb)
        lt, lu = t.block_factor(b), u.block_factor(b)
        # n_b x 2^-48 (double-float sums over ~1,900 terms, and 48-bit slices of every tensor-core
        # product term) on O(1) row scales: 6.7e-12; measured ~1.3e-12 (tensor cores), ~5e-13 (SIMT)
        bound = sb.shape[0] * 2.0 ** -48
        assert np.abs(lt - ref).max() <= bound
        assert np.abs(lu - ref).max() <= bound
        assert np.abs(lt - lu).max() <= bound


def test_double_float_and_fp64_factor_agree_downstream(nl, sys1):
    a = nl.Nolsm(precision=nl.PREC_FP32, chol_precision=nl.CHOL_FP64).build(sys1)
    d = nl.Nolsm(precision=nl.PREC_FP32, chol_precision=nl.CHOL_DF64).build(sys1)
    for b in [0, 17, 63]:
        la, ld = a.block_matrix(b, 5), d.block_matrix(b, 5)
        big = np.abs(la) >= 1e-4           # below, the normwise ~1e-13 of the sliced updates shows
        assert np.mean(la[big] == ld[big]) >= 0.999
        np.testing.assert_allclose(ld, la, rtol=0, atol=np.spacing(np.float32(4.0)))
        for which in (1, 0):
            x, y = a.block_matrix(b, which), d.block_matrix(b, which)
            np.testing.assert_allclose(y, x, rtol=0, atol=1e-5 * max(1.0, float(np.abs(x).max())))


def _sampled_parity(nl, s, precision, n_sample, seed=0):
    lib = nl.Nolsm(precision=precision).build(s)
    mu, n, _ = lib.set_mu(s.n_electrons, tol_n=1e-3)
    d = lib.density().cpu().numpy()
    sample = np.random.default_rng(seed).choice(s.n_blocks, n_sample, replace=False)
    o = NolsmOracle.from_system(s, blocks=sample).prepare()
    assert min(np.min(np.abs(e - mu)) for e in o.eps) >= 1e-3
    own = np.isin(s.col, np.concatenate([s.block_cols(int(b)) for b in sample]))
    ref = o.density(mu)
    return np.abs(d[own] - ref[own]).max()


def test_fp32_path_resident_slab_n512(nl):
    s = water_box(10, seed=7, neighbourhood=8.0)        # n_b ~470, n_pad 512
    assert _sampled_parity(nl, s, nl.PREC_FP32, 6) <= 1e-6


def test_fp32_path_blocks_beyond_resident_slab(nl):
    s = water_box(6, seed=5, neighbourhood=9.0)         # n_b ~560, n_pad 640
    assert _sampled_parity(nl, s, nl.PREC_FP32, 6) <= 1e-6


def test_mixed_path_blocks_beyond_resident_slab(nl):
    s = water_box(8, seed=5, neighbourhood=10.0)        # n_b ~850, n_pad 896
    assert _sampled_parity(nl, s, nl.PREC_MIXED_FP16, 6) <= 1e-3


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_congruence_matches_fp64_product(nl, sys1, orc1, precision):
    prec = nl.PREC_FP32 if precision == "fp32" else nl.PREC_MIXED_FP16
    lib = nl.Nolsm(precision=prec).build(sys1)
    for b in [0, 9, 40, 63]:
        _, hb, _ = orc1.submatrices(b)
        li = lib.block_matrix(b, 1).astype(np.float64)
        ref = li @ hb.astype(np.float32).astype(np.float64) @ li.T
        a0 = lib.block_matrix(b, 0).astype(np.float64)
        np.testing.assert_array_equal(a0, a0.T)              # exactly symmetric
        # FP32 path: SIMT FP32 products; mixed path: three TF32 passes (~2^-21 per product term,
        # two products, ~200-term sums)
        tol = 1e-6 if precision == "fp32" else 1e-5
        assert np.abs(a0 - ref).max() <= tol * np.abs(ref).max()
