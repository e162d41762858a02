"""The own-column refinement and traces on the tensor cores (mixed paths) against the FP32 SIMT
kernels and the FP64 oracle.

Both refinement paths start from the same final iterate X (same products, same stopping rules), so
their densities differ only by the refinement's arithmetic: the tensor-core path multiplies X as
stored by the FP32 slab split into hi + lo in the iterate's format (FP16: ~2^-22 relative or 2^-24
absolute; BF16: ~2^-16 relative) with FP32 accumulation.  Cases: one-molecule blocks (6 own columns,
one narrow piece), 36-molecule clusters (216 own columns: a 192-column wide piece plus a 24-column
narrow one) and the 32-molecule clusters with an 8 A halo of the 1,000,000-molecule system's block
shape (n_b ~ 1,870).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.nolsm import NolsmOracle  # noqa: E402
from synth import make_config, water_clusters  # noqa: E402
from oracle_pool import oracle_blocks, trace_bounds  # noqa: E402


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
    return NolsmOracle.from_system(sys1).prepare()


@pytest.fixture(scope="module")
def mu1(orc1):
    return orc1.bisect(tol_rel=1e-3)[0]


def both_paths(nl, system, mu, **kw):
    out = {}
    for path in (nl.REFINE_TENSOR, nl.REFINE_SIMT):
        lib = nl.Nolsm(refine_path=path, **kw).build(system)
        st = lib.sign_batch(mu)
        out[path] = (st, lib.iters(), lib.density().cpu().numpy())
        lib.close()
    return out[nl.REFINE_TENSOR], out[nl.REFINE_SIMT]


@pytest.mark.parametrize("refine", [0, 1, 2])
@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_refine_paths_agree_on_molecule_blocks(nl, sys1, orc1, mu1, refine, prec):
    precision = nl.PREC_MIXED_FP16 if prec == "fp16" else nl.PREC_MIXED_BF16
    (st, it, d), (st2, it2, d2) = both_paths(nl, sys1, mu1, precision=precision, refine_iters=refine)
    np.testing.assert_array_equal(it, it2)               # the same iterate feeds both refinements
    tol = 2e-6 if prec == "fp16" else 5e-5
    assert np.abs(d - d2).max() <= tol
    assert st["n_electrons"] == pytest.approx(st2["n_electrons"], rel=tol)
    # without a refinement step the FP16 iteration stops at ||X^2 - I||_F <= 0.05 (the stopping rule
    # leaves the last digits to the FP32 steps), so only refined results are held to the 1e-3 bar
    if prec == "fp16" and refine >= 1:
        assert np.abs(d - orc1.density(mu1)).max() <= 1e-3


def test_wide_and_narrow_pieces_of_one_block(nl):
    """216 own columns per block: one 192-column piece and one 24-column piece whose traces are
    summed; n_b ~ 2,000 (n_pad 2,048)."""
    s = water_clusters(12, seed=41, cluster=(3, 3, 4))
    assert s.n_blocks == 48 and len(s.block_cols(0)) == 216
    lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16).build(s)
    mu, n, _ = lib.set_mu(s.n_electrons, tol_n=1e-3)
    lib.close()
    (st, it, d), (st2, it2, d2) = both_paths(nl, s, mu, precision=nl.PREC_MIXED_FP16)
    np.testing.assert_array_equal(it, it2)
    # FP32 accumulation over K = 1,920 in two different orders (tensor memory vs the SIMT
    # kernel's compensated sums) through nine chained products: a few 1e-6 on O(1) entries
    assert np.abs(d - d2).max() <= 1e-5
    assert st["n_electrons"] == pytest.approx(st2["n_electrons"], rel=1e-6)
    assert st["band_energy"] == pytest.approx(st2["band_energy"], rel=1e-6)
    sample = np.array([3, 30])
    o = NolsmOracle.from_system(s, blocks=sample).prepare()
    own = np.isin(s.col, np.concatenate([s.block_cols(int(b)) for b in sample]))
    assert np.abs(d[own] - o.density(mu)[own]).max() <= 1e-3


def test_cluster_blocks_sampled_parity(nl):
    """32-molecule clusters with an 8 A halo (432 blocks, n_b ~ 1,870) through set_mu on the
    default path; the oracle checks 16 sampled blocks at the GPU's mu: D on their own columns and
    each block's share of N = Tr(D S) and E = 2 Tr(D H0) (within what max|dD| <= 1e-3 allows)."""
    s = make_config(5)
    lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16).build(s)
    mu, n, _ = lib.set_mu(s.n_electrons, tol_n=1e-3)
    assert abs(n - s.n_electrons) <= 1e-3 * s.n_electrons
    d = lib.density().cpu().numpy()
    e = lib.band_energy()
    n_b, e_b = lib.block_traces()
    lib.close()
    sample = np.sort(np.random.default_rng(5).choice(s.n_blocks, 16, replace=False))
    o_n, o_e, pos, o_d = oracle_blocks(s, sample, mu)
    assert np.abs(d[pos] - o_d).max() <= 1e-3
    bn, be = trace_bounds(s, sample, 1e-3)
    assert np.all(np.abs(n_b[sample] - o_n) <= bn)
    assert np.all(np.abs(e_b[sample] - o_e) <= be)
    assert n_b.sum() == pytest.approx(n, rel=1e-12) and np.isfinite(e)


def test_schedules_agree_on_large_blocks(nl):
    """n_pad 2,048: the per-product launches deal tiles round-robin over the SMs; the persistent
    pair kernel takes whole blocks.  Same arithmetic and stopping rules, so the same iterations."""
    s = water_clusters(12, seed=41, cluster=(3, 3, 4))
    out = {}
    for sched in (nl.SCHEDULE_PERSISTENT, nl.SCHEDULE_PER_PRODUCT, nl.SCHEDULE_AUTO):
        lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16, schedule=sched).build(s)
        st = lib.sign_batch(-0.45)
        out[sched] = (lib.iters(), lib.density().cpu().numpy(), st["n_electrons"])
        lib.close()
    (ia, da, na), (ib, db, nb) = out[nl.SCHEDULE_PERSISTENT], out[nl.SCHEDULE_PER_PRODUCT]
    assert np.mean(ia == ib) >= 0.95
    assert np.abs(da - db).max() <= 1e-4
    assert na == pytest.approx(nb, rel=1e-5)
    np.testing.assert_array_equal(out[nl.SCHEDULE_AUTO][1], db)   # AUTO picks per-product here
