"""The chunked solve (nolsm_solve_chunked) and the 1,000,000-molecule configuration.

Blocks are independent (Section II), so streaming them through the pools in chunks must give, block
for block, what one build of all blocks gives at the same chemical potential.  The 1,000,000-molecule
water system (6,000,000 basis functions, 31,250 blocks of 32-molecule clusters with an 8 A halo) is
generated on the device by synth.device (pinned to the numpy generator in test_synth.py and below),
solved with the learned bounds, and checked against the oracle on sampled blocks.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import water_clusters  # noqa: E402
from synth.device import water_clusters_device  # noqa: E402
from oracle_pool import oracle_device_blocks, trace_bounds_device  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2205_12182_gb300", "weights", "bounds_mlp.json")


@pytest.fixture(scope="module")
def nl():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2205_12182_gb300 import nolsm
    return nolsm


def learned(nl, **kw):
    lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16, bounds=nl.BOUNDS_LEARNED, **kw)
    lib.set_predictor(nl.BoundPredictor.load(WEIGHTS))
    return lib


def test_device_generator_matches_numpy():
    a = water_clusters(8, seed=31)
    b = water_clusters_device(8, seed=31, device="cuda")
    np.testing.assert_array_equal(a.row_ptr, b.row_ptr.cpu().numpy())
    np.testing.assert_array_equal(a.col, b.col.cpu().numpy())
    np.testing.assert_allclose(b.h.cpu().numpy(), a.h, rtol=0, atol=1e-15)
    np.testing.assert_allclose(b.s.cpu().numpy(), a.s, rtol=0, atol=1e-15)
    for k in ("blk_ptr", "blk_cols", "extra_ptr", "extra_idx"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))


@pytest.fixture(scope="module")
def clusters():
    """1,728 waters in 54 blocks of 32-molecule clusters with an 8 A halo (n_b ~ 1,800)."""
    return water_clusters_device(12, seed=41)


def test_chunked_equals_one_build(nl, clusters):
    s = clusters
    d_c = torch.zeros(s.nnz, dtype=torch.float64, device="cuda")
    lib = learned(nl)
    st = lib.solve_chunked(s, d_c, tol_n=1e-3, chunk_blocks=16, block_traces=True)
    lib.close()
    assert st["chunks"] == 4 and st["passes"] >= 1 and st["n_blocks"] == 54
    assert abs(st["n_electrons"] - s.n_electrons) <= 1e-3 * s.n_electrons
    one = learned(nl)
    one.build(s)
    ref = one.sign_batch(st["mu"])
    d_1 = one.density().cpu().numpy()
    n_b, e_b = one.block_traces()
    e_1 = one.band_energy()
    one.close()
    # block for block the same arithmetic: the same D, counts and energies
    np.testing.assert_array_equal(d_c.cpu().numpy(), d_1)
    np.testing.assert_array_equal(st["block_n"], n_b)
    np.testing.assert_array_equal(st["block_e"], e_b)
    assert st["n_electrons"] == pytest.approx(ref["n_electrons"], rel=1e-13)
    assert st["band_energy"] == pytest.approx(e_1, rel=1e-13)
    # D's entries are the FP32 products L^-T Y, the traces FP64 sums over the FP32 slabs: the two
    # energies agree to FP32 rounding
    assert abs(st["band_energy_traces"] - st["band_energy"]) / s.n_atoms <= 1e-5


def test_chunked_bisection_passes(nl, clusters):
    """A count tolerance the first point cannot meet: the passes follow the bisection, and the D left
    behind belongs to the mu returned."""
    s = clusters
    d_c = torch.zeros(s.nnz, dtype=torch.float64, device="cuda")
    lib = learned(nl)
    st = lib.solve_chunked(s, d_c, tol_n=1e-12, max_passes=3, chunk_blocks=20)
    lib.close()
    assert st["passes"] == 3 and st["chunks"] == 3
    one = learned(nl)
    one.build(s)
    ref = one.sign_batch(st["mu"])
    np.testing.assert_array_equal(d_c.cpu().numpy(), one.density().cpu().numpy())
    one.close()
    assert st["n_electrons"] == pytest.approx(ref["n_electrons"], rel=1e-13)


def test_million_molecules_sampled_parity(nl):
    """The 1,000,000-molecule configuration end to end (chunks sized to the free memory), mu to
    1e-3 relative, the oracle on 32 sampled blocks at the returned mu: D on their own columns and
    each block's share of N and E."""
    ds = water_clusters_device(100, seed=31)
    assert ds.n_blocks == 31250 and ds.n_basis == 6_000_000
    d = torch.zeros(ds.nnz, dtype=torch.float64, device="cuda")
    lib = learned(nl)
    st = lib.solve_chunked(ds, d, tol_n=1e-3, block_traces=True)
    lib.close()
    assert st["chunks"] > 1 and abs(st["n_electrons"] - ds.n_electrons) <= 1e-3 * ds.n_electrons
    assert abs(st["band_energy_traces"] - st["band_energy"]) / ds.n_atoms <= 1e-5
    sample = np.sort(np.random.default_rng(31).choice(ds.n_blocks, 32, replace=False))
    o_n, o_e, pos, o_d = oracle_device_blocks(ds, sample, st["mu"])
    dd = d[torch.from_numpy(pos).cuda()].cpu().numpy()
    assert np.abs(dd - o_d).max() <= 1e-3
    bn, be = trace_bounds_device(ds, sample, 1e-3)
    assert np.all(np.abs(st["block_n"][sample] - o_n) <= bn)
    assert np.all(np.abs(st["block_e"][sample] - o_e) <= be)
