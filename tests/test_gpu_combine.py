"""Combined submatrices (Section III-B-1, Eq. 9 / Eq. 10) through the GPU path, against the oracle.

* The library's own index sets of the combined blocks (nolsm_block_index_set) are the unions the
  combination reports, entry for entry.
* The density of the combined blocks on the mixed path (and on the FP32 path) matches the oracle
  evaluated on the same combined blocks at the GPU's mu, on sampled blocks.
* p(n) measurement: one point of the table script gives a finite, positive time per flop.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import combine as oc  # noqa: E402
from oracle.nolsm import NolsmOracle  # noqa: E402
from synth import water_box  # noqa: E402


@pytest.fixture(scope="module")
def nl():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2205_12182_gb300 import nolsm
    return nolsm


def pn_table(nl):
    import os
    if os.path.exists(nl.PN_TABLE):
        return nl.load_pn_table()
    return np.array([128, 512, 1024, 4096], np.int32), np.array([4e-15, 2e-15, 1e-15, 0.9e-15])


@pytest.fixture(scope="module")
def combined(nl):
    s = water_box(8, 5, neighbourhood=8.0)
    s2, r = nl.combine_blocks(s, nl.COMBINE_PERFORMANCE, pn_table(nl))
    assert r["n_blocks"] < s.n_blocks
    return s, s2, r


def test_index_sets_of_combined_blocks(nl, combined):
    s, s2, r = combined
    lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16).build(s2)
    sets = oc.index_sets(s2.row_ptr, s2.col, s2.blk_ptr, s2.blk_cols, s2.extra_ptr, s2.extra_idx)
    for b in range(s2.n_blocks):
        idx = nl.nolsm_block_index_set(lib.ctx, b)
        np.testing.assert_array_equal(idx, np.array(sorted(sets[b])))
        assert len(idx) == r["dim"][b]
    lib.close()


@pytest.mark.parametrize("prec", ["mixed", "fp32"])
def test_combined_blocks_density_parity(nl, combined, prec):
    s, s2, r = combined
    precision = nl.PREC_MIXED_FP16 if prec == "mixed" else nl.PREC_FP32
    lib = nl.Nolsm(precision=precision).build(s2)
    mu, n, _ = lib.set_mu(s2.n_electrons, tol_n=1e-3)
    d = lib.density().cpu().numpy()
    lib.close()
    order = np.argsort(r["dim"])
    sample = np.unique([order[0], order[len(order) // 2], order[-1]])     # smallest, median, largest
    o = NolsmOracle.from_system(s2, blocks=sample).prepare()
    own = np.isin(s2.col, np.concatenate([s2.block_cols(int(b)) for b in sample]))
    tol = 1e-3 if prec == "mixed" else 1e-6
    assert np.abs(d[own] - o.density(mu)[own]).max() <= tol


def test_measure_pn_point(nl):
    from paper_2205_12182_gb300.measure_pn import measure
    row = measure(nl, 256, reps=1, max_entries=2e6)
    assert np.isfinite(row["time_per_flop"]) and row["time_per_flop"] > 0
    assert row["blocks"] >= 4 and row["iters_avg"] > 0
