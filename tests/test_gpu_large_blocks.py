"""Submatrices above 4,096 (the paper's Table II reaches 10,737): the index sets take the wide
stride, the products run per-product launches, and the result matches the FP64 oracle.

One dense block of n = 8,000 (synth.dense_blocks: S = I + E, H0 = diag(-1 or +0.5) + F, a gap
around -0.25 Ha), and three identical blocks of n = 4,200 beside a small one, so that blocks below
and above 4,096 share a build.  Mixed FP16 path; max|dD| <= 1e-3, the electron count within 1e-6
relative and the band energy within 1e-4 Ha per basis function (the blocks have no atoms), at the
oracle's mu in the gap.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.nolsm import NolsmOracle  # noqa: E402
from synth import dense_blocks  # noqa: E402


@pytest.fixture(scope="module")
def nl():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2205_12182_gb300 import nolsm
    return nolsm


def _check(nl, s, oracle_blocks):
    o = NolsmOracle.from_system(s, blocks=oracle_blocks).prepare()
    mu = -0.25
    lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16).build(s)
    dims = [nl.nolsm_block_info(lib.ctx, b)[0] for b in range(s.n_blocks)]
    st = lib.sign_batch(mu)
    d = lib.density().cpu().numpy()
    n_b, e_b = lib.block_traces()
    lib.close()
    own = np.isin(s.col, np.concatenate([s.block_cols(int(b)) for b in oracle_blocks]))
    assert np.abs(d[own] - o.density(mu)[own]).max() <= 1e-3
    n_ref = 2 * o.electron_count(mu)
    assert n_b[oracle_blocks].sum() == pytest.approx(n_ref, rel=1e-6)
    e_ref = o.band_energy_of_mu(mu)
    n_bf = sum(len(s.block_cols(int(b))) for b in oracle_blocks)
    assert abs(e_b[oracle_blocks].sum() - e_ref) / n_bf <= 1e-4
    return dims, st


def test_one_block_of_8000(nl):
    s = dense_blocks(8000, 1, seed=80)
    dims, st = _check(nl, s, np.array([0]))
    assert dims == [8000] and st["iters_max"] < 100


def test_blocks_above_and_below_4096_in_one_build(nl):
    big = dense_blocks(4200, 3, seed=42, n_unique=1)
    small = dense_blocks(300, 1, seed=43)
    # the two block-diagonal systems side by side (uncoupled): three blocks of 4,200, one of 300
    import dataclasses
    nb_big = big.n_basis
    s = dataclasses.replace(
        big, row_ptr=np.concatenate([big.row_ptr, big.row_ptr[-1] + small.row_ptr[1:]]),
        col=np.concatenate([big.col, small.col + nb_big]).astype(np.int32), h=np.concatenate([big.h, small.h]),
        s=np.concatenate([big.s, small.s]), blk_ptr=np.concatenate([big.blk_ptr, big.blk_ptr[-1] + small.blk_ptr[1:]]),
        blk_cols=np.concatenate([big.blk_cols, small.blk_cols + nb_big]).astype(np.int32),
        coords=np.zeros((nb_big + small.n_basis, 3)), element=np.concatenate([big.element, small.element]),
        atom_bf_ptr=np.arange(nb_big + small.n_basis + 1), n_electrons=big.n_electrons + small.n_electrons)
    dims, st = _check(nl, s, np.array([0, 3]))
    assert dims == [4200, 4200, 4200, 300]
