"""Bounds carried from one geometry to the next (the density step reruns every MD time step).

After the sign evaluation of one geometry, nolsm_keep_bounds runs Lanczos on A0 and on |A0 - mu|
and keeps per block (lambda_min, lambda_max, log10 distance of mu to the spectrum); the next
geometry (every atom displaced by 0.02 A, same blocks) is built on the same context and its sign
evaluations take those values as the scale and lower bound (NOLSM_BOUNDS_GIVEN), with mu searched
in a bracket around the previous one.  Checked against the oracle on the new geometry, and against
the iteration count of Gershgorin bounds with no knowledge of the gap (lower bound 1e-3).  The caller can also hand in bounds (here: the oracle's
exact spectra of the 64-water box).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.nolsm import NolsmOracle  # noqa: E402
from synth import displaced, make_config, water_box  # noqa: E402


@pytest.fixture(scope="module")
def nl():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2205_12182_gb300 import nolsm
    return nolsm


def test_bounds_kept_for_the_next_geometry(nl):
    s0 = water_box(10, seed=7, neighbourhood=8.0)
    s1 = displaced(s0, 0.02, seed=8)
    lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16, bounds=nl.BOUNDS_GIVEN).build(s0)
    mu0, n0, _ = lib.set_mu(s0.n_electrons, tol_n=1e-3)          # none kept yet: Gershgorin
    assert abs(n0 - s0.n_electrons) <= 1e-3 * s0.n_electrons
    lib.keep_bounds(64)
    lib.build(s1)
    mu1, n1, steps = lib.set_mu(s1.n_electrons, mu_lo=mu0 - 0.02, mu_hi=mu0 + 0.02, tol_n=1e-3)
    assert abs(n1 - s1.n_electrons) <= 1e-3 * s1.n_electrons
    st = lib.sign_batch(mu1)
    d = lib.density().cpu().numpy()
    lib.close()
    g = nl.Nolsm(precision=nl.PREC_MIXED_FP16, lower_bound=1e-3).build(s1)
    sg = g.sign_batch(mu1)
    g.close()
    assert st["iters_avg"] < sg["iters_avg"]
    sample = np.random.default_rng(3).choice(s1.n_blocks, 6, replace=False)
    o = NolsmOracle.from_system(s1, blocks=sample).prepare()
    own = np.isin(s1.col, np.concatenate([s1.block_cols(int(b)) for b in sample]))
    assert np.abs(d[own] - o.density(mu1)[own]).max() <= 1e-3


def test_bounds_given_by_the_caller(nl):
    s = make_config(1)
    o = NolsmOracle.from_system(s).prepare()
    mu = o.bisect(tol_rel=1e-3)[0]
    given = np.array([[e.min(), e.max(), np.log10(np.min(np.abs(e - mu)))] for e in o.eps], np.float32)
    lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16, bounds=nl.BOUNDS_GIVEN).build(s)
    lib.set_block_bounds(given)
    st = lib.sign_batch(mu)
    d = lib.density().cpu().numpy()
    lib.close()
    g = nl.Nolsm(precision=nl.PREC_MIXED_FP16, lower_bound=1e-3).build(s)
    sg = g.sign_batch(mu)
    g.close()
    assert np.abs(d - o.density(mu)).max() <= 1e-3
    assert st["iters_avg"] < sg["iters_avg"] and st["n_restarted"] == 0
