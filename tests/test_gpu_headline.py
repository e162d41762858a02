"""Whole-system parity of the benchmark's configuration against the FP64 oracle.

The 4,096-molecule water box (24,576 basis functions, 8 A neighbourhood) solved exactly as the
benchmark times it: FP16 products with FP32 accumulation, learned spectral bounds, the double-float
S factor and the AUTO schedule, mu from nolsm_set_mu.  The oracle evaluates every one of the 4,096
blocks at the mu the GPU returned (a spawn pool on the host cores), and the test compares
  * D on every stored entry (max|dD| <= 1e-3, the mixed path's tolerance),
  * the electron count N = Tr(D S) (relative 1e-6) and every block's share of it,
  * the band energy E = 2 Tr(D H0) (1e-4 Ha per atom) and every block's share of it.
A block's shares may differ from the oracle's by at most what max|dD| <= 1e-3 on its own columns
allows (tests/oracle_pool.trace_bounds).
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import make_config  # noqa: E402
from oracle_pool import oracle_blocks, trace_bounds  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2205_12182_gb300", "weights", "bounds_mlp.json")


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2205_12182_gb300 import nolsm
    s = make_config(2)
    lib = nolsm.Nolsm(precision=nolsm.PREC_MIXED_FP16, bounds=nolsm.BOUNDS_LEARNED,
                      chol_precision=nolsm.CHOL_DF64, schedule=nolsm.SCHEDULE_AUTO)
    lib.set_predictor(nolsm.BoundPredictor.load(WEIGHTS))
    lib.build(s)
    mu, n, steps = lib.set_mu(s.n_electrons, tol_n=1e-3)
    d = lib.density().cpu().numpy()
    e = lib.band_energy()
    n_b, e_b = lib.block_traces()
    lib.close()
    o_n, o_e, pos, o_d = oracle_blocks(s, np.arange(s.n_blocks), mu)
    return dict(s=s, mu=mu, n=n, d=d, e=e, n_b=n_b, e_b=e_b, o_n=o_n, o_e=o_e, pos=pos, o_d=o_d)


def test_every_entry_of_d(run):
    s = run["s"]
    assert len(run["pos"]) == s.nnz                # every stored entry belongs to one block's column
    assert np.abs(run["d"][run["pos"]] - run["o_d"]).max() <= 1e-3


def test_electron_count(run):
    n_ref = run["o_n"].sum()
    assert abs(run["n"] - n_ref) <= 1e-6 * n_ref
    assert run["n_b"].sum() == pytest.approx(run["n"], rel=1e-12)


def test_band_energy(run):
    s = run["s"]
    e_ref = run["o_e"].sum()
    assert abs(run["e"] - e_ref) / s.n_atoms <= 1e-4
    assert abs(run["e_b"].sum() - e_ref) / s.n_atoms <= 1e-4


def test_block_shares(run):
    s = run["s"]
    bn, be = trace_bounds(s, np.arange(s.n_blocks), 1e-3)
    assert np.all(np.abs(run["n_b"] - run["o_n"]) <= bn)
    assert np.all(np.abs(run["e_b"] - run["o_e"]) <= be)
