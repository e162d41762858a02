"""The FP8 experiment (FP8 operands as a measured alternative): the first fp8_iters Newton-Schulz
iterations round both product outputs to FP8 E4M3 values (the operand precision of an FP8 MMA,
without its rate).  fp8_iters = 0 is the default path bit for bit.  One or two FP8 iterations
still converge (finite, electron count within 1 %) but miss the accuracy bar by two orders of
magnitude: the rounding error a product leaves in the iterate is not removed by the later
iterations (they converge to the sign of the perturbed iterate), so FP8's 3-bit mantissa costs
about 0.1 in D.  The option needs a persistent schedule."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.nolsm import NolsmOracle  # noqa: E402
from synth import make_config  # noqa: E402


@pytest.fixture(scope="module")
def nl():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2205_12182_gb300 import nolsm
    return nolsm


@pytest.fixture(scope="module")
def case():
    s = make_config(1)
    o = NolsmOracle.from_system(s).prepare()
    return s, o, o.bisect(tol_rel=1e-3)[0]


def run(nl, s, mu, **kw):
    lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16, schedule=nl.SCHEDULE_PERSISTENT, **kw).build(s)
    st = lib.sign_batch(mu)
    d = lib.density().cpu().numpy()
    lib.close()
    return st, d


def test_zero_fp8_iterations_is_the_default_path(nl, case):
    s, o, mu = case
    st0, d0 = run(nl, s, mu)
    st1, d1 = run(nl, s, mu, fp8_iters=0)
    np.testing.assert_array_equal(d0, d1)


@pytest.mark.parametrize("k", [1, 2])
def test_fp8_iterations_converge_but_miss_the_bar(nl, case, k):
    s, o, mu = case
    st, d = run(nl, s, mu, fp8_iters=k)
    assert np.all(np.isfinite(d))
    assert st["n_electrons"] == pytest.approx(2 * o.electron_count(mu), rel=1e-2)
    assert np.abs(d - o.density(mu)).max() > 1e-2


def test_fp8_needs_a_persistent_schedule(nl, case):
    s, o, mu = case
    lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16, schedule=nl.SCHEDULE_PER_PRODUCT, fp8_iters=2).build(s)
    with pytest.raises(nl.NolsmError) as e:
        lib.sign_batch(mu)
    assert e.value.status == nl.EINVAL
