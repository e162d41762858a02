"""Failure detection through status codes, with the failures made on the host (no GPU fault).

Each case breaks one input or limit and checks the status the library returns, and that the
context recovers with a fresh nolsm_build_submatrices.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import make_config  # noqa: E402


@pytest.fixture(scope="module")
def nl():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2205_12182_gb300 import nolsm
    return nolsm


@pytest.fixture(scope="module")
def sys1():
    return make_config(1)


def modified(system, **arrays):
    import copy
    s = copy.copy(system)
    for k, v in arrays.items():
        setattr(s, k, v)
    return s


def test_overlap_not_positive_definite(nl, sys1):
    s_bad = sys1.s.copy()
    rows = np.repeat(np.arange(sys1.n_basis), np.diff(sys1.row_ptr))
    off = rows != sys1.col
    s_bad[off] *= 6.0                     # off-diagonal overlaps blown up: T_b(S) indefinite
    lib = nl.Nolsm(precision=nl.PREC_FP32)
    with pytest.raises(nl.NolsmError) as e:
        lib.build(modified(sys1, s=s_bad))
    assert e.value.status == nl.ENOTPD
    lib.build(sys1)                       # a good build clears the sticky error
    lib.sign_batch(-0.45)


def test_nan_in_hamiltonian(nl, sys1):
    h_bad = sys1.h.copy()
    h_bad[17] = np.nan
    lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16)
    with pytest.raises(nl.NolsmError) as e:
        lib.build(modified(sys1, h=h_bad))
    assert e.value.status == nl.ENONFINITE


def test_iteration_limit(nl, sys1):
    lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16, max_iter=1).build(sys1)
    with pytest.raises(nl.NolsmError) as e:
        lib.sign_batch(-0.45)
    assert e.value.status == nl.ENOCONV
    with pytest.raises(nl.NolsmError) as e2:      # sticky until the next build
        lib.sign_batch(-0.45)
    assert e2.value.status == nl.ENOCONV


def test_unbracketed_electron_count(nl, sys1):
    lib = nl.Nolsm(precision=nl.PREC_FP32).build(sys1)
    with pytest.raises(nl.NolsmError) as e:       # far below the count that mu in [-3, -2.9] holds
        lib.set_mu(sys1.n_electrons, mu_lo=-3.0, mu_hi=-2.9, tol_n=1e-3)
    assert e.value.status == nl.EBRACKET


def test_bad_pattern_rejected(nl, sys1):
    col_bad = sys1.col.copy()
    r0 = int(sys1.row_ptr[5])
    col_bad[r0], col_bad[r0 + 1] = col_bad[r0 + 1], col_bad[r0]     # columns out of order in row 5
    lib = nl.Nolsm(precision=nl.PREC_FP32)
    with pytest.raises(nl.NolsmError) as e:
        lib.build(modified(sys1, col=col_bad))
    assert e.value.status == nl.EINVAL


@pytest.mark.parametrize("stage", ["build", "sign", "sign_interleaved"])
def test_device_wait_budget_runs_out(nl, sys1, stage):
    """A one-poll budget on the tensor-core kernels' mbarrier waits (the congruence in the build, the
    Newton-Schulz products in the sign evaluation, one or two blocks per cluster): the kernel records
    ETIMEOUT, drains its own copies and products, frees tensor memory and returns; the context
    recovers."""
    kw = {"schedule": nl.SCHEDULE_PERSISTENT_INTERLEAVED} if stage == "sign_interleaved" else {}
    lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16, wait_budget=1 if stage == "build" else 1 << 22, **kw)
    with pytest.raises(nl.NolsmError) as e:
        lib.build(sys1)
        lib.set_wait_budget(1)
        lib.sign_batch(-0.45)
    assert e.value.status == nl.ETIMEOUT
    torch.cuda.synchronize()
    ok = nl.Nolsm(precision=nl.PREC_MIXED_FP16).build(sys1)
    st = ok.sign_batch(-0.45)
    assert np.isfinite(st["n_electrons"])
