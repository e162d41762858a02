"""The allocation-free band energy entry point agrees with the context-based one.

nolsm_band_energy_noalloc serves callers that may not allocate device memory (it keeps its
partial sums in a fixed array inside the library).  It must give the energy of
nolsm_band_energy for the same density, call after call, and refuse inputs larger than its
fixed scratch can reduce.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_band_energy_noalloc_matches_context_call():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2205_12182_gb300 import nolsm
    from synth import make_config

    s = make_config(1)
    lib = nolsm.Nolsm(precision=nolsm.PREC_FP32).build(s)
    lib.sign_batch(-0.45)
    d = lib.density()
    e_ref = lib.band_energy()
    h = torch.from_numpy(np.ascontiguousarray(s.h)).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out.fill_(float("nan"))
        nolsm.nolsm_band_energy_noalloc(s.nnz, d, h, 2.0, out, stream)
        torch.cuda.synchronize()
        e = out.item()
        assert abs(e - e_ref) / s.n_atoms <= 1e-4          # the suite's band-energy tolerance
        assert e == pytest.approx(e_ref, rel=1e-12)        # same sum, another order
    with pytest.raises(nolsm.NolsmError):
        nolsm.nolsm_band_energy_noalloc(2 ** 28 + 1, d, h, 2.0, out, stream)
    lib.close()
