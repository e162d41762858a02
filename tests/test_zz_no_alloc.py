"""The allocation-free band energy entry point agrees with the context-based one.

nolsm_band_energy_noalloc serves callers that may not allocate device memory where they need the
energy (a molecular-dynamics step under a fixed memory budget, a runtime that owns every device
allocation through its own pool): it keeps its partial sums in a fixed array inside the library.
It must give the energy of nolsm_band_energy (and of the oracle's Tr(D H0)) for the same density,
call after call, allocate nothing once its module is loaded, and refuse inputs larger than its
fixed scratch can reduce.

The file is named so that pytest collects it last: its first call loads the array's module into
the context, and a run that stops at the first failure has then already run every other test.  It
does not depend on that order: it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_band_energy_noalloc_matches_context_call():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from oracle.nolsm import NolsmOracle
    from paper_2205_12182_gb300 import nolsm
    from synth import make_config

    s = make_config(1)
    lib = nolsm.Nolsm(precision=nolsm.PREC_FP32).build(s)
    lib.sign_batch(-0.45)
    d = lib.density()
    e_ref = lib.band_energy()
    e_oracle = NolsmOracle.from_system(s).band_energy(d.cpu().numpy())
    h = torch.from_numpy(np.ascontiguousarray(s.h)).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    # the first call loads the library's module that holds the array (lazy loading); the second
    # call must then allocate nothing, neither through torch's allocator nor on the device
    for k in range(2):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        before = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
        nolsm.nolsm_band_energy_noalloc(s.nnz, d, h, 2.0, out, stream)
        torch.cuda.synchronize()
        after = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
        if k == 1:
            assert after == before, (before, after)
        e = out.item()
        assert abs(e - e_ref) / s.n_atoms <= 1e-4          # the suite's band-energy tolerance
        assert e == pytest.approx(e_ref, rel=1e-12)        # same sum, another order
        assert abs(e - e_oracle) / s.n_atoms <= 1e-4       # the oracle's Tr(D H0) of the same D
    with pytest.raises(nolsm.NolsmError):
        nolsm.nolsm_band_energy_noalloc(2 ** 28 + 1, d, h, 2.0, out, stream)
    lib.close()
