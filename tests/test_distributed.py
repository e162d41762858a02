"""Shared-mu bisection over ranks (gloo, world size 2, CPU): same mu as one process over all blocks."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2205_12182_gb300.distributed import aufbau_point, bisect_shared


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from oracle.nolsm import NolsmOracle
    from synth import make_config
    from paper_2205_12182_gb300.distributed import allreduce_minmax, allreduce_sum, allgather_floats, aufbau_point
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = make_config(1)
    blocks = np.arange(rank, s.n_blocks, world)          # this rank's blocks
    o = NolsmOracle.from_system(s, blocks=blocks).prepare()
    lo, hi = o.spectral_bounds()
    lo, hi = allreduce_minmax(lo - 1e-3, hi + 1e-3)
    mu, n, steps = bisect_shared(lambda m: 2 * o.electron_count(m), allreduce_sum, s.n_electrons, lo, hi, 1e-3)
    # a stand-in for the own-column diagonal of A0: the on-site energies of this rank's own columns
    own = np.concatenate([s.block_cols(int(b)) for b in blocks])
    diag = s.h[s.row_ptr[own] + np.array([np.searchsorted(s.col[s.row_ptr[c]:s.row_ptr[c + 1]], c) for c in own])]
    gathered = allgather_floats(diag.astype(np.float32))
    mu0 = aufbau_point(gathered, s.n_electrons)
    mu_a, n_a, steps_a = bisect_shared(lambda m: 2 * o.electron_count(m), allreduce_sum, s.n_electrons, lo, hi, 1e-3,
                                       mu0=mu0)
    out[rank] = (mu, n, steps, np.sort(gathered).tolist(), mu0, mu_a, n_a, steps_a)
    dist.destroy_process_group()


def test_two_ranks_agree_with_single_process():
    from oracle.nolsm import NolsmOracle
    from synth import make_config
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 1000
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    s = make_config(1)
    o = NolsmOracle.from_system(s).prepare()
    lo, hi = o.spectral_bounds()
    mu1, n1, st1 = bisect_shared(lambda m: 2 * o.electron_count(m), lambda v: v, s.n_electrons, lo - 1e-3, hi + 1e-3, 1e-3)
    assert out[0] == out[1]
    assert out[0][0] == pytest.approx(mu1, abs=1e-12)
    assert out[0][1] == pytest.approx(n1, rel=1e-12)
    assert out[0][2] == st1
    # the Aufbau first point from the gathered diagonals is that of one process over all columns
    diag_all = np.array([s.h[s.row_ptr[c] + np.searchsorted(s.col[s.row_ptr[c]:s.row_ptr[c + 1]], c)]
                         for c in range(s.n_basis)], np.float32)
    np.testing.assert_array_equal(np.array(out[0][3], np.float32), np.sort(diag_all))
    mu0 = aufbau_point(diag_all, s.n_electrons)
    assert out[0][4] == mu0
    d = np.sort(diag_all.astype(np.float64))
    k = int(s.n_electrons // 2)
    assert mu0 == 0.5 * (d[k - 1] + d[k])            # between the k-th and (k+1)-th smallest
    mu_a, n_a, st_a = bisect_shared(lambda m: 2 * o.electron_count(m), lambda v: v, s.n_electrons, lo - 1e-3,
                                    hi + 1e-3, 1e-3, mu0=mu0)
    assert out[0][5] == pytest.approx(mu_a, abs=1e-12) and out[0][7] == st_a


def test_aufbau_point_rule():
    d = np.array([0.3, -1.0, -0.5, 0.1, -0.2], np.float32)
    assert aufbau_point(d, 4.0) == pytest.approx(0.5 * (-0.5 + -0.2))
    assert aufbau_point(d, 0.0) is None and aufbau_point(d, 10.0) is None


def test_bracket_error():
    with pytest.raises(RuntimeError):
        bisect_shared(lambda m: 0.0, lambda v: v, 10.0, -1.0, 1.0, 1e-6, max_steps=80)
