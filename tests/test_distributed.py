"""Shared-mu bisection over ranks (gloo, world size 2, CPU): same mu as one process over all blocks."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2205_12182_gb300.distributed import bisect_shared


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from oracle.nolsm import NolsmOracle
    from synth import make_config
    from paper_2205_12182_gb300.distributed import allreduce_minmax, allreduce_sum
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = make_config(1)
    blocks = np.arange(rank, s.n_blocks, world)          # this rank's blocks
    o = NolsmOracle.from_system(s, blocks=blocks).prepare()
    lo, hi = o.spectral_bounds()
    lo, hi = allreduce_minmax(lo - 1e-3, hi + 1e-3)
    mu, n, steps = bisect_shared(lambda m: 2 * o.electron_count(m), allreduce_sum, s.n_electrons, lo, hi, 1e-3)
    out[rank] = (mu, n, steps)
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


def test_bracket_error():
    with pytest.raises(RuntimeError):
        bisect_shared(lambda m: 0.0, lambda v: v, 10.0, -1.0, 1.0, 1e-6, max_steps=80)
