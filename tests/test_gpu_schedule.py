"""The measured schedule table (nolsm_set_schedule_table) drives NOLSM_SCHEDULE_AUTO.

A ragged batch -- eight dense blocks of 300 and two of 1,500 side by side -- with a table that puts
n_pad <= 1,024 on the persistent kernel and larger blocks on per-product launches runs a split
evaluation: one persistent launch for the small blocks, then per-product launches for the large ones.
Every block runs the same arithmetic as under the single schedules (the persistent and per-product
schedules agree to 1e-4, see test_gpu_parity.py), and the density matches the oracle.  A table with one
schedule everywhere reproduces that schedule bit for bit.
"""
import dataclasses

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


def side_by_side(a, b):
    """Two uncoupled block-diagonal systems as one (b's indices shifted past a's)."""
    na = a.n_basis
    return dataclasses.replace(
        a, row_ptr=np.concatenate([a.row_ptr, a.row_ptr[-1] + b.row_ptr[1:]]),
        col=np.concatenate([a.col, b.col + na]).astype(np.int32), h=np.concatenate([a.h, b.h]),
        s=np.concatenate([a.s, b.s]), blk_ptr=np.concatenate([a.blk_ptr, a.blk_ptr[-1] + b.blk_ptr[1:]]),
        blk_cols=np.concatenate([a.blk_cols, b.blk_cols + na]).astype(np.int32),
        coords=np.zeros((na + b.n_basis, 3)), element=np.concatenate([a.element, b.element]),
        atom_bf_ptr=np.arange(na + b.n_basis + 1), n_electrons=a.n_electrons + b.n_electrons)


@pytest.fixture(scope="module")
def ragged():
    return side_by_side(dense_blocks(300, 8, seed=5, n_unique=2), dense_blocks(1500, 2, seed=6, n_unique=1))


def run(nl, s, schedule=None, table=None):
    lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16, **({} if schedule is None else {"schedule": schedule}))
    if table is not None:
        lib.set_schedule_table(table)
    lib.build(s)
    st = lib.sign_batch(-0.25)
    out = dict(st=st, iters=lib.iters(), d=lib.density().cpu().numpy(), sched=lib.last_schedule())
    lib.close()
    return out


def test_split_evaluation(nl, ragged):
    table = (np.array([1024, 8192]), np.array([nl.SCHEDULE_PERSISTENT, nl.SCHEDULE_PER_PRODUCT]))
    r = run(nl, ragged, table=table)
    assert r["sched"] == (-2, 8)          # split: the eight small blocks in the persistent launch
    ref = run(nl, ragged, schedule=nl.SCHEDULE_PER_PRODUCT)
    assert ref["sched"][0] == nl.SCHEDULE_PER_PRODUCT
    assert np.mean(r["iters"] == ref["iters"]) >= 0.9
    assert np.abs(r["d"] - ref["d"]).max() <= 1e-4
    # the large blocks took the same per-product launches in both runs
    big = np.arange(8, 10)
    np.testing.assert_array_equal(r["iters"][big], ref["iters"][big])
    o = NolsmOracle.from_system(ragged, blocks=np.array([0, 8])).prepare()
    own = np.isin(ragged.col, np.concatenate([ragged.block_cols(0), ragged.block_cols(8)]))
    assert np.abs(r["d"][own] - o.density(-0.25)[own]).max() <= 1e-3


@pytest.mark.parametrize("kind", ["persistent", "per_product"])
def test_single_schedule_tables(nl, ragged, kind):
    sched = nl.SCHEDULE_PERSISTENT if kind == "persistent" else nl.SCHEDULE_PER_PRODUCT
    r = run(nl, ragged, table=(np.array([4096]), np.array([sched])))
    ref = run(nl, ragged, schedule=sched)
    assert r["sched"][0] == sched and ref["sched"][0] == sched
    np.testing.assert_array_equal(r["iters"], ref["iters"])
    np.testing.assert_array_equal(r["d"], ref["d"])


def test_predicted_choice_with_times(nl, ragged):
    """With per-block times AUTO predicts the batch: times that make the persistent launch's tail
    cost more than the split saves give one schedule for every block; times that make the split
    clearly cheaper keep it."""
    n_pad = np.array([1024, 8192])
    sched = np.array([nl.SCHEDULE_PERSISTENT, nl.SCHEDULE_PER_PRODUCT])
    # persistent barely faster on the small bin, far slower on the large one: no split
    ms = np.array([[1.00, 1.01, 1.2], [50.0, 5.0, 90.0]])
    r = run(nl, ragged, table=(n_pad, sched, ms))
    assert r["sched"] == (nl.SCHEDULE_PER_PRODUCT, 0)
    # persistent far faster on the small bin (even with the tail of its last block): split
    ms = np.array([[0.001, 1.0, 0.002], [50.0, 5.0, 90.0]])
    r = run(nl, ragged, table=(n_pad, sched, ms))
    assert r["sched"] == (-2, 8)
    # every block fits the persistent kernel and it is predicted fastest: one persistent launch
    ms = np.array([[0.001, 1.0, 0.002], [0.5, 5.0, 0.7]])
    r = run(nl, ragged, table=(n_pad, np.array([nl.SCHEDULE_PERSISTENT, nl.SCHEDULE_PERSISTENT]), ms))
    assert r["sched"] == (nl.SCHEDULE_PERSISTENT, 10)


def test_bad_tables_are_refused(nl):
    lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16)
    with pytest.raises(nl.NolsmError):
        nl.nolsm_set_schedule_table(lib.ctx, np.array([512, 256]), np.array([0, 1]))
    with pytest.raises(nl.NolsmError):
        nl.nolsm_set_schedule_table(lib.ctx, np.array([512]), np.array([nl.SCHEDULE_AUTO]))
    with pytest.raises(nl.NolsmError):
        nl.nolsm_set_schedule_table(lib.ctx, np.array([512]), np.array([nl.SCHEDULE_PERSISTENT]),
                                    np.array([[1.0, -1.0, 1.0]]))
    nl.nolsm_set_schedule_table(lib.ctx, np.array([], np.int32), np.array([], np.int32))   # removes it
    lib.close()


def test_graph_loop_equals_host_loop(nl, ragged):
    """The per-product iteration as one captured graph (a device-side while loop) runs the same kernels
    in the same order as the host-driven loop: identical iterations and density, at two chemical
    potentials in a row (the graph is captured once and reused; mu is read on the device), with the
    restart path of learned-style bounds exercised by Lanczos bounds."""
    out = {}
    for loop in (nl.LOOP_HOST, nl.LOOP_GRAPH):
        lib = nl.Nolsm(precision=nl.PREC_MIXED_FP16, schedule=nl.SCHEDULE_PER_PRODUCT, loop=loop,
                       bounds=nl.BOUNDS_LANCZOS)
        lib.build(ragged)
        res = []
        for mu in (-0.25, -0.3):
            st = lib.sign_batch(mu)
            res.append((lib.iters().copy(), lib.density().cpu().numpy(), st["n_electrons"]))
        out[loop] = res
        lib.close()
    for (ih, dh, nh), (ig, dg, ng) in zip(out[nl.LOOP_HOST], out[nl.LOOP_GRAPH]):
        np.testing.assert_array_equal(ig, ih)
        np.testing.assert_array_equal(dg, dh)
        assert ng == nh
