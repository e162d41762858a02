"""nolsm_combine_blocks (host code behind the C ABI, no GPU needed) against the combination reference.

Index work, so the bar is bit-exact: the same groups, merge for merge, as oracle/combine.py on
the 64-water box, 343- and 512-water boxes with the 8 A neighbourhood and random ring patterns
(with extra lists and a small max_dim), for Eq. 9 and Eq. 10.  At the benchmark size (4,096
waters) the reference is too slow, so the result is checked for what holds at any size: a
partition of the input blocks, dimensions that are the unions' sizes, the max_dim cap, and no
neighbouring pair of combined blocks left whose combination pays.
"""
import os

import numpy as np
import pytest

from oracle import combine as oc
from synth import make_config, water_box

from test_combine_oracle import random_instance

nl = pytest.importorskip("paper_2205_12182_gb300.nolsm")

PN_SYNTH = (np.array([128, 512, 1024, 4096], np.int32), np.array([4e-15, 2e-15, 1e-15, 0.9e-15]))


def native(system_like, criterion, pn=PN_SYNTH, max_dim=4096):
    row_ptr, col, blk_ptr, blk_cols, ep, ei = system_like
    n = len(row_ptr) - 1
    return nl.nolsm_combine_blocks(n, row_ptr, col, blk_ptr, blk_cols, ep, ei, criterion, pn[0], pn[1], max_dim)


def arrays(s):
    return s.row_ptr, s.col, s.blk_ptr, s.blk_cols, s.extra_ptr, s.extra_idx


def pn_tables():
    out = [("synthetic", PN_SYNTH)]
    if os.path.exists(nl.PN_TABLE):
        out.append(("measured", nl.load_pn_table()))
    return out


@pytest.mark.parametrize("criterion", [oc.CUBIC, oc.PERFORMANCE])
@pytest.mark.parametrize("which", ["water64", "water343", "water512"])
def test_same_groups_as_reference_on_water_boxes(which, criterion):
    s = {"water64": lambda: make_config(1), "water343": lambda: water_box(7, 5, neighbourhood=8.0),
         "water512": lambda: water_box(8, 5, neighbourhood=8.0)}[which]()
    for name, (dims, times) in pn_tables():
        r = native(arrays(s), criterion, (dims, times))
        g, merges = oc.combine(*arrays(s), criterion, dims, times)
        np.testing.assert_array_equal(r["group"], g, err_msg=name)
        assert r["n_blocks"] == g.max() + 1
        np.testing.assert_array_equal(r["dim"], oc.combined_dims(*arrays(s), g))
        base = oc.combined_dims(*arrays(s), np.arange(s.n_blocks))
        assert r["cost_in"] == pytest.approx(sum(oc.cost(int(n), criterion, dims, times) for n in base), rel=1e-12)
        assert r["cost_out"] == pytest.approx(sum(oc.cost(int(n), criterion, dims, times) for n in r["dim"]),
                                              rel=1e-12)
        if criterion == oc.PERFORMANCE and name == "synthetic":
            break


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("criterion", [oc.CUBIC, oc.PERFORMANCE])
def test_same_groups_as_reference_on_random_patterns(seed, criterion):
    row_ptr, col, blk_ptr, blk_cols, ep, ei, _ = random_instance(seed, with_extra=seed % 2 == 1)
    pn = (np.array([1, 8, 20, 72], np.int32), np.array([3.0, 2.0, 0.9, 0.8]))
    max_dim = 16 if seed % 3 == 0 else 4096
    r = native((row_ptr, col, blk_ptr, blk_cols, ep, ei), criterion, pn, max_dim)
    g, _ = oc.combine(row_ptr, col, blk_ptr, blk_cols, ep, ei, criterion, pn[0], pn[1], max_dim)
    np.testing.assert_array_equal(r["group"], g)


def test_outputs_describe_the_combined_blocks():
    s = water_box(7, 5, neighbourhood=8.0)
    r = native(arrays(s), oc.CUBIC)
    assert r["n_blocks"] < s.n_blocks
    for k in range(r["n_blocks"]):
        mem = np.flatnonzero(r["group"] == k)
        cols = r["blk_cols"][r["blk_ptr"][k]:r["blk_ptr"][k + 1]]
        np.testing.assert_array_equal(cols, np.concatenate([s.block_cols(int(b)) for b in mem]))
        ex = r["extra_idx"][r["extra_ptr"][k]:r["extra_ptr"][k + 1]]
        np.testing.assert_array_equal(ex, np.unique(np.concatenate([s.block_extra(int(b)) for b in mem])))
    # the combined blocks, given back as input, do not combine further
    again = native((s.row_ptr, s.col, r["blk_ptr"], r["blk_cols"], r["extra_ptr"], r["extra_idx"]), oc.CUBIC)
    assert again["n_blocks"] == r["n_blocks"]


def test_combine_blocks_returns_a_system():
    s = make_config(1)
    s2, r = nl.combine_blocks(s, nl.COMBINE_CUBIC)
    assert s2.n_blocks == r["n_blocks"] and s2.row_ptr is s.row_ptr
    assert sorted(s2.blk_cols.tolist()) == sorted(s.blk_cols.tolist())


@pytest.mark.parametrize("criterion", [oc.CUBIC, oc.PERFORMANCE])
def test_benchmark_size_properties(criterion):
    """4,096 waters, 8 A neighbourhood: properties that hold at any size."""
    s = make_config(2)
    pn = pn_tables()[-1][1]
    max_dim = 2048
    r = native(arrays(s), criterion, pn, max_dim)
    g = r["group"]
    m = r["n_blocks"]
    assert 0 < m < s.n_blocks and g.min() == 0 and g.max() == m - 1
    first = np.array([np.flatnonzero(g == k)[0] for k in range(m)])
    assert np.all(np.diff(first) > 0)                               # numbered by smallest member
    base = oc.combined_dims(*arrays(s), np.arange(s.n_blocks))
    sets = oc.index_sets(s.row_ptr, s.col, r["blk_ptr"], r["blk_cols"], r["extra_ptr"], r["extra_idx"])
    dims = np.array([len(x) for x in sets])
    np.testing.assert_array_equal(dims, r["dim"])
    assert np.all((dims <= max_dim) | (np.bincount(g) == 1))
    assert dims.max() <= max(max_dim, base.max())
    # no neighbouring pair of combined blocks whose combination pays
    owner = np.full(s.n_basis, -1)
    for k in range(m):
        owner[r["blk_cols"][r["blk_ptr"][k]:r["blk_ptr"][k + 1]]] = k
    own = [set(r["blk_cols"][r["blk_ptr"][k]:r["blk_ptr"][k + 1]].tolist()) for k in range(m)]
    checked = 0
    for a in range(m):
        for b in set(owner[list(sets[a])].tolist()) - {-1, a}:
            assert sets[a] & own[b]
            nm = len(sets[a] | sets[b])
            if nm <= max_dim:
                assert oc.saving(len(sets[a]), len(sets[b]), len(sets[a] & sets[b]), criterion, *pn) <= 0
                checked += 1
    assert checked > m


def test_errors_are_reported_before_any_output():
    s = make_config(1)
    cols = s.blk_cols.copy()
    cols[7] = cols[3]                                           # a column owned twice
    with pytest.raises(nl.NolsmError):
        nl.nolsm_combine_blocks(s.n_basis, s.row_ptr, s.col, s.blk_ptr, cols)
    with pytest.raises(nl.NolsmError):                          # sizes not ascending
        nl.nolsm_combine_blocks(s.n_basis, s.row_ptr, s.col, s.blk_ptr, s.blk_cols, None, None,
                                nl.COMBINE_PERFORMANCE, [512, 128], [1e-15, 2e-15])
    with pytest.raises(nl.NolsmError):                          # a non-positive time per flop
        nl.nolsm_combine_blocks(s.n_basis, s.row_ptr, s.col, s.blk_ptr, s.blk_cols, None, None,
                                nl.COMBINE_PERFORMANCE, [128, 512], [1e-15, 0.0])
    with pytest.raises(nl.NolsmError):                          # Eq. 10 without a table
        nl.nolsm_combine_blocks(s.n_basis, s.row_ptr, s.col, s.blk_ptr, s.blk_cols, None, None,
                                nl.COMBINE_PERFORMANCE)
    with pytest.raises(nl.NolsmError):
        nl.nolsm_combine_blocks(s.n_basis, s.row_ptr, s.col, s.blk_ptr, s.blk_cols, max_dim=0)


@pytest.mark.parametrize("reach,keep,n_blocks", [(2, 0.5, 10), (2, 1.0, 30), (6, 0.5, 30), (6, 1.0, 10)])
@pytest.mark.parametrize("criterion", [oc.CUBIC, oc.PERFORMANCE])
@pytest.mark.parametrize("seed", [20, 21])
def test_same_groups_across_pattern_shapes(reach, keep, n_blocks, criterion, seed):
    """Sparser and denser local couplings, few and many blocks, with extra lists and a cap that
    binds: the native combination follows the reference merge for merge."""
    row_ptr, col, blk_ptr, blk_cols, ep, ei, _ = random_instance(seed, n=96, n_blocks=n_blocks, reach=reach,
                                                                 keep=keep, with_extra=True)
    pn = (np.array([1, 6, 16, 40, 96], np.int32), np.array([5.0, 2.5, 1.2, 0.9, 0.85]))
    for max_dim in (12, 40, 4096):
        r = native((row_ptr, col, blk_ptr, blk_cols, ep, ei), criterion, pn, max_dim)
        g, _ = oc.combine(row_ptr, col, blk_ptr, blk_cols, ep, ei, criterion, pn[0], pn[1], max_dim)
        np.testing.assert_array_equal(r["group"], g)
        np.testing.assert_array_equal(r["dim"], oc.combined_dims(row_ptr, col, blk_ptr, blk_cols, ep, ei, g))


def test_measured_tables_are_usable():
    """The committed p(n) tables (products and whole step): ascending sizes 64..4096, positive times
    per flop, accepted by the native combination; the batch sizing of the measurement script."""
    from paper_2205_12182_gb300.measure_pn import batch_size
    for path in (nl.PN_TABLE, nl.PN_STEP_TABLE):
        dims, times = nl.load_pn_table(path)
        assert dims[0] == 64 and dims[-1] == 4096 and np.all(np.diff(dims) > 0)
        assert np.all(times > 0) and np.all(np.isfinite(times))
        r = native(arrays(make_config(1)), oc.PERFORMANCE, (dims, times))
        assert r["n_blocks"] >= 1
    assert batch_size(4096) == 5 and batch_size(64) == 16384
    assert all(4 <= batch_size(n) and batch_size(n) * n * n <= max(1e8, 4 * n * n) for n in range(64, 4097, 64))


def test_committed_schedule_table_is_usable():
    """The autotuner's committed schedule table: ascending n_pad from 128 to 4,096, schedules the
    library accepts in a table (persistent, per-product, persistent interleaved), one timing per
    schedule and size, and the recorded choice the fastest of them."""
    import json
    d = json.load(open(nl.SCHEDULE_TABLE))
    n_pad, sched, ms = nl.load_schedule_table()
    assert ms.shape == (len(n_pad), 3) and np.all(ms > 0)
    assert n_pad[0] == 128 and n_pad[-1] == 4096 and np.all(np.diff(n_pad) > 0)
    assert set(sched.tolist()) <= {nl.SCHEDULE_PERSISTENT, nl.SCHEDULE_PER_PRODUCT, nl.SCHEDULE_PERSISTENT_INTERLEAVED}
    kind = {"persistent": nl.SCHEDULE_PERSISTENT, "interleaved": nl.SCHEDULE_PERSISTENT_INTERLEAVED,
            "per_product": nl.SCHEDULE_PER_PRODUCT}
    for i in range(len(n_pad)):
        times = {k: d["ms"][k][i] for k in kind}
        assert all(t > 0 for t in times.values())
        assert sched[i] == kind[min(times, key=times.get)]
