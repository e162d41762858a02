"""Pins of the combination reference (oracle/combine.py) against facts that do not come from it.

* Eq. 9 on two blocks: closed-form thresholds (equal sizes: combine iff the overlap exceeds
  (2 - 2^(1/3)) n; containment always combines; disjoint blocks never do).
* Eq. 10 special cases: a constant p(n) is Eq. 9; p(n) = c / n turns the cubic test into a
  quadratic one.
* The interpolated p(n) at, between and beyond its table sizes.
* The best-first order, replayed by brute force on small random patterns: every recorded merge is
  the best pair of the partition it was made from, and the final partition has no paying pair.
* Table II's trend on a water box: each criterion gives fewer and larger submatrices than the one
  before it.
"""
import numpy as np
import pytest

from oracle import combine as oc
from synth import water_box


def test_eq9_equal_sizes_threshold():
    for n in (1, 2, 7, 64, 480, 1000):
        for o in range(n + 1):
            pays = oc.saving(n, n, o, oc.CUBIC) > 0
            assert pays == (o > (2.0 - 2.0 ** (1.0 / 3.0)) * n), (n, o)


@pytest.mark.parametrize("na,nb", [(3, 1), (480, 200), (1000, 999), (4096, 17)])
def test_eq9_containment_and_disjoint(na, nb):
    assert oc.saving(na, nb, nb, oc.CUBIC) > 0               # I_b inside I_a: n stays n_a
    assert oc.saving(na, nb, 0, oc.CUBIC) < 0                # nothing shared: (a + b)^3 > a^3 + b^3


def test_eq10_reduces_to_eq9_for_constant_p():
    rng = np.random.default_rng(0)
    dims, times = [100, 1000, 4000], [2e-15, 2e-15, 2e-15]
    for _ in range(2000):
        na, nb = rng.integers(1, 3000, size=2)
        o = int(rng.integers(0, min(na, nb) + 1))
        assert (oc.saving(na, nb, o, oc.CUBIC) > 0) == (oc.saving(na, nb, o, oc.PERFORMANCE, dims, times) > 0)


def test_eq10_with_time_per_flop_inverse_in_n():
    """A table holding p(n) = 1 / n at every size 1..4096: p(n) n^3 = n^2, so Eq. 10 combines iff
    (n_a + n_b - n_ab)^2 < n_a^2 + n_b^2 (cases within rounding of a tie are skipped)."""
    dims = list(range(1, 4097))
    times = [1.0 / d for d in dims]
    rng = np.random.default_rng(1)
    for _ in range(2000):
        na, nb = (int(x) for x in rng.integers(1, 2000, size=2))
        o = int(rng.integers(0, min(na, nb) + 1))
        nm = na + nb - o
        quad = nm * nm < na * na + nb * nb
        if abs(nm * nm - (na * na + nb * nb)) > 2:                   # away from rounding ties
            assert (oc.saving(na, nb, o, oc.PERFORMANCE, dims, times) > 0) == quad


def test_time_per_flop_interpolation():
    dims, times = [128, 512, 1024], [4.0, 2.0, 1.0]
    assert oc.time_per_flop(128, dims, times) == 4.0
    assert oc.time_per_flop(512, dims, times) == 2.0
    assert oc.time_per_flop(1024, dims, times) == 1.0
    assert oc.time_per_flop(320, dims, times) == pytest.approx(3.0)
    assert oc.time_per_flop(768, dims, times) == pytest.approx(1.5)
    assert oc.time_per_flop(5, dims, times) == 4.0
    assert oc.time_per_flop(9999, dims, times) == 1.0


def random_instance(seed, n=72, n_blocks=20, reach=4, keep=0.8, with_extra=False):
    """A random structurally symmetric pattern with local coupling (points on a ring coupled to
    the ones within `reach` steps, each such pair kept with probability `keep`), the full diagonal,
    and blocks of 1-4 consecutive columns covering part of the ring (test input only)."""
    rng = np.random.default_rng(seed)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ring = np.minimum(np.abs(i - j), n - np.abs(i - j))
    a = (ring <= reach) & (rng.random((n, n)) < keep)
    a = np.triu(a, 1)
    a = a | a.T | np.eye(n, dtype=bool)
    row_ptr = np.zeros(n + 1, np.int64)
    row_ptr[1:] = np.cumsum(a.sum(1))
    col = np.concatenate([np.flatnonzero(a[r]) for r in range(n)]).astype(np.int32)
    sizes = rng.integers(1, 5, size=n_blocks)
    start = int(rng.integers(0, n))
    blk_ptr = np.zeros(n_blocks + 1, np.int32)
    blk_ptr[1:] = np.cumsum(sizes)
    blk_cols = ((start + np.arange(blk_ptr[-1])) % n).astype(np.int32)
    ep = ei = None
    if with_extra:
        ex = [np.sort(rng.choice(n, size=int(rng.integers(0, 4)), replace=False)) for _ in range(n_blocks)]
        ep = np.zeros(n_blocks + 1, np.int32)
        ep[1:] = np.cumsum([len(e) for e in ex])
        ei = np.concatenate(ex).astype(np.int32)
    return row_ptr, col, blk_ptr, blk_cols, ep, ei, a


def brute_sets(a, blk_ptr, blk_cols, ep, ei, members):
    """Index set and own columns of a union of input blocks, straight from the dense pattern."""
    rows, own = set(), set()
    for b in members:
        for c in blk_cols[blk_ptr[b]:blk_ptr[b + 1]]:
            own.add(int(c))
            rows.update(int(r) for r in np.flatnonzero(a[:, c]))
        if ep is not None:
            rows.update(int(r) for r in ei[ep[b]:ep[b + 1]])
    return rows, own


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("criterion", [oc.CUBIC, oc.PERFORMANCE])
def test_best_first_order_by_brute_force(seed, criterion):
    row_ptr, col, blk_ptr, blk_cols, ep, ei, a = random_instance(seed, with_extra=seed % 2 == 1)
    dims, times = [1, 8, 20, 72], [3.0, 2.0, 0.9, 0.8]
    max_dim = 16 if seed % 3 == 0 else 4096
    group, merges = oc.combine(row_ptr, col, blk_ptr, blk_cols, ep, ei, criterion, dims, times, max_dim)

    def t(n):
        return float(n) ** 3 * (1.0 if criterion == oc.CUBIC else np.interp(n, dims, times))

    parts = {b: [b] for b in range(len(blk_ptr) - 1)}

    def best_pair():
        best = None
        ids = sorted(parts)
        for i, x in enumerate(ids):
            for y in ids[i + 1:]:
                rx, ox = brute_sets(a, blk_ptr, blk_cols, ep, ei, parts[x])
                ry, oy = brute_sets(a, blk_ptr, blk_cols, ep, ei, parts[y])
                if not (rx & oy or ry & ox) or len(rx | ry) > max_dim:
                    continue
                g = t(len(rx)) + t(len(ry)) - t(len(rx | ry))
                if g > 1e-9 * t(len(rx | ry)) and (best is None or g > best[0] * (1 + 1e-12)):
                    best = (g, x, y)
        return best

    for (x, y, g) in merges:
        bp = best_pair()
        assert bp is not None and (bp[1], bp[2]) == (x, y)
        assert g == pytest.approx(bp[0], rel=1e-9)
        parts[x] = parts[x] + parts.pop(y)
    assert best_pair() is None                                   # nothing left that pays
    # the returned groups are the replayed partition, numbered by smallest member
    for k, x in enumerate(sorted(parts)):
        assert sorted(np.flatnonzero(group == k).tolist()) == sorted(parts[x])
    dims_out = oc.combined_dims(row_ptr, col, blk_ptr, blk_cols, ep, ei, group)
    assert dims_out.max() <= max(max_dim, max(len(brute_sets(a, blk_ptr, blk_cols, ep, ei, [b])[0])
                                              for b in range(len(blk_ptr) - 1)))


def test_index_sets_match_the_dense_pattern():
    row_ptr, col, blk_ptr, blk_cols, ep, ei, a = random_instance(3, with_extra=True)
    sets = oc.index_sets(row_ptr, col, blk_ptr, blk_cols, ep, ei)
    for b, s in enumerate(sets):
        assert s == brute_sets(a, blk_ptr, blk_cols, ep, ei, [b])[0]


def test_table2_trend_on_a_water_box():
    """Table II (Section III-B-1): no combination, Eq. 9, Eq. 10 with a time per flop that falls
    with n give fewer submatrices and a larger average dimension in that order, and Eq. 10's
    predicted time is below Eq. 9's."""
    s = water_box(7, 5, neighbourhood=8.0)
    dims, times = [128, 512, 1024, 4096], [4e-15, 2e-15, 1e-15, 0.9e-15]
    out = {}
    for crit in (oc.CUBIC, oc.PERFORMANCE):
        g, _ = oc.combine(s.row_ptr, s.col, s.blk_ptr, s.blk_cols, s.extra_ptr, s.extra_idx, crit, dims, times)
        out[crit] = oc.combined_dims(s.row_ptr, s.col, s.blk_ptr, s.blk_cols, s.extra_ptr, s.extra_idx, g)
    base = oc.combined_dims(s.row_ptr, s.col, s.blk_ptr, s.blk_cols, s.extra_ptr, s.extra_idx,
                            np.arange(s.n_blocks))
    assert len(base) > len(out[oc.CUBIC]) > len(out[oc.PERFORMANCE])
    assert base.mean() < out[oc.CUBIC].mean() < out[oc.PERFORMANCE].mean()

    def predicted(d):
        return sum(oc.cost(int(n), oc.PERFORMANCE, dims, times) for n in d)
    assert predicted(out[oc.PERFORMANCE]) < predicted(out[oc.CUBIC]) < predicted(base)
    # the cubic criterion never raises the flop count; Eq. 10 may (Table II: 1.54 -> 1.66 PFLOP)
    assert (out[oc.CUBIC].astype(float) ** 3).sum() < (base.astype(float) ** 3).sum()


def test_shared_rows_without_coupling_are_not_candidates():
    """Columns 0 and 1 both couple to rows 2..9 but not to each other: their index sets share 8 of
    9 rows (Eq. 9 would pay: 10^3 < 2 * 9^3), yet neither holds the other's own column, so the two
    blocks are not neighbours and stay apart.  A third block owning columns 2..9 (index set: all
    ten rows) is a neighbour of both and takes them in turn."""
    n = 10
    a = np.eye(n, dtype=bool)
    a[0, 2:] = a[2:, 0] = True
    a[1, 2:] = a[2:, 1] = True
    row_ptr = np.zeros(n + 1, np.int64)
    row_ptr[1:] = np.cumsum(a.sum(1))
    col = np.concatenate([np.flatnonzero(a[r]) for r in range(n)]).astype(np.int32)
    group, merges = oc.combine(row_ptr, col, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32))
    assert merges == [] and group.tolist() == [0, 1]
    group, merges = oc.combine(row_ptr, col, np.array([0, 1, 2, 10], np.int32), np.arange(10, dtype=np.int32))
    assert group.tolist() == [0, 0, 0] and len(merges) == 2
