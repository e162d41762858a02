"""Plain CPU reference of the submatrix combination (Section III-B-1, Eq. 9 and Eq. 10).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this module.  The
library's combination (``nolsm_combine_blocks``) shares no code with it.

What the paper fixes (Section III-B-1):

* Each column block b has a submatrix of dimension n_b = |I_b| (its index set,
  step (1) of the method).  Combining two blocks i and j gives one submatrix
  whose index set is the union, of dimension n_i + n_j - n_{i^j}, n_{i^j} the
  number of shared indices.
* Eq. 9 (cubic metric): the combination pays iff
  (n_i + n_j - n_{i^j})^3 < n_i^3 + n_j^3 -- the flops of the dense products.
* Eq. 10 (performance-aware): the same comparison of predicted run times
  p(n) n^3, p(n) obtained by measuring the product throughput of the GPU at a
  set of sizes and interpolating.

Readings (the paper is silent or garbled on these points; the readings are stated here in full):

* p(n) is a time per flop (the reciprocal of the measured FLOP/s at size n):
  the paper calls it a performance but multiplies it by n^3 to get a run
  time, and its Table II speedups are FLOPs / performance.  The table is
  interpolated linearly in n between its sizes and held constant beyond its
  ends.
* The order in which pairs are combined belongs to an earlier publication of
  the authors that is not reproduced in this paper.  This reference uses a
  best-first greedy order: the candidates are the neighbouring pairs (the
  index set of one holds an own column of the other), every step combines the
  candidate pair with the largest saving t(n_i) + t(n_j) - t(n_merged) > 0
  whose merged dimension is at most max_dim (ties to the smallest pair of
  block ids), the combined block takes the smaller id, and it stops when no
  candidate pays.

Everything here is written for clarity, not speed: each step scans every pair
of current blocks for the best saving; a pair's saving is computed from the two
index sets once and forgotten when either block changes.
"""
from __future__ import annotations

import numpy as np

CUBIC = 0          # Eq. 9
PERFORMANCE = 1    # Eq. 10


def index_sets(row_ptr, col, blk_ptr, blk_cols, extra_ptr=None, extra_idx=None) -> list:
    """Step (1) of the method for every block, as Python sets: the rows with a stored entry in an
    own column (the pattern is symmetric, so column c's rows are row c's columns), the own columns
    themselves and the block's extra list."""
    out = []
    for b in range(len(blk_ptr) - 1):
        rows = set()
        for c in blk_cols[blk_ptr[b]:blk_ptr[b + 1]]:
            c = int(c)
            rows.add(c)
            rows.update(int(r) for r in col[row_ptr[c]:row_ptr[c + 1]])
        if extra_ptr is not None:
            rows.update(int(r) for r in extra_idx[extra_ptr[b]:extra_ptr[b + 1]])
        out.append(rows)
    return out


def time_per_flop(n: int, pn_dim, pn_time) -> float:
    """p(n) of Eq. 10: the measured time per flop, linear in n between the table's sizes and
    constant beyond its first and last size."""
    if n <= pn_dim[0]:
        return float(pn_time[0])
    if n >= pn_dim[-1]:
        return float(pn_time[-1])
    k = 0
    while pn_dim[k + 1] < n:
        k += 1
    n0, n1 = int(pn_dim[k]), int(pn_dim[k + 1])
    p0, p1 = float(pn_time[k]), float(pn_time[k + 1])
    return p0 + (p1 - p0) * (float(n - n0) / float(n1 - n0))


def cost(n: int, criterion: int, pn_dim=None, pn_time=None) -> float:
    """The quantity each side of Eq. 9 (n^3) or Eq. 10 (p(n) n^3) adds up for one submatrix."""
    n3 = float(n * n * n)
    if criterion == CUBIC:
        return n3
    return n3 * time_per_flop(n, pn_dim, pn_time)


def saving(na: int, nb: int, n_ab: int, criterion: int, pn_dim=None, pn_time=None) -> float:
    """t(n_a) + t(n_b) - t(n_a + n_b - n_ab): positive iff Eq. 9 / Eq. 10 says combine."""
    nm = na + nb - n_ab
    return (cost(na, criterion, pn_dim, pn_time) + cost(nb, criterion, pn_dim, pn_time)) \
        - cost(nm, criterion, pn_dim, pn_time)


def combine(row_ptr, col, blk_ptr, blk_cols, extra_ptr=None, extra_idx=None, criterion=CUBIC,
            pn_dim=None, pn_time=None, max_dim=4096):
    """Best-first greedy combination of the column blocks.

    Returns (group, merges): group[b] = index of the combined block that input block b belongs to
    (combined blocks numbered by their smallest member), and the list of merges in the order made,
    each (a, b, saving) with a < b the ids of the two blocks at that step.
    """
    n_in = len(blk_ptr) - 1
    I = index_sets(row_ptr, col, blk_ptr, blk_cols, extra_ptr, extra_idx)
    own = [set(int(c) for c in blk_cols[blk_ptr[b]:blk_ptr[b + 1]]) for b in range(n_in)]
    members = {b: [b] for b in range(n_in)}
    sets = {b: I[b] for b in range(n_in)}
    owns = {b: own[b] for b in range(n_in)}

    def pair_saving(a, b):
        """The saving of combining a and b, or None when they are not neighbours or too large."""
        if not (sets[a] & owns[b] or sets[b] & owns[a]):
            return None
        na, nb = len(sets[a]), len(sets[b])
        n_ab = len(sets[a] & sets[b])
        if na + nb - n_ab > max_dim:
            return None
        return saving(na, nb, n_ab, criterion, pn_dim, pn_time)

    known = {}     # (a, b) -> saving of the current blocks a and b (dropped when either changes)
    merges = []
    while True:
        best = None
        alive = sorted(sets)
        for i, a in enumerate(alive):
            for b in alive[i + 1:]:
                if (a, b) not in known:
                    known[(a, b)] = pair_saving(a, b)
                g = known[(a, b)]
                if g is not None and g > 0 and (best is None or g > best[0]):   # ties: smallest ids
                    best = (g, a, b)
        if best is None:
            break
        g, a, b = best
        sets[a] = sets[a] | sets.pop(b)
        owns[a] = owns[a] | owns.pop(b)
        members[a] = members[a] + members.pop(b)
        known = {k: v for k, v in known.items() if a not in k and b not in k}
        merges.append((a, b, g))
    group = np.empty(n_in, dtype=np.int64)
    for k, a in enumerate(sorted(members)):
        group[members[a]] = k
    return group, merges


def combined_dims(row_ptr, col, blk_ptr, blk_cols, extra_ptr, extra_idx, group) -> np.ndarray:
    """Dimension of every combined block: the size of the union of its members' index sets."""
    I = index_sets(row_ptr, col, blk_ptr, blk_cols, extra_ptr, extra_idx)
    n_out = int(group.max()) + 1
    u = [set() for _ in range(n_out)]
    for b, g in enumerate(group):
        u[int(g)] |= I[b]
    return np.array([len(s) for s in u], dtype=np.int64)
