// Submatrix combination (Section III-B-1, Eq. 9 and Eq. 10): host-side planning of the column
// blocks before nolsm_build_submatrices.
//
// Combining blocks a and b gives one submatrix on I_a u I_b, of dimension n_a + n_b - n_ab.  Its
// cost is t(n) = n^3 (Eq. 9, the flops of the dense products up to a constant) or p(n) n^3 (Eq. 10,
// the predicted run time; p(n) is a measured time per flop, linear in n between the table's sizes
// and constant beyond its ends).  The combination pays iff t(n_merged) < t(n_a) + t(n_b).
//
// The paper takes the order of the combinations from an earlier publication of its authors; this
// file uses a best-first greedy order: candidates are neighbouring blocks (the index set of one
// holds an own column of the other), each step combines the candidate pair with the largest
// saving (ties to the smallest pair of ids) whose merged dimension is at most max_dim, the result
// keeps the smaller id, and the loop ends when no candidate pays.  Savings sit in a max-heap; an
// entry carries the version of both blocks and is dropped when either has changed since.
//
// This file is compiled with -ffp-contract=off so that p(n) n^3 and the savings round the same on
// every host (no fused multiply-add), and the decisions do not depend on the machine.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <queue>
#include <vector>

#include "nolsm.h"

namespace {

struct CostModel {
  int32_t criterion;
  int32_t n_points;
  const int32_t* dim;
  const double* time;

  // p(n): the table's time per flop, linear in n between neighbouring sizes
  double time_per_flop(int64_t n) const {
    if (n <= dim[0]) return time[0];
    if (n >= dim[n_points - 1]) return time[n_points - 1];
    // the first size at or above n closes the interval (binary search over the ascending sizes)
    const int32_t k = (int32_t)(std::lower_bound(dim + 1, dim + n_points, n,
                                                 [](int32_t d, int64_t v) { return (int64_t)d < v; }) -
                                (dim + 1));
    const int64_t n0 = dim[k], n1 = dim[k + 1];
    const double p0 = time[k], p1 = time[k + 1];
    const double frac = (double)(n - n0) / (double)(n1 - n0);
    const double step = (p1 - p0) * frac;
    return p0 + step;
  }
  // one side of Eq. 9 (n^3) or Eq. 10 (p(n) n^3) for a submatrix of dimension n
  double cost(int64_t n) const {
    const double n3 = (double)(n * n * n);
    if (criterion == NOLSM_COMBINE_CUBIC) return n3;
    return n3 * time_per_flop(n);
  }
  double saving(int64_t na, int64_t nb, int64_t nm) const {
    const double two = cost(na) + cost(nb);
    return two - cost(nm);
  }
};

struct Candidate {
  double saving;
  int32_t a, b;          // a < b
  uint32_t va, vb;       // versions of a and b when the saving was computed
};

// max-heap order: larger saving first, then the smaller (a, b)
struct Later {
  bool operator()(const Candidate& x, const Candidate& y) const {
    if (x.saving != y.saving) return x.saving < y.saving;
    if (x.a != y.a) return x.a > y.a;
    return x.b > y.b;
  }
};

void sorted_insert(std::vector<int32_t>& v, int32_t x) {
  auto it = std::lower_bound(v.begin(), v.end(), x);
  if (it == v.end() || *it != x) v.insert(it, x);
}

void sorted_erase(std::vector<int32_t>& v, int32_t x) {
  auto it = std::lower_bound(v.begin(), v.end(), x);
  if (it != v.end() && *it == x) v.erase(it);
}

}  // namespace

extern "C" nolsm_status nolsm_combine_blocks(const nolsm_csr* pattern, int32_t n_blocks, const int32_t* blk_ptr,
                                             const int32_t* blk_cols, const int32_t* extra_ptr,
                                             const int32_t* extra_idx, int32_t criterion, int32_t n_points,
                                             const int32_t* pn_dim, const double* pn_time, int32_t max_dim,
                                             int32_t* n_out, int32_t* group, int32_t* out_blk_ptr,
                                             int32_t* out_blk_cols, int32_t* out_extra_ptr, int32_t* out_extra_idx,
                                             int32_t* out_dim, double* cost) {
  // ---- argument checks (nothing is written before they pass)
  if (!pattern || !blk_ptr || !blk_cols || !n_out || !group || n_blocks <= 0 || max_dim < 1)
    return NOLSM_EINVAL;
  if (pattern->memory != NOLSM_MEM_HOST || !pattern->row_ptr || !pattern->col || pattern->n <= 0 ||
      pattern->n > INT32_MAX)
    return NOLSM_EINVAL;
  if ((extra_ptr == nullptr) != (extra_idx == nullptr)) return NOLSM_EINVAL;
  if ((out_extra_ptr || out_extra_idx) && !extra_ptr) return NOLSM_EINVAL;
  if (criterion != NOLSM_COMBINE_CUBIC && criterion != NOLSM_COMBINE_PERFORMANCE) return NOLSM_EINVAL;
  if (criterion == NOLSM_COMBINE_PERFORMANCE) {
    if (n_points < 1 || !pn_dim || !pn_time) return NOLSM_EINVAL;
    for (int32_t k = 0; k < n_points; ++k) {
      if (pn_dim[k] < 1 || !(pn_time[k] > 0.0) || !std::isfinite(pn_time[k])) return NOLSM_EINVAL;
      if (k > 0 && pn_dim[k] <= pn_dim[k - 1]) return NOLSM_EINVAL;
    }
  }
  const int64_t N = pattern->n;
  const int64_t* rp = pattern->row_ptr;
  const int32_t* col = pattern->col;
  if (rp[0] != 0) return NOLSM_EINVAL;
  for (int64_t r = 0; r < N; ++r)
    if (rp[r + 1] < rp[r]) return NOLSM_EINVAL;
  if (blk_ptr[0] != 0) return NOLSM_EINVAL;
  for (int32_t b = 0; b < n_blocks; ++b)
    if (blk_ptr[b + 1] < blk_ptr[b]) return NOLSM_EINVAL;
  if (extra_ptr) {
    if (extra_ptr[0] != 0) return NOLSM_EINVAL;
    for (int32_t b = 0; b < n_blocks; ++b)
      if (extra_ptr[b + 1] < extra_ptr[b]) return NOLSM_EINVAL;
    for (int32_t k = 0; k < extra_ptr[n_blocks]; ++k)
      if (extra_idx[k] < 0 || extra_idx[k] >= N) return NOLSM_EINVAL;
  }
  const CostModel model{criterion, n_points, pn_dim, pn_time};

  try {
    // ---- owner of every column; index sets I_b (sorted, distinct)
    std::vector<int32_t> owner((size_t)N, -1);
    for (int32_t b = 0; b < n_blocks; ++b)
      for (int32_t k = blk_ptr[b]; k < blk_ptr[b + 1]; ++k) {
        const int32_t c = blk_cols[k];
        if (c < 0 || c >= N || owner[c] >= 0) return NOLSM_EINVAL;   // out of range or owned twice
        owner[c] = b;
      }
    for (int64_t e = 0; e < rp[N]; ++e)
      if (col[e] < 0 || col[e] >= N) return NOLSM_EINVAL;
    std::vector<std::vector<int32_t>> idx((size_t)n_blocks);
    for (int32_t b = 0; b < n_blocks; ++b) {
      std::vector<int32_t>& s = idx[b];
      for (int32_t k = blk_ptr[b]; k < blk_ptr[b + 1]; ++k) {
        const int32_t c = blk_cols[k];
        s.push_back(c);
        s.insert(s.end(), col + rp[c], col + rp[c + 1]);   // the pattern is symmetric: column c = row c
      }
      if (extra_ptr) s.insert(s.end(), extra_idx + extra_ptr[b], extra_idx + extra_ptr[b + 1]);
      std::sort(s.begin(), s.end());
      s.erase(std::unique(s.begin(), s.end()), s.end());
    }
    // ---- neighbours: b' owns a row of I_b (either direction)
    std::vector<std::vector<int32_t>> nbr((size_t)n_blocks);
    for (int32_t b = 0; b < n_blocks; ++b)
      for (int32_t r : idx[b]) {
        const int32_t o = owner[r];
        if (o >= 0 && o != b) { nbr[b].push_back(o); nbr[o].push_back(b); }
      }
    for (auto& v : nbr) {
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
    }
    double cost_in = 0.0;
    for (int32_t b = 0; b < n_blocks; ++b) cost_in += model.cost((int64_t)idx[b].size());

    // ---- best-first merging
    std::vector<uint32_t> version((size_t)n_blocks, 0);
    std::vector<char> alive((size_t)n_blocks, 1);
    std::vector<std::vector<int32_t>> members((size_t)n_blocks);
    for (int32_t b = 0; b < n_blocks; ++b) members[b].push_back(b);
    std::priority_queue<Candidate, std::vector<Candidate>, Later> heap;
    // |I_a n I_x| for the neighbours x of one block a: a's rows are stamped once, then each
    // neighbour's rows are counted (O(n_a + sum n_x) instead of a merge per pair)
    std::vector<uint32_t> stamp((size_t)N, 0u);
    uint32_t epoch = 0;
    auto stamp_rows = [&](int32_t a) {
      if (++epoch == 0) {                        // wrapped: clear and start again
        std::fill(stamp.begin(), stamp.end(), 0u);
        epoch = 1;
      }
      for (int32_t r : idx[a]) stamp[r] = epoch;
    };
    auto stamped = [&](int32_t x) {
      int64_t c = 0;
      for (int32_t r : idx[x]) c += stamp[r] == epoch;
      return c;
    };
    // the saving of combining a (rows stamped) with x, pushed when it pays
    auto consider = [&](int32_t a_st, int32_t x) {
      const int32_t a = std::min(a_st, x), b = std::max(a_st, x);
      const int64_t na = (int64_t)idx[a].size(), nb = (int64_t)idx[b].size();
      const int64_t nm = na + nb - stamped(x);
      if (nm > max_dim) return;
      const double g = model.saving(na, nb, nm);
      if (g > 0.0) heap.push(Candidate{g, a, b, version[a], version[b]});
    };
    for (int32_t a = 0; a < n_blocks; ++a) {
      stamp_rows(a);
      for (int32_t b : nbr[a])
        if (b > a) consider(a, b);
    }
    std::vector<int32_t> merged;
    while (!heap.empty()) {
      const Candidate c = heap.top();
      heap.pop();
      if (!alive[c.a] || !alive[c.b] || version[c.a] != c.va || version[c.b] != c.vb) continue;
      const int32_t a = c.a, b = c.b;     // a keeps the combined block
      merged.clear();
      std::set_union(idx[a].begin(), idx[a].end(), idx[b].begin(), idx[b].end(), std::back_inserter(merged));
      idx[a].swap(merged);
      std::vector<int32_t>().swap(idx[b]);
      members[a].insert(members[a].end(), members[b].begin(), members[b].end());
      std::vector<int32_t>().swap(members[b]);
      std::vector<int32_t> nm;
      std::set_union(nbr[a].begin(), nbr[a].end(), nbr[b].begin(), nbr[b].end(), std::back_inserter(nm));
      sorted_erase(nm, a);
      sorted_erase(nm, b);
      for (int32_t x : nm) {
        sorted_erase(nbr[x], b);
        sorted_insert(nbr[x], a);
      }
      nbr[a].swap(nm);
      std::vector<int32_t>().swap(nbr[b]);
      alive[b] = 0;
      ++version[a];
      stamp_rows(a);
      for (int32_t x : nbr[a]) consider(a, x);
    }

    // ---- outputs, combined blocks in ascending order of their smallest member
    int32_t k = 0, pc = 0, pe = 0;
    double cost_out = 0.0;
    if (out_blk_ptr) out_blk_ptr[0] = 0;
    if (out_extra_ptr) out_extra_ptr[0] = 0;
    std::vector<int32_t> ex;
    for (int32_t a = 0; a < n_blocks; ++a) {
      if (!alive[a]) continue;
      std::vector<int32_t>& mem = members[a];
      std::sort(mem.begin(), mem.end());
      for (int32_t b : mem) {
        group[b] = k;
        if (out_blk_cols)
          for (int32_t j = blk_ptr[b]; j < blk_ptr[b + 1]; ++j) out_blk_cols[pc++] = blk_cols[j];
        else
          pc += blk_ptr[b + 1] - blk_ptr[b];
      }
      if (out_blk_ptr) out_blk_ptr[k + 1] = pc;
      if (out_extra_ptr || out_extra_idx) {
        ex.clear();
        for (int32_t b : mem) ex.insert(ex.end(), extra_idx + extra_ptr[b], extra_idx + extra_ptr[b + 1]);
        std::sort(ex.begin(), ex.end());
        ex.erase(std::unique(ex.begin(), ex.end()), ex.end());
        if (out_extra_idx) std::memcpy(out_extra_idx + pe, ex.data(), sizeof(int32_t) * ex.size());
        pe += (int32_t)ex.size();
        if (out_extra_ptr) out_extra_ptr[k + 1] = pe;
      }
      if (out_dim) out_dim[k] = (int32_t)idx[a].size();
      cost_out += model.cost((int64_t)idx[a].size());
      ++k;
    }
    *n_out = k;
    if (cost) { cost[0] = cost_in; cost[1] = cost_out; }
    return NOLSM_OK;
  } catch (const std::bad_alloc&) {
    return NOLSM_ENOMEM;
  }
}
