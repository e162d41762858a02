// Step 1 of the submatrix method on the GPU: the pattern checks, the transpose position of every
// stored entry, and the index set I_b of every block -- the rows holding a stored entry in any of
// the block's own columns (on the combined pattern of H0 and S), unioned with the block's extra
// indices -- sorted ascending, with the local positions of the own columns.
#include "internal.h"

#include <climits>

namespace nolsm {
namespace {

__device__ __forceinline__ void set_error(DevFlags* f, int code) { atomicCAS(&f->error, 0, code); }

// One warp per row r: column range/order checks, the diagonal, and for entry (r, c) the
// position of (c, r) in row c (binary search; a miss means the pattern is not symmetric).
__global__ void transpose_kernel(int64_t n, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                 int64_t* __restrict__ transpose, DevFlags* flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
    const int64_t e0 = row_ptr[r], e1 = row_ptr[r + 1];
    bool diag = false;
    if (e1 < e0) set_error(flags, NOLSM_EINVAL);
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      const int32_t c = col[e];
      if (c < 0 || c >= n || (e > e0 && col[e - 1] >= c)) { set_error(flags, NOLSM_EINVAL); continue; }
      if (c == r) diag = true;
      int64_t lo = row_ptr[c], hi = row_ptr[c + 1];
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < r) lo = mid + 1; else hi = mid;
      }
      if (lo < row_ptr[c + 1] && col[lo] == r) transpose[e] = lo;
      else set_error(flags, NOLSM_EINVAL);
    }
    if (!__any_sync(0xffffffffu, diag) && lane == 0) set_error(flags, NOLSM_EINVAL);
  }
}

// Sort cand[0, m) ascending (bitonic, padded to a power of two with INT_MAX) and write its distinct
// values to I (at most max_dim of them; the count is returned in full).  The distinct values are then
// copied back to cand[0, count) so that further candidates can be appended.
__device__ int sort_unique(int32_t* cand, int m, int32_t* __restrict__ I, int32_t* warp_tot, int32_t* s_base,
                           int max_dim) {
  const int tid = threadIdx.x;
  int p2 = 1;
  while (p2 < m) p2 <<= 1;
  for (int i = m + tid; i < p2; i += blockDim.x) cand[i] = INT_MAX;
  __syncthreads();
  for (int k = 2; k <= p2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < p2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const int32_t a = cand[i], c = cand[l];
          const bool up = (i & k) == 0;
          if ((a > c) == up) { cand[i] = c; cand[l] = a; }
        }
      }
      __syncthreads();
    }
  // unique: positions by a block-wide scan over chunks of blockDim
  if (tid == 0) *s_base = 0;
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i0 = 0; i0 < m; i0 += blockDim.x) {
    const int i = i0 + tid;
    const int keep = (i < m) && (i == 0 || cand[i] != cand[i - 1]);
    const unsigned ballot = __ballot_sync(0xffffffffu, keep);
    const int before = __popc(ballot & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[warp] = __popc(ballot);
    __syncthreads();
    int off = *s_base;
    for (int w = 0; w < warp; ++w) off += warp_tot[w];
    const int32_t v = (i < m) ? cand[i] : 0;
    __syncthreads();
    if (keep && off + before < max_dim) I[off + before] = v;
    if (tid == 0) {
      int t = 0;
      for (int w = 0; w < nw; ++w) t += warp_tot[w];
      *s_base += t;
    }
    __syncthreads();
  }
  const int nb = *s_base;
  for (int i = tid; i < min(nb, max_dim); i += blockDim.x) cand[i] = I[i];
  __syncthreads();
  return nb;
}

// One CTA per block: gather the candidate rows into shared memory, bitonic sort, keep the first
// of every run of equal values.  I_b goes to idx[b * max_dim ...], |I_b| to n_out[b], and the
// local position of own column j to own[blk_ptr[b] + j].  When the next column's rows (or the next
// piece of the extra list) would overflow the cap entries, the candidates so far are sorted and made
// distinct first (at most max_dim remain).  More than max_dim distinct rows, or one column with more
// than cap - max_dim rows, is counted in flags->oversize while max_dim < kMaxDimLarge (the build
// then widens the stride and runs again) and is an EINVAL error for the block at kMaxDimLarge.
__global__ void __launch_bounds__(512) index_set_kernel(int64_t n, const int64_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ col,
                                                        const int32_t* __restrict__ blk_ptr,
                                                        const int32_t* __restrict__ blk_cols,
                                                        const int32_t* __restrict__ extra_ptr,
                                                        const int32_t* __restrict__ extra_idx, int cap,
                                                        int max_dim, int32_t* __restrict__ idx,
                                                        int32_t* __restrict__ own, int32_t* __restrict__ n_out,
                                                        DevFlags* flags) {
  extern __shared__ int32_t cand[];          // cap entries
  __shared__ int32_t warp_tot[16];
  __shared__ int32_t s_base;
  const int b = blockIdx.x;
  const int tid = threadIdx.x;
  int32_t* I = idx + (int64_t)b * max_dim;
  int m = 0;                                 // block-uniform candidate count
  bool bad = false;
  // candidates: the rows of every own column (row c's columns: the pattern is symmetric) + extras
  const int32_t c0 = blk_ptr[b], c1 = blk_ptr[b + 1];
  for (int32_t k = c0; k < c1 && !bad; ++k) {
    const int32_t c = blk_cols[k];
    if (c < 0 || c >= n) { if (tid == 0) set_error(flags, NOLSM_EINVAL); continue; }
    const int64_t e0 = row_ptr[c], e1 = row_ptr[c + 1];
    const int deg = (int)(e1 - e0);
    if (m + deg > cap) {
      m = sort_unique(cand, m, I, warp_tot, &s_base, max_dim);
      if (m > max_dim || m + deg > cap) { bad = true; break; }
    }
    for (int i = tid; i < deg; i += blockDim.x) cand[m + i] = col[e0 + i];
    m += deg;
    __syncthreads();
  }
  if (extra_ptr && !bad) {
    const int32_t x0 = extra_ptr[b], x1 = extra_ptr[b + 1];
    for (int32_t s = x0; s < x1 && !bad;) {
      if (m == cap) {
        m = sort_unique(cand, m, I, warp_tot, &s_base, max_dim);
        if (m >= cap || m > max_dim) { bad = true; break; }
      }
      const int take = min(x1 - s, cap - m);
      for (int i = tid; i < take; i += blockDim.x) {
        const int32_t v = extra_idx[s + i];
        if (v < 0 || v >= n) set_error(flags, NOLSM_EINVAL);
        cand[m + i] = min(max(v, 0), (int32_t)n - 1);
      }
      m += take;
      s += take;
      __syncthreads();
    }
  }
  const int nb = bad ? max_dim + 1 : sort_unique(cand, m, I, warp_tot, &s_base, max_dim);
  if (tid == 0) n_out[b] = bad ? 0 : nb;
  if (nb > max_dim) {
    if (tid == 0) {
      if (max_dim < kMaxDimLarge) atomicAdd(&flags->oversize, 1);
      else set_error(flags, NOLSM_EINVAL);
    }
    return;
  }
  // own-column positions (every own column is its own row's diagonal, so it is in I_b)
  for (int32_t k = c0 + tid; k < c1; k += blockDim.x) {
    const int32_t c = blk_cols[k];
    int lo = 0, hi = nb;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (I[mid] < c) lo = mid + 1; else hi = mid;
    }
    own[k] = lo;
  }
}

}  // namespace

cudaError_t launch_transpose(nolsm_ctx* ctx) {
  if (!ctx->d_row_ptr || !ctx->d_col || !ctx->d_transpose || !ctx->d_flags) return cudaErrorInvalidValue;
  const int threads = 256;
  const int64_t warps_needed = ctx->n;
  const int grid = (int)std::min<int64_t>((warps_needed * 32 + threads - 1) / threads, (int64_t)ctx->num_sms * 16);
  transpose_kernel<<<grid, threads, 0, ctx->stream>>>(ctx->n, ctx->d_row_ptr, ctx->d_col, ctx->d_transpose,
                                                      ctx->d_flags);
  return cudaGetLastError();
}

cudaError_t launch_index_sets(nolsm_ctx* ctx, const int32_t* d_blk_ptr, const int32_t* d_extra_ptr,
                              const int32_t* d_extra_idx, int32_t* d_nb, int cap, int max_dim) {
  if (!d_blk_ptr || !d_nb || !ctx->d_blk_cols || !ctx->d_idx || !ctx->d_own || (cap & (cap - 1)) != 0)
    return cudaErrorInvalidValue;
  const size_t smem = sizeof(int32_t) * (size_t)cap;
  static size_t attr = 0;
  if (smem > 48 * 1024 && smem > attr) {
    cudaError_t e = cudaFuncSetAttribute(index_set_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = smem;
  }
  index_set_kernel<<<ctx->n_blocks, 512, smem, ctx->stream>>>(ctx->n, ctx->d_row_ptr, ctx->d_col, d_blk_ptr,
                                                              ctx->d_blk_cols, d_extra_ptr, d_extra_idx, cap,
                                                              max_dim, ctx->d_idx, ctx->d_own, d_nb, ctx->d_flags);
  return cudaGetLastError();
}

}  // namespace nolsm
