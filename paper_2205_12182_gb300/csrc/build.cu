// Everything that does not depend on mu: submatrix gather (step 1 of the submatrix
// method), the Cholesky factor of T_b(S) and its inverse, the congruence
// A0 = L^-1 T_b(H0) L^-T (Eq. 8 rewritten with S = L L^T), the own-column slabs and
// the Gershgorin bounds of A0.
#include "internal.h"

#include <cfloat>

namespace nolsm {
namespace {

__device__ __forceinline__ int lower_bound_i32(const int32_t* a, int n, int32_t key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void set_error(DevFlags* f, int code) { atomicCAS(&f->error, 0, code); }

// ----------------------------------------------------------------------------------------------
// FP64 -> double-float pair with integer operations (the FP64 pipe of this GPU issues at 1/64 of
// the FP32 rate): h = x rounded to nearest-even FP32, l = x - h rounded to FP32 -- the same pair as
// (float)x and (float)(x - (double)(float)x).  Zero and |x| outside [2^-60, 2^101) take the FP64
// route.
__device__ __forceinline__ float2 df_pair_from_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((b >> 52) & 0x7FFu) - 1023;
  if (be < -60 || be > 100) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
  }
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);   // 53-bit significand
  unsigned int top = (unsigned int)(m >> 29);                             // its leading 24 bits
  const unsigned int rest = (unsigned int)(m & 0x1FFFFFFFull);            // the other 29
  const bool up = rest > 0x10000000u || (rest == 0x10000000u && (top & 1u));
  top += up ? 1u : 0u;
  const int lm = (int)rest - (up ? 0x20000000 : 0);                       // x - h in units of 2^(be-52)
  float h = (float)top * __int_as_float((be - 23 + 127) << 23);           // exact
  float l = (float)lm * __int_as_float((be - 52 + 127) << 23);            // rounded to 24 bits, then exact
  if (b >> 63) { h = -h; l = -l; }
  return make_float2(h, l);
}

// ----------------------------------------------------------------------------------------------
// Gather: dense T_b(H0) (FP32) and T_b(S) (FP64, or double-float pairs in the same 8 bytes when
// `pairs`), ld = n_pad, from the CSR rows listed in I_b.  One CTA per block: it first writes the
// block's whole padded region (zeros, and a unit diagonal of S on the padding), then one warp per
// local row scatters the row's stored entries; I_b sits in shared memory for the column lookup
// (binary search).
__global__ void gather_kernel(const BlockDesc* __restrict__ blocks, const int32_t* __restrict__ idx_pool,
                              const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                              const double* __restrict__ hval, const double* __restrict__ sval,
                              float* __restrict__ hb, double* __restrict__ sb, DevFlags* flags, int pairs) {
  extern __shared__ int32_t s_idx[];
  const BlockDesc bd = blocks[blockIdx.x];
  const int n = bd.n, ld = bd.n_pad;
  float* H = hb + bd.off_mat;
  double* S = sb + bd.off_mat;
  float2* S2 = reinterpret_cast<float2*>(S);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int r = warp; r < ld; r += nwarps)
    for (int c = lane; c < ld; c += 32) {
      H[(int64_t)r * ld + c] = 0.f;
      if (pairs) S2[(int64_t)r * ld + c] = make_float2((r == c && r >= n) ? 1.f : 0.f, 0.f);
      else S[(int64_t)r * ld + c] = (r == c && r >= n) ? 1.0 : 0.0;
    }
  for (int i = threadIdx.x; i < n; i += blockDim.x) s_idx[i] = idx_pool[bd.off_idx + i];
  __syncthreads();
  for (int p = warp; p < n; p += nwarps) {
    const int32_t r = s_idx[p];
    const int64_t e0 = row_ptr[r], e1 = row_ptr[r + 1];
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      const int32_t c = col[e];
      const int q = lower_bound_i32(s_idx, n, c);
      if (q < n && s_idx[q] == c) {
        const double h = hval[e], s = sval[e];
        if (!isfinite(h) || !isfinite(s)) set_error(flags, NOLSM_ENONFINITE);
        H[(int64_t)p * ld + q] = (float)h;
        if (pairs) S2[(int64_t)p * ld + q] = df_pair_from_f64(s);
        else S[(int64_t)p * ld + q] = s;
      }
    }
  }
}

// The same gather for blocks up to n_pad kGatherRowMax, written row by row: a warp assembles a dense
// row of T_b(H0) and T_b(S) in its own shared-memory buffer (zeros, the row's stored entries, the
// unit diagonal on the padding) and writes it once with 16-byte stores, so every byte written is
// written once and coalesced.  In the double-float modes only the lower triangle of T_b(S) (up to the
// pair that holds the diagonal) is written: the factor reads no other entry (the trailing updates'
// boxes that reach above the diagonal are read and written back unused).  Dynamic shared memory: I_b,
// then per warp n_pad floats and n_pad 8-byte entries.
constexpr int kGatherRowMax = 2048;
constexpr int kGatherWarps = 8;
__global__ void __launch_bounds__(kGatherWarps * 32) gather_rows_kernel(
    const BlockDesc* __restrict__ blocks, const int32_t* __restrict__ idx_pool, const int64_t* __restrict__ row_ptr,
    const int32_t* __restrict__ col, const double* __restrict__ hval, const double* __restrict__ sval,
    float* __restrict__ hb, double* __restrict__ sb, DevFlags* flags, int pairs, int max_n, int max_ld) {
  extern __shared__ __align__(16) uint8_t g_smem[];
  int32_t* s_idx = reinterpret_cast<int32_t*>(g_smem);
  const BlockDesc bd = blocks[blockIdx.x];
  const int n = bd.n, ld = bd.n_pad;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* wbuf = g_smem + (((size_t)max_n * 4 + 15) & ~(size_t)15) + (size_t)warp * max_ld * 12;
  float* hrow = reinterpret_cast<float*>(wbuf);
  double* srow = reinterpret_cast<double*>(wbuf + (size_t)max_ld * 4);
  float2* srow2 = reinterpret_cast<float2*>(srow);
  for (int i = threadIdx.x; i < n; i += blockDim.x) s_idx[i] = idx_pool[bd.off_idx + i];
  __syncthreads();
  for (int p = warp; p < ld; p += kGatherWarps) {
    for (int c = lane; c < ld; c += 32) {
      hrow[c] = 0.f;
      const bool one = c == p && p >= n;
      if (pairs) srow2[c] = make_float2(one ? 1.f : 0.f, 0.f);
      else srow[c] = one ? 1.0 : 0.0;
    }
    __syncwarp();
    if (p < n) {
      const int32_t r = s_idx[p];
      const int64_t e0 = row_ptr[r], e1 = row_ptr[r + 1];
      // eight entries per lane in flight: their loads are issued before the first lookup
      for (int64_t eb = e0; eb < e1; eb += 8 * 32) {
        int32_t cv[8];
        double hv[8], sv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int64_t e = eb + lane + 32 * u;
          cv[u] = e < e1 ? col[e] : -1;
          hv[u] = e < e1 ? hval[e] : 0.0;
          sv[u] = e < e1 ? sval[e] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (cv[u] < 0) continue;
          const int q = lower_bound_i32(s_idx, n, cv[u]);
          if (q < n && s_idx[q] == cv[u]) {
            if (!isfinite(hv[u]) || !isfinite(sv[u])) set_error(flags, NOLSM_ENONFINITE);
            hrow[q] = (float)hv[u];
            if (pairs) srow2[q] = df_pair_from_f64(sv[u]);
            else srow[q] = sv[u];
          }
        }
      }
    }
    __syncwarp();
    float4* H = reinterpret_cast<float4*>(hb + bd.off_mat + (int64_t)p * ld);
    float4* S = reinterpret_cast<float4*>(sb + bd.off_mat + (int64_t)p * ld);
    for (int c = lane; c < ld / 4; c += 32) H[c] = reinterpret_cast<const float4*>(hrow)[c];
    const int s_end = pairs ? p / 2 + 1 : ld / 2;   // 16-byte units (two entries) of row p written
    for (int c = lane; c < s_end; c += 32) S[c] = reinterpret_cast<const float4*>(srow)[c];
    __syncwarp();
  }
}

// ----------------------------------------------------------------------------------------------
// Warp-tile helper: a warp computes a 32x32 tile acc[r] (lane = output column) of
//   acc[r][lane] = sum_k Arow[r][k] * Bcol[k][lane]
// with both operands streamed through the warp's private shared-memory chunk of 32 k.
template <typename T>
struct WarpChunk {
  T a[32][33];
  T b[32][33];
};

// Cholesky S = L L^T, left-looking by 32-column panels, in place (lower triangle).
// One CTA (8 warps) per block.  For each panel j0:
//   R[r, j0:j0+32] = S[r, j0:j0+32] - L[r, 0:j0] L[j0:j0+32, 0:j0]^T  for rows r >= j0 (warp tiles)
//   factor the 32x32 diagonal of R (warp 0), then L[r, panel] = R[r, panel] L_jj^-T (row solves).
// The strictly upper triangle is zeroed at the end.
template <typename T, int NW>
__global__ void __launch_bounds__(NW * 32) cholesky_kernel(const BlockDesc* __restrict__ blocks, T* __restrict__ pool,
                                                           float* __restrict__ l32, DevFlags* flags) {
  __shared__ WarpChunk<T> chunks[NW];
  __shared__ T diag[32][33];
  __shared__ T rdiag[32];
  __shared__ int s_bad;
  const BlockDesc bd = blocks[blockIdx.x];
  const int n = bd.n, ld = bd.n_pad;
  T* A = pool + bd.off_mat;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpChunk<T>& ch = chunks[warp];
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int jb = min(32, n - j0);
    // --- update panel columns with the previous panels: row tiles of 32 rows, one per warp
    for (int r0 = j0 + warp * 32; r0 < n; r0 += NW * 32) {
      T acc[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) acc[r] = T(0);
      for (int k0 = 0; k0 < j0; k0 += 32) {
        // a: L[r0+r, k0+k] ; b: L[j0+lane, k0+k] stored as b[k][lane]
        for (int r = 0; r < 32; ++r) {
          const int gr = r0 + r;
          ch.a[r][lane] = (gr < n) ? A[(int64_t)gr * ld + k0 + lane] : T(0);
          const int gc = j0 + r;
          ch.b[lane][r] = (gc < n) ? A[(int64_t)gc * ld + k0 + lane] : T(0);
        }
        __syncwarp();
#pragma unroll 4
        for (int k = 0; k < 32; ++k) {
          const T bv = ch.b[k][lane];
#pragma unroll
          for (int r = 0; r < 32; ++r) acc[r] = fma(-ch.a[r][k], bv, acc[r]);
        }
        __syncwarp();
      }
      if (lane < jb) {
        for (int r = 0; r < 32; ++r) {
          const int gr = r0 + r;
          if (gr < n) A[(int64_t)gr * ld + j0 + lane] += acc[r];
        }
      }
    }
    __syncthreads();
    // --- factor the diagonal 32x32 block (warp 0, lane = row); keep 1 / L_kk for the panel solve
    if (warp == 0) {
      for (int r = 0; r < 32; ++r) diag[r][lane] = (r < jb && lane < jb) ? A[(int64_t)(j0 + r) * ld + j0 + lane] : T(r == lane);
      __syncwarp();
      for (int k = 0; k < 32; ++k) {
        if (lane == k) {
          T d = diag[k][k];
          if (!(d > T(0))) { s_bad = 1; d = T(1); }
          const T s = sqrt(d);
          diag[k][k] = s;
          rdiag[k] = T(1) / s;
        }
        __syncwarp();
        if (lane > k) diag[lane][k] *= rdiag[k];
        __syncwarp();
        if (lane > k) {
          const T lk = diag[lane][k];
          for (int j = k + 1; j <= lane; ++j) diag[lane][j] -= lk * diag[j][k];
        }
        __syncwarp();
      }
      for (int r = 0; r < jb; ++r)
        if (lane <= r) A[(int64_t)(j0 + r) * ld + j0 + lane] = diag[r][lane];
    }
    __syncthreads();
    // --- panel rows below: x L_jj^T = r by forward substitution, one warp per 32-row tile held in
    //     shared memory (lane = row), multiplying by the reciprocals instead of dividing
    for (int r0 = j0 + jb + warp * 32; r0 < n; r0 += NW * 32) {
      for (int r = 0; r < 32; ++r) {
        const int gr = r0 + r;
        ch.a[r][lane] = (gr < n && lane < jb) ? A[(int64_t)gr * ld + j0 + lane] : T(0);
      }
      __syncwarp();
      for (int k = 0; k < jb; ++k) {
        T v = ch.a[lane][k];
        for (int q = 0; q < k; ++q) v = fma(-ch.a[lane][q], diag[k][q], v);
        ch.a[lane][k] = v * rdiag[k];
      }
      __syncwarp();
      for (int r = 0; r < 32; ++r) {
        const int gr = r0 + r;
        if (gr < n && lane < jb) A[(int64_t)gr * ld + j0 + lane] = ch.a[r][lane];
      }
      __syncwarp();
    }
    __syncthreads();
  }
  // Only the lower triangle of A is the factor (the strict upper part still holds S).  With
  // l32 given, the factor is also written there in FP32, zero above the diagonal and on the
  // padding.
  if (l32) {
    float* Lf = l32 + bd.off_mat;
    for (int r = warp; r < ld; r += NW)
      for (int c = lane; c < ld; c += 32)
        Lf[(int64_t)r * ld + c] = (r < n && c <= r) ? (float)A[(int64_t)r * ld + c] : 0.f;
  }
  if (threadIdx.x == 0 && s_bad) set_error(flags, NOLSM_ENOTPD);
}

// ----------------------------------------------------------------------------------------------
// Double-float arithmetic (Dekker 1971, "A floating-point technique for extending the available
// precision"): a value is the unevaluated sum h + l of two FP32 numbers with |l| <= ulp(h)/2, a
// 48-bit significand.  Products use the exact FMA split p + e = a*b (TwoProd); sums use Knuth's
// branch-free TwoSum.  The multiply-accumulate below drops a.l*b.l and the rounding of the low
// word, so k terms carry an error of order k * 2^-48 times the sum of |terms| -- the FP64
// bound with 2^-48 in place of 2^-53.  On this GPU the FP32 pipe issues ~58 times the FP64 pipe's
// multiply-adds, so one pair update (12 FP32 instructions) is ~5 times cheaper than one DFMA.
struct __align__(8) df32 {
  float h, l;
};

__device__ __forceinline__ double df_to_double(df32 a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ df32 df_from_double(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
// TwoSum renormalisation: h = fl(h + l), l = the exact remainder.
__device__ __forceinline__ df32 df_norm(df32 a) {
  const float s = a.h + a.l;
  const float bb = s - a.h;
  return {s, (a.h - (s - bb)) + (a.l - bb)};
}
// acc += a * b
__device__ __forceinline__ void df_fma(df32& acc, df32 a, df32 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const float s = acc.h + p;
  const float bb = s - acc.h;
  const float err = (acc.h - (s - bb)) + (p - bb);
  acc.h = s;
  acc.l += err + e;
}
__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  const float err = (a.h - (s - bb)) + (b.h - bb);
  return df_norm({s, err + a.l + b.l});
}
__device__ __forceinline__ df32 df_neg(df32 a) { return {-a.h, -a.l}; }

// acc -= a * b
__device__ __forceinline__ void df_fms(df32& acc, df32 a, df32 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const float s = acc.h - p;
  const float bb = s - acc.h;
  const float err = (acc.h - (s - bb)) - (p + bb);
  acc.h = s;
  acc.l += err - e;
}

// a * b, renormalised (the low-by-low product is below the pair's precision)
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return df_norm({p, e});
}
// sqrt(a) for a > 0: the FP32 root s plus one Newton correction (a - s^2) / (2 s), s^2 exact by FMA
__device__ __forceinline__ df32 df_sqrt(df32 a) {
  const float s = sqrtf(a.h);
  const float r = fmaf(-s, s, a.h) + a.l;
  return df_norm({s, r / (2.f * s)});
}
// 1 / a: the FP32 reciprocal r plus one Newton correction r (1 - a r), the residual in pairs
__device__ __forceinline__ df32 df_recip(df32 a) {
  const float r = 1.f / a.h;
  const float e = fmaf(-a.h, r, 1.f) - a.l * r;
  return df_norm({r, r * e});
}

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Cholesky S = L L^T in double-float, left-looking by 32-column panels, in place over the pool of
// pairs the gather wrote (a pair occupies the 8 bytes of a double).  One CTA of 4 warps per block;
// every 32-row tile is shared by the 4 warps, each taking 8 of every 32 k (no idle warps when a
// panel has few tiles), the four partial tiles summed in shared memory.  One launch covers the
// columns [c_beg, c_end): the whole factor (0, n), or one panel of the blocked factorization whose
// trailing updates run on the tensor cores (the columns before c_beg are then already subtracted
// from the panel, so the left-looking sums start at c_beg).
//   0. (c_beg = 0, scale_exp given) each row's slicing exponent e_r (2^e_r >= sqrt(S_rr) >= |L_rk|);
//   for each 32-column panel j0 in [c_beg, c_end):
//   1. R[r, panel] = S[r, panel] - L[r, 0:j0] L[panel, 0:j0]^T for rows r >= j0: 32 x 32 operand
//      chunks double-buffered in shared memory with cp.async;
//   2. warp 0 factors the 32x32 diagonal block of R in FP64 and inverts it (FP64), keeping
//      L_jj^-T as pairs;
//   3. L[r, panel] = R[r, panel] L_jj^-T for the rows below (same split over k).
//   4. (c_end >= n) with l32 given, the factor's FP32 rounding is written there (zero above the
//      diagonal and on the padding); the pool keeps the pairs.
// The diagonal blocks are O(n 32^2) of the O(n^3/6) work, so FP64 there costs little.
constexpr int kCholWarps = 4;

__global__ void __launch_bounds__(kCholWarps * 32, 3) cholesky_df_kernel(const BlockDesc* __restrict__ blocks,
                                                                         double* __restrict__ pool,
                                                                         float* __restrict__ l32, DevFlags* flags,
                                                                         int c_beg, int c_end,
                                                                         int32_t* __restrict__ scale_exp, int r_end,
                                                                         float2* __restrict__ wout) {
  __shared__ df32 As[2][32][32];          // read as broadcasts: no padding
  __shared__ df32 Bs[2][32][33];          // read by rows (lane = row): padded
  __shared__ df32 red[kCholWarps][32][32];
  __shared__ df32 binv[32][32];
  __shared__ df32 rd[32];
  __shared__ int s_bad;
  const BlockDesc bd = blocks[blockIdx.x];
  const int n = bd.n, ld = bd.n_pad;
  if (c_beg >= n) return;
  const int rmax = min(n, r_end);   // rows this launch factors (the panel's diagonal block in the blocked mode)
  float2* A = reinterpret_cast<float2*>(pool + bd.off_mat);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // phase-2 scratch over the reduction buffers (idle then)
  df32(*dg)[33] = reinterpret_cast<df32(*)[33]>(&red[0][0][0]);
  df32(*dinv)[33] = reinterpret_cast<df32(*)[33]>(&red[0][0][0] + 32 * 33);
  if (tid == 0) s_bad = 0;
  if (c_beg == 0 && scale_exp) {
    // 2^e_r >= sqrt(S_rr), which bounds every |L_rk| (sum_k L_rk^2 = S_rr); padding rows get 0
    for (int r = tid; r < ld; r += kCholWarps * 32) {
      int e = 0;
      if (r < n) {
        const float2 d = A[(int64_t)r * ld + r];
        frexp(sqrt(fmax((double)d.x + (double)d.y, 1e-300)), &e);
      }
      scale_exp[bd.row_off + r] = e;
    }
  }
  __syncthreads();
  // rows [row0, row0 + 32) x columns [col0, col0 + 32) of the pair matrix into a 32x32 chunk
  auto load_chunk = [&](auto dst, int row0, int col0) {
#pragma unroll
    for (int i = 0; i < 1024 / (kCholWarps * 32); ++i) {
      const int e = tid + i * kCholWarps * 32;
      const int r = e >> 5, c = e & 31;
      if (row0 + r < n) cp_async8(&dst[r][c], A + (int64_t)(row0 + r) * ld + col0 + c);
      else dst[r][c] = {0.f, 0.f};
    }
  };
  // the four warps' partial tiles (in red) summed and stored as pairs at rows r0.., columns j0..
  // (lower triangle and c < jb only)
  auto reduce_store = [&](int r0, int j0, int jb) {
    __syncthreads();
    for (int e = tid; e < 1024; e += kCholWarps * 32) {
      const int r = e >> 5, c = e & 31;
      const int gr = r0 + r;
      if (gr < n && c < jb && j0 + c <= gr) {
        df32 v = red[0][r][c];
#pragma unroll
        for (int w = 1; w < kCholWarps; ++w) v = df_add(v, red[w][r][c]);
        v = df_norm(v);
        A[(int64_t)gr * ld + j0 + c] = make_float2(v.h, v.l);
      }
    }
    __syncthreads();
  };
  const int kw = warp * (32 / kCholWarps);   // this warp's 8 k of every chunk
  for (int j0 = c_beg; j0 < min(n, c_end); j0 += 32) {
    const int jb = min(32, n - j0);
    // 1. panel update over the columns [c_beg, j0) (nothing to subtract for the first panel)
    const int nch = (j0 - c_beg) / 32;
    if (nch == 1) {
      // one 32-wide chunk (the second half of a 64-column panel): whole tiles per warp, no split
      // over k.  B = L[panel rows, c_beg..] is shared (Bs[0], lane = row); each warp stages its A
      // rows in its own quarter of `red`.
      for (int e = tid; e < 1024; e += kCholWarps * 32) {
        const int r = e >> 5, c = e & 31;
        const float2 v = (j0 + r < n) ? A[(int64_t)(j0 + r) * ld + c_beg + c] : make_float2(0.f, 0.f);
        Bs[0][r][c] = {v.x, v.y};
      }
      __syncthreads();
      df32(*Aw)[32] = red[warp];
      for (int r0 = j0 + 32 * warp; r0 < rmax; r0 += 32 * kCholWarps) {
        df32 acc[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const bool in = r0 + r < n;
          const float2 a = in ? A[(int64_t)(r0 + r) * ld + c_beg + lane] : make_float2(0.f, 0.f);
          const float2 s0 = (in && lane < jb && j0 + lane <= r0 + r) ? A[(int64_t)(r0 + r) * ld + j0 + lane]
                                                                     : make_float2(0.f, 0.f);
          Aw[r][lane] = {a.x, a.y};
          acc[r] = {s0.x, s0.y};
        }
        __syncwarp();
#pragma unroll 2
        for (int k = 0; k < 32; ++k) {
          const df32 bv = Bs[0][lane][k];
#pragma unroll
          for (int r = 0; r < 32; ++r) df_fms(acc[r], Aw[r][k], bv);
        }
#pragma unroll
        for (int r = 0; r < 32; ++r)
          if (r0 + r < n && lane < jb && j0 + lane <= r0 + r) {
            const df32 v = df_norm(acc[r]);
            A[(int64_t)(r0 + r) * ld + j0 + lane] = make_float2(v.h, v.l);
          }
        __syncwarp();
      }
      __syncthreads();
    } else if (nch > 1) {
      for (int r0 = j0; r0 < rmax; r0 += 32) {
        // warp 0 starts from S itself (its loads overlap the first chunk's copies), the others from 0
        df32 acc[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          acc[r] = {0.f, 0.f};
          if (warp == 0 && r0 + r < n && lane < jb && j0 + lane <= r0 + r) {
            const float2 s0 = A[(int64_t)(r0 + r) * ld + j0 + lane];
            acc[r] = {s0.x, s0.y};
          }
        }
        load_chunk(As[0], r0, c_beg);
        load_chunk(Bs[0], j0, c_beg);
        cp_async_commit();
        for (int c = 0; c < nch; ++c) {
          const int buf = c & 1;
          if (c + 1 < nch) {
            load_chunk(As[buf ^ 1], r0, c_beg + (c + 1) * 32);
            load_chunk(Bs[buf ^ 1], j0, c_beg + (c + 1) * 32);
            cp_async_commit();
            cp_async_wait_group<1>();
          } else {
            cp_async_wait_group<0>();
          }
          __syncthreads();
#pragma unroll 2
          for (int kk = 0; kk < 32 / kCholWarps; ++kk) {
            const df32 bv = Bs[buf][lane][kw + kk];
#pragma unroll
            for (int r = 0; r < 32; ++r) df_fms(acc[r], As[buf][r][kw + kk], bv);
          }
          __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < 32; ++r) red[warp][r][lane] = acc[r];
        reduce_store(r0, j0, jb);
      }
    }
    // 2. diagonal block (warp 0, lane = row) in pairs, then its inverse (lane = column): the FP64 pipe
    //    of this GPU issues at 1/64 of the FP32 rate, so the pivots run in double-float too
    if (warp == 0) {
      for (int r = 0; r < 32; ++r) {
        df32 v = {(r == lane) ? 1.f : 0.f, 0.f};
        if (r < jb && lane < jb && lane <= r) {
          const float2 s = A[(int64_t)(j0 + r) * ld + j0 + lane];
          v = {s.x, s.y};
        }
        dg[r][lane] = v;
      }
      __syncwarp();
      for (int k = 0; k < 32; ++k) {
        if (lane == k) {
          df32 d = dg[k][k];
          if (!(d.h > 0.f)) { s_bad = 1; d = {1.f, 0.f}; }
          const df32 s = df_sqrt(d);
          dg[k][k] = s;
          rd[k] = df_recip(s);
        }
        __syncwarp();
        if (lane > k) dg[lane][k] = df_mul(dg[lane][k], rd[k]);
        __syncwarp();
        if (lane > k) {
          const df32 lk = dg[lane][k];
          for (int j = k + 1; j <= lane; ++j) df_fms(dg[lane][j], lk, dg[j][k]);
        }
        __syncwarp();
      }
      // column `lane` of L_jj^-1 by forward substitution (zero above the diagonal); the sum over q
      // runs as four independent chains
      for (int r = 0; r < 32; ++r) {
        df32 v = {(r == lane) ? 1.f : 0.f, 0.f};
        if (r > lane) {
          df32 part[4] = {v, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
          int q = lane;
          for (; q + 3 < r; q += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) df_fms(part[u], dg[r][q + u], dinv[q + u][lane]);
          }
          for (; q < r; ++q) df_fms(part[0], dg[r][q], dinv[q][lane]);
          v = df_add(df_add(part[0], part[1]), df_add(part[2], part[3]));
        }
        dinv[r][lane] = (r >= lane) ? df_mul(v, rd[r]) : df32{0.f, 0.f};
      }
      for (int r = 0; r < jb; ++r)
        if (lane <= r) {
          const df32 v = df_norm(dg[r][lane]);
          A[(int64_t)(j0 + r) * ld + j0 + lane] = make_float2(v.h, v.l);
        }
      __syncwarp();
      for (int k = 0; k < 32; ++k) binv[k][lane] = dinv[lane][k];
      if (wout && j0 == c_beg)   // L_aa^-T of the panel's first half, kept for W
        for (int k = 0; k < 32; ++k) As[0][k][lane] = binv[k][lane];
    }
    __syncthreads();
    // 3. rows below the diagonal block: L[r, panel] = R[r, panel] L_jj^-T, whole 32-row tiles per
    //    warp (A rows staged in the warp's quarter of `red`; binv shared)
    {
      df32(*Aw)[32] = red[warp];
      for (int r0 = j0 + jb + 32 * warp; r0 < rmax; r0 += 32 * kCholWarps) {
        df32 acc[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          // columns j0 + jb.. of these rows lie past the panel: zero weights below
          const float2 a = (r0 + r < n) ? A[(int64_t)(r0 + r) * ld + j0 + lane] : make_float2(0.f, 0.f);
          Aw[r][lane] = {a.x, a.y};
          acc[r] = {0.f, 0.f};
        }
        __syncwarp();
#pragma unroll 2
        for (int k = 0; k < 32; ++k) {
          const df32 bv = binv[k][lane];
#pragma unroll
          for (int r = 0; r < 32; ++r) df_fma(acc[r], Aw[r][k], bv);
        }
#pragma unroll
        for (int r = 0; r < 32; ++r)
          if (r0 + r < n && lane < jb) {
            const df32 v = df_norm(acc[r]);
            A[(int64_t)(r0 + r) * ld + j0 + lane] = make_float2(v.h, v.l);
          }
        __syncwarp();
      }
      __syncthreads();
    }
  }
  if (wout && c_end - c_beg == 64 && n > c_beg + 64) {
    // W = L11^-T of the 64 x 64 diagonal block [[L_aa, 0], [L_ba, L_cc]] for the rows below:
    // L11^-1 = [[L_aa^-1, 0], [X, L_cc^-1]] with X = -L_cc^-1 L_ba L_aa^-1.  As[0] holds L_aa^-T,
    // binv L_cc^-T (both as pairs); T = L_ba L_aa^-1 goes to red[1], X to red[2].
    df32(*Lba)[32] = red[0];
    df32(*T)[32] = red[1];
    df32(*X)[32] = red[2];
    for (int e = tid; e < 1024; e += kCholWarps * 32) {
      const int r = e >> 5, c = e & 31;
      const float2 v = A[(int64_t)(c_beg + 32 + r) * ld + c_beg + c];
      Lba[r][c] = {v.x, v.y};
    }
    __syncthreads();
    for (int i = warp * 8; i < warp * 8 + 8; ++i) {     // T[i][lane] = sum_k L_ba[i][k] (L_aa^-1)[k][lane]
      df32 acc = {0.f, 0.f};
      for (int k = 0; k < 32; ++k) df_fma(acc, Lba[i][k], As[0][lane][k]);
      T[i][lane] = df_norm(acc);
    }
    __syncthreads();
    for (int i = warp * 8; i < warp * 8 + 8; ++i) {     // X[i][lane] = -sum_k (L_cc^-1)[i][k] T[k][lane]
      df32 acc = {0.f, 0.f};
      for (int k = 0; k < 32; ++k) df_fms(acc, binv[k][i], T[k][lane]);
      X[i][lane] = df_norm(acc);
    }
    __syncthreads();
    float2* W = wout + (int64_t)blockIdx.x * 4096;      // W[k][c], k, c < 64
    for (int e = tid; e < 4096; e += kCholWarps * 32) {
      const int k = e >> 6, c = e & 63;
      df32 v = {0.f, 0.f};
      if (k < 32 && c < 32) v = As[0][k][c];
      else if (k >= 32 && c >= 32) v = binv[k - 32][c - 32];
      else if (k < 32) v = X[c - 32][k];
      W[e] = make_float2(v.h, v.l);
    }
  }
  if (c_end < n) {
    if (threadIdx.x == 0 && s_bad) set_error(flags, NOLSM_ENOTPD);
    return;
  }
  // 4. the FP32 copy of the factor: fl(h + l) is the pair's value rounded to nearest (zero above
  //    the diagonal and on the padding); four independent loads at a time
  __syncthreads();
  if (l32) {
    float* Lf = l32 + bd.off_mat;
    for (int r = warp; r < ld; r += kCholWarps)
      for (int c0 = 0; c0 < ld; c0 += 128) {
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = c0 + 32 * u + lane;
          v[u] = (r < n && c <= r) ? A[(int64_t)r * ld + c] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) Lf[(int64_t)r * ld + c0 + 32 * u + lane] = v[u].x + v[u].y;
      }
  }
  if (tid == 0 && s_bad) set_error(flags, NOLSM_ENOTPD);
}

// ---- the 64 x 64 diagonal block of the blocked double-float Cholesky ----------------------------
// The CTA (kDiagWarps warps) factors a 32 x 32 SPD block in shared memory, P = L L^T in place (lower
// triangle), and writes X = L^-1 (lower triangle, zero above).  Right-looking in both, one barrier
// per column: every thread forms the pivot and its reciprocal itself, an update scales the column
// entries it needs on the fly, and the scaled column is written back one column later (when no
// thread reads it any more), so every entry takes the same operations as with a scaled column
// written first.  rk receives the reciprocal pivots.  Sets *bad when a pivot is not positive (it is
// then taken as 1).
constexpr int kDiagWarps = 8;
constexpr int kDiagThreads = 32 * kDiagWarps;
constexpr int kDiagRows = 32 / kDiagWarps;       // rows of a 32 x 32 product per warp
__device__ __forceinline__ void pivot32(df32 (*P)[65], df32 (*X)[33], df32* rk, int* bad) {
  // lane = column, warp w takes the rows w, w + kDiagWarps, ...: no index arithmetic beyond the loops, and
  // a lane's scaled column entry is formed once per step
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < 32; ++k) {
    df32 d = P[k][k];
    if (!(d.h > 0.f)) {
      if (tid == 0) *bad = 1;
      d = {1.f, 0.f};
    }
    const df32 sq = df_sqrt(d);
    const df32 r = df_recip(sq);
    // lane c forms the scaled entry of row c once; row i's entry reaches the other lanes by shuffles
    // (the same value each lane would form itself)
    const df32 b = df_mul(P[lane][k], r);
    const df32 own = (tid > k && tid < 32) ? b : df32{0.f, 0.f};
    for (int i = k + 1 + warp; i < 32; i += kDiagWarps) {
      const df32 bi = {__shfl_sync(0xffffffffu, b.h, i), __shfl_sync(0xffffffffu, b.l, i)};
      if (lane > k && lane <= i) df_fms(P[i][lane], bi, b);
    }
    __syncthreads();                            // column k read by every thread; P[k+1][k+1] final
    if (tid == 0) {
      P[k][k] = sq;
      rk[k] = r;
    }
    if (tid > k && tid < 32) P[tid][k] = own;
  }
  for (int e = tid; e < 1024; e += kDiagThreads) X[e >> 5][e & 31] = {((e >> 5) == (e & 31)) ? 1.f : 0.f, 0.f};
  __syncthreads();
  for (int q = 0; q < 32; ++q) {
    // row q of X is final once scaled: X[q][c] = (delta_qc - sum_{p<q} L[q][p] X[p][c]) / L[q][q];
    // the updates below scale it on the fly, thread c stores it after the barrier
    const df32 own = (tid <= q) ? df_mul(X[q][tid], rk[q]) : df32{0.f, 0.f};
    if (lane <= q) {                            // X[r][c] -= L[r][q] X[q][c] for r > q, c <= q
      const df32 xq = df_mul(X[q][lane], rk[q]);
      for (int rr = q + 1 + warp; rr < 32; rr += kDiagWarps) df_fms(X[rr][lane], P[rr][q], xq);
    }
    __syncthreads();
    if (tid <= q) X[q][tid] = own;
  }
  __syncthreads();
}

// The 64 x 64 diagonal block [c0, c0 + 64) of a panel, whose earlier panels' contributions are
// already subtracted: L11 in place (pairs) and, when rows follow below, Minv = L11^-1 for the TRSM of
// the rows below (chol_trsm_tc_kernel) as kOzSlices BF16 slice planes, row c on the scale 2^f_c >=
// max_k |Minv[c, k]|, with f_0 .. f_63 and g = max_k e_k over the panel's rows in mout_f.  The CTA
// runs the two 32 x 32 pivots (pivot32) and shares the 32 x 32 x 32 products between its warps:
//   L_ba = A_ba L_aa^-T,  A_cc -= L_ba L_ba^T,  T = L_ba L_aa^-1,  X = -L_cc^-1 T,
// so that L11^-1 = [[L_aa^-1, 0], [X, L_cc^-1]].  Entries past n are taken as the identity.  In the
// first panel each row's slicing exponent e_r (2^e_r >= sqrt(S_rr)) is written first.
__global__ void __launch_bounds__(kDiagThreads, 4) chol_diag64_kernel(const BlockDesc* __restrict__ blocks,
                                                             double* __restrict__ pool, DevFlags* flags, int c0,
                                                             int32_t* __restrict__ scale_exp,
                                                             uint16_t* __restrict__ mout,
                                                             int32_t* __restrict__ mout_f,
                                                             float* __restrict__ l32,
                                                             float* __restrict__ x32) {
  // the block (lower triangle); its unused upper-right 32 x 32 quarter holds the temporary T, and
  // once L11 is written out its lower-left quarter receives X (four CTAs per SM fit)
  __shared__ df32 M[64][65];
  __shared__ df32 Xa[32][33], Xc[32][33];
  __shared__ df32 rk[32];
  __shared__ int fexp[64];
  __shared__ int s_bad;
  const BlockDesc bd = blocks[blockIdx.x];
  const int n = bd.n, ld = bd.n_pad;
  if (c0 >= n) return;
  float2* A = reinterpret_cast<float2*>(pool + bd.off_mat);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nb = min(64, n - c0);
  if (tid == 0) s_bad = 0;
  if (c0 == 0 && scale_exp)
    for (int r = tid; r < ld; r += kDiagThreads) {
      int e = 0;
      if (r < n) {
        const float2 d = A[(int64_t)r * ld + r];
        frexp(sqrt(fmax((double)d.x + (double)d.y, 1e-300)), &e);
      }
      scale_exp[bd.row_off + r] = e;
    }
  for (int e = tid; e < 64 * 64; e += kDiagThreads) {
    const int r = e >> 6, c = e & 63;
    df32 v = {(r == c) ? 1.f : 0.f, 0.f};
    if (r < nb && c <= r) {
      const float2 s = A[(int64_t)(c0 + r) * ld + c0 + c];
      v = {s.x, s.y};
    }
    M[r][c] = v;
  }
  __syncthreads();
  pivot32(M, Xa, rk, &s_bad);
  // The 32 x 32 x 32 products below take two rows per pass: two independent double-float chains per
  // thread (every sum keeps its own order).
  // L_ba[i][j] = sum_{k <= j} A_ba[i][k] (L_aa^-1)[j][k]
  for (int i = warp * kDiagRows; i < warp * kDiagRows + kDiagRows; i += 2) {
    df32 acc0 = {0.f, 0.f}, acc1 = {0.f, 0.f};
    for (int k = 0; k <= lane; ++k) {
      const df32 x = Xa[lane][k];
      df_fma(acc0, M[32 + i][k], x);
      df_fma(acc1, M[33 + i][k], x);
    }
    M[i][32 + lane] = df_norm(acc0);
    M[i + 1][32 + lane] = df_norm(acc1);
  }
  __syncthreads();
  for (int i = warp * kDiagRows; i < warp * kDiagRows + kDiagRows; ++i) M[32 + i][lane] = M[i][32 + lane];
  __syncthreads();
  // A_cc[i][j] -= sum_k L_ba[i][k] L_ba[j][k]   (j <= i)
  for (int i = warp * kDiagRows; i < warp * kDiagRows + kDiagRows; i += 2) {
    if (lane > i + 1) continue;
    const bool both = lane <= i;
    df32 acc0 = both ? M[32 + i][32 + lane] : df32{0.f, 0.f};
    df32 acc1 = M[33 + i][32 + lane];
    for (int k = 0; k < 32; ++k) {
      const df32 y = M[32 + lane][k];
      if (both) df_fms(acc0, M[32 + i][k], y);
      df_fms(acc1, M[33 + i][k], y);
    }
    if (both) M[32 + i][32 + lane] = df_norm(acc0);
    M[33 + i][32 + lane] = df_norm(acc1);
  }
  __syncthreads();
  pivot32(reinterpret_cast<df32(*)[65]>(&M[32][32]), Xc, rk, &s_bad);
  for (int e = tid; e < 64 * 64; e += kDiagThreads) {
    const int r = e >> 6, c = e & 63;
    if (r < nb && c <= r) {
      const int64_t o = (int64_t)(c0 + r) * ld + c0 + c;
      A[o] = make_float2(M[r][c].h, M[r][c].l);
      if (l32) l32[bd.off_mat + o] = M[r][c].h + M[r][c].l;   // the factor's FP32 rounding fl(h + l)
    }
  }
  // the FP32 factor's padding rows are read as operands (times zeros of the inverse): zero them once,
  // in the block's last panel; its strict upper triangle is never read
  if (l32 && n <= c0 + 64)
    for (int64_t e = tid; e < (int64_t)(ld - n) * ld; e += kDiagThreads) l32[bd.off_mat + (int64_t)n * ld + e] = 0.f;
  const bool want_m = mout && n > c0 + 64;
  if (want_m || x32) {
    // T = L_ba L_aa^-1, X = -L_cc^-1 T (two rows per pass; row i's X sum stops at k = i, since
    // L_cc^-1 is lower triangular)
    for (int i = warp * kDiagRows; i < warp * kDiagRows + kDiagRows; i += 2) {
      df32 acc0 = {0.f, 0.f}, acc1 = {0.f, 0.f};
      for (int k = lane; k < 32; ++k) {
        const df32 x = Xa[k][lane];
        df_fma(acc0, M[32 + i][k], x);
        df_fma(acc1, M[33 + i][k], x);
      }
      M[i][32 + lane] = df_norm(acc0);           // T
      M[i + 1][32 + lane] = df_norm(acc1);
    }
    __syncthreads();                             // T complete, L_ba (and L11's write-out) read
    for (int i = warp * kDiagRows; i < warp * kDiagRows + kDiagRows; i += 2) {
      df32 acc0 = {0.f, 0.f}, acc1 = {0.f, 0.f};
      for (int k = 0; k <= i; ++k) {
        const df32 t = M[k][32 + lane];
        df_fms(acc0, Xc[i][k], t);
        df_fms(acc1, Xc[i + 1][k], t);
      }
      df_fms(acc1, Xc[i + 1][i + 1], M[i + 1][32 + lane]);
      M[32 + i][lane] = df_norm(acc0);           // X
      M[33 + i][lane] = df_norm(acc1);
    }
    __syncthreads();
  }
  // Minv[c][k] = (L11^-1)[c][k]: lower triangular
  auto minv = [&](int c, int k) -> df32 {
    if (k < 32 && c < 32) return Xa[c][k];
    if (k >= 32 && c >= 32) return Xc[c - 32][k - 32];
    if (k < 32) return M[c][k];                  // X
    return df32{0.f, 0.f};
  };
  if (x32) {
    // the FP32 rounding of L11^-1 as the diagonal 64 x 64 block of the mixed paths' L^-1 (zero above
    // the diagonal and on the padding rows)
    float* Xo = x32 + bd.off_mat + (int64_t)c0 * ld + c0;
    for (int e = tid; e < 4096; e += kDiagThreads) {
      const int r = e >> 6, c = e & 63;
      float v = 0.f;
      if (r < nb && c <= r) {
        const df32 m = minv(r, c);
        v = m.h + m.l;
      }
      Xo[(int64_t)r * ld + c] = v;
    }
  }
  if (want_m) {
    int32_t* F = mout_f + (int64_t)blockIdx.x * 68;
    if (tid < 64) {
      float mx = 0.f;
      for (int k = 0; k <= tid; ++k) mx = fmaxf(mx, fabsf(minv(tid, k).h));
      int e = 0;
      frexpf(mx > 0.f ? mx : 1.f, &e);     // 2^e > max |h|, so 2^e >= max |h + l|
      fexp[tid] = e;
      F[tid] = e;
    } else if (tid == 64) {
      int g = -1000;
      for (int k = 0; k < 64; ++k) g = max(g, scale_exp[bd.row_off + c0 + k]);
      F[64] = g;
    }
    __syncthreads();
    uint16_t* P = mout + (int64_t)blockIdx.x * kOzSlices * 4096;   // plane s: 64 rows c x 64 columns k
    for (int e = tid; e < 4096; e += kDiagThreads) {
      const int c = e >> 6, k = e & 63;
      const df32 v = minv(c, k);
      float q[kOzSlices];
      oz_slices(v.h, v.l, oz_scale(fexp[c]), q);
#pragma unroll
      for (int sl = 0; sl < kOzSlices; ++sl) {
        const __nv_bfloat16 b = __float2bfloat16_rn(q[sl]);
        P[sl * 4096 + e] = *reinterpret_cast<const uint16_t*>(&b);
      }
    }
  }
  if (tid == 0 && s_bad) set_error(flags, NOLSM_ENOTPD);
}

// Inverse of the lower-triangular L into X (out of place), by block rows of 32:
//   X[i-block, c-block] = -L_ii^-1 sum_{k=c}^{i-1} L_ik X_kc   (c < i),   X_ii = L_ii^-1.
// Phase 1 forms R = sum_k L_ik X_kc with warp tiles (one 32x32 tile per c-block), phase 2
// solves L_ii Y = (E - R) column by column (thread per column).
template <typename T, int NW>
__global__ void __launch_bounds__(NW * 32) trinv_kernel(const BlockDesc* __restrict__ blocks,
                                                        const T* __restrict__ lpool, T* __restrict__ xpool) {
  __shared__ WarpChunk<T> chunks[NW];
  __shared__ T lii[32][33];
  __shared__ T rli[32];
  const BlockDesc bd = blocks[blockIdx.x];
  const int n = bd.n, ld = bd.n_pad;
  const T* L = lpool + bd.off_mat;
  T* X = xpool + bd.off_mat;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpChunk<T>& ch = chunks[warp];
  // the output's upper triangle and padding stay zero
  for (int r = warp; r < ld; r += NW)
    for (int c = lane; c < ld; c += 32) X[(int64_t)r * ld + c] = T(0);
  __syncthreads();
  const int nbk = (n + 31) / 32;
  for (int ib = 0; ib < nbk; ++ib) {
    const int i0 = ib * 32, ibw = min(32, n - i0);
    // phase 1: R for every c-block < ib, written into X's block row (as -R) for phase 2
    for (int cb = warp; cb < ib; cb += NW) {
      const int c0 = cb * 32;
      T acc[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) acc[r] = T(0);
      for (int k0 = c0; k0 < i0; k0 += 32) {
        for (int r = 0; r < 32; ++r) {
          ch.a[r][lane] = (r < ibw) ? L[(int64_t)(i0 + r) * ld + k0 + lane] : T(0);
          ch.b[r][lane] = X[(int64_t)(k0 + r) * ld + c0 + lane];   // b[k][col]
        }
        __syncwarp();
#pragma unroll 4
        for (int k = 0; k < 32; ++k) {
          const T bv = ch.b[k][lane];
#pragma unroll
          for (int r = 0; r < 32; ++r) acc[r] = fma(ch.a[r][k], bv, acc[r]);
        }
        __syncwarp();
      }
      for (int r = 0; r < ibw; ++r) X[(int64_t)(i0 + r) * ld + c0 + lane] = -acc[r];
    }
    if (threadIdx.x < 32) {
      for (int r = 0; r < 32; ++r)
        lii[r][threadIdx.x] = (r < ibw && (int)threadIdx.x < ibw) ? L[(int64_t)(i0 + r) * ld + i0 + threadIdx.x]
                                                                  : T(r == (int)threadIdx.x);
      rli[threadIdx.x] = T(1) / ((threadIdx.x < (unsigned)ibw) ? L[(int64_t)(i0 + threadIdx.x) * ld + i0 + threadIdx.x]
                                                                : T(1));
    }
    __syncthreads();
    // phase 2: for every column j of the block row, L_ii y = rhs with rhs = -R (c < i) or e_j
    // (diagonal block); one warp per 32 columns held in shared memory (lane = column)
    const int ncols = i0 + ibw;
    for (int jc = warp * 32; jc < ncols; jc += NW * 32) {
      const int j = jc + lane;
      for (int r = 0; r < 32; ++r) {
        T v = T(0);
        if (j < ncols && r < ibw) v = (j >= i0) ? T((i0 + r) == j) : X[(int64_t)(i0 + r) * ld + j];
        ch.a[r][lane] = v;
      }
      __syncwarp();
      for (int r = 0; r < ibw; ++r) {
        T v = ch.a[r][lane];
        for (int q = 0; q < r; ++q) v = fma(-lii[r][q], ch.a[q][lane], v);
        ch.a[r][lane] = v * rli[r];
      }
      __syncwarp();
      if (j < ncols)
        for (int r = 0; r < ibw; ++r) X[(int64_t)(i0 + r) * ld + j] = ch.a[r][lane];
      __syncwarp();
    }
    __syncthreads();
  }
}

// L^-1 in FP32 by block rows of 32, one CTA of four warps per block:
//   X_ii = L_ii^-1 (32 x 32, one warp, column-parallel forward substitution with reciprocals),
//   X_ic = -X_ii R_ic,  R_ic = sum_{k=c}^{i-1} L_ik X_kc  for every column block c < i.
// Each 32 x 32 product R_ic is shared by the four warps over k (8 of every 32; no warp idles when
// a block row has few column blocks), operand chunks double-buffered in shared memory with cp.async,
// the four partial tiles summed in shared memory (which also makes the k-sum two-level).
constexpr int kInvWarps = 4;
static_assert(32 / kInvWarps == 8, "the product loop of trinv_tile_kernel takes 8 values of k per warp");

__device__ __forceinline__ void cp_async16_b(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}

__global__ void __launch_bounds__(kInvWarps * 32, 4) trinv_tile_kernel(const BlockDesc* __restrict__ blocks,
                                                                       const float* __restrict__ lpool,
                                                                       float* __restrict__ xpool) {
  __shared__ __align__(16) float As[2][32][32];   // L_ik chunk, read as broadcasts
  __shared__ __align__(16) float Bs[2][32][32];   // X_kc chunk, row k contiguous
  __shared__ float red[kInvWarps][32][32];
  __shared__ float Xi[32][33];
  __shared__ float Li[32][33];
  __shared__ float rli[32];
  const BlockDesc bd = blocks[blockIdx.x];
  const int n = bd.n, ld = bd.n_pad;
  const float* L = lpool + bd.off_mat;
  float* X = xpool + bd.off_mat;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // entries never written below: the strict upper triangle and the padding stay zero
  for (int r = warp; r < ld; r += kInvWarps)
    for (int c = lane; c < ld; c += 32)
      if (c > r || r >= n) X[(int64_t)r * ld + c] = 0.f;
  // rows [row0, row0 + 32) x columns [col0, col0 + 32) of a matrix into a chunk (zero rows >= rows)
  auto load_chunk = [&](float(*dst)[32], const float* src, int row0, int col0, int rows) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int e = tid + i * kInvWarps * 32;   // 256 16-byte pieces
      const int r = e >> 3, c4 = (e & 7) * 4;
      if (row0 + r < rows) cp_async16_b(&dst[r][c4], src + (int64_t)(row0 + r) * ld + col0 + c4);
      else *reinterpret_cast<float4*>(&dst[r][c4]) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  const int kw = warp * (32 / kInvWarps);
  const int nbk = (n + 31) / 32;
  __syncthreads();
  for (int ib = 0; ib < nbk; ++ib) {
    const int i0 = ib * 32, ibw = min(32, n - i0);
    // X_ii = L_ii^-1: lane = column, forward substitution (identity on the padding)
    if (warp == 0) {
      for (int r = 0; r < 32; ++r)
        Li[r][lane] = (r < ibw && lane < ibw && lane <= r) ? L[(int64_t)(i0 + r) * ld + i0 + lane] : (r == lane ? 1.f : 0.f);
      __syncwarp();
      rli[lane] = 1.f / Li[lane][lane];
      __syncwarp();
      // right-looking, lane = column, the partial rows in registers: once row q is final, its terms
      // leave every later row.  Row r still takes -L_rq x_q for q = 0, 1, ..., r - 1 in that order, and
      // the terms with q < lane are exact zeros, so the result is the left-looking sum's bit for bit.
      float acc[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) acc[r] = (r == lane) ? 1.f : 0.f;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float xq = (q >= lane) ? acc[q] * rli[q] : 0.f;
        Xi[q][lane] = xq;
#pragma unroll
        for (int r = q + 1; r < 32; ++r) acc[r] = fmaf(-Li[r][q], xq, acc[r]);
      }
    }
    __syncthreads();
    for (int cb = 0; cb < ib; ++cb) {
      const int c0 = cb * 32;
      float acc[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) acc[r] = 0.f;
      const int nch = ib - cb;               // chunks k0 = c0, ..., i0 - 32 (X_kc = 0 for k < c)
      load_chunk(As[0], L, i0, c0, n);
      load_chunk(Bs[0], X, c0, c0, n);
      cp_async_commit();
      for (int ch = 0; ch < nch; ++ch) {
        const int buf = ch & 1;
        if (ch + 1 < nch) {
          const int k1 = c0 + (ch + 1) * 32;
          load_chunk(As[buf ^ 1], L, i0, k1, n);
          load_chunk(Bs[buf ^ 1], X, k1, c0, n);
          cp_async_commit();
          cp_async_wait_group<1>();
        } else {
          cp_async_wait_group<0>();
        }
        __syncthreads();
        // this warp's 8 values of k in two halves of 4: X_kc in registers, each row's L_ik as one
        // 16-byte broadcast (every accumulator still takes its 8 terms in k order)
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          float bv[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) bv[j] = Bs[buf][kw + 4 * h + j][lane];
#pragma unroll
          for (int r = 0; r < 32; ++r) {
            const float4 a = *reinterpret_cast<const float4*>(&As[buf][r][kw + 4 * h]);
            float v = acc[r];
            v = fmaf(a.x, bv[0], v);
            v = fmaf(a.y, bv[1], v);
            v = fmaf(a.z, bv[2], v);
            v = fmaf(a.w, bv[3], v);
            acc[r] = v;
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int r = 0; r < 32; ++r) red[warp][r][lane] = acc[r];
      __syncthreads();
      // R = sum of the four partials (into red[0]), then X_ic = -X_ii R
      for (int e = tid; e < 1024; e += kInvWarps * 32) {
        const int r = e >> 5, c = e & 31;
        red[0][r][c] = (red[0][r][c] + red[1][r][c]) + (red[2][r][c] + red[3][r][c]);
      }
      __syncthreads();
      for (int j = 0; j < 8; ++j) {
        const int r = warp + kInvWarps * j;
        float v = 0.f;
        for (int k = 0; k <= r; ++k) v = fmaf(Xi[r][k], red[0][k][lane], v);
        if (r < ibw) X[(int64_t)(i0 + r) * ld + c0 + lane] = -v;
      }
      __syncthreads();
    }
    for (int e = tid; e < 1024; e += kInvWarps * 32) {
      const int r = e >> 5, c = e & 31;
      if (r < ibw && c <= r) X[(int64_t)(i0 + r) * ld + i0 + c] = Xi[r][c];
    }
    __syncthreads();
  }
}

// FP64 -> FP32 square copy with zero padding; optional transpose-free.
template <typename T>
__global__ void to_f32_kernel(const BlockDesc* __restrict__ blocks, const T* __restrict__ src, float* __restrict__ dst,
                              int lower_only) {
  const BlockDesc bd = blocks[blockIdx.y];
  const int n = bd.n, ld = bd.n_pad;
  const int64_t total = (int64_t)ld * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ld), c = (int)(e % ld);
    float v = 0.f;
    if (r < n && c < n && (!lower_only || c <= r)) v = (float)src[bd.off_mat + e];
    dst[bd.off_mat + e] = v;
  }
}

// Own-column slabs (column-major, ld = n_pad, zero beyond n):
//   W[:, j] = L^-1[:, p_j]            Z[:, j] = (L^-1 H_b)[:, p_j]       Lc[:, j] = L[p_j, :]^T
// with p_j the local position of the block's j-th own column.
template <typename T>
__global__ void slabs_kernel(const BlockDesc* __restrict__ blocks, const int32_t* __restrict__ own_pool,
                             const T* __restrict__ lfac, const float* __restrict__ linv32, const float* __restrict__ t1,
                             float* __restrict__ w, float* __restrict__ z, float* __restrict__ lc) {
  const BlockDesc bd = blocks[blockIdx.x];
  const int n = bd.n, ld = bd.n_pad;
  for (int j = 0; j < bd.c; ++j) {
    const int p = own_pool[bd.off_own + j];
    for (int i = threadIdx.x; i < ld; i += blockDim.x) {
      const int64_t o = bd.off_slab + (int64_t)j * ld + i;
      if (i < n) {
        w[o] = i >= p ? linv32[bd.off_mat + (int64_t)i * ld + p] : 0.f;   // L^-1 is lower triangular
        z[o] = t1[bd.off_mat + (int64_t)i * ld + p];
        lc[o] = (i <= p) ? (float)lfac[bd.off_mat + (int64_t)p * ld + i] : 0.f;
      } else {
        w[o] = 0.f; z[o] = 0.f; lc[o] = 0.f;
      }
    }
  }
}

// Diagonal of A0 at each own column, in blk_cols order (the Aufbau first point of the mu search).
__global__ void own_diag_kernel(const BlockDesc* __restrict__ blocks, const int32_t* __restrict__ own_pool,
                                const float* __restrict__ row_diag, float* __restrict__ out) {
  const BlockDesc bd = blocks[blockIdx.x];
  for (int j = threadIdx.x; j < bd.c; j += blockDim.x)
    out[bd.off_own + j] = row_diag[bd.off_idx + own_pool[bd.off_own + j]];
}

inline dim3 sq_grid(int n_blocks) { return dim3(64, n_blocks); }

}  // namespace

cudaError_t launch_gather(nolsm_ctx* ctx, float* hb, double* sb) {
  int max_n = 0, max_ld = 0;
  for (auto& b : ctx->h_blocks) {
    max_n = std::max(max_n, b.n);
    max_ld = std::max(max_ld, b.n_pad);
  }
  const int pairs_ = ctx->opt.chol_precision == NOLSM_CHOL_DF64 || ctx->opt.chol_precision == NOLSM_CHOL_DF64_SIMT;
  if (max_ld <= kGatherRowMax) {
    const size_t rsmem = (((size_t)max_n * 4 + 15) & ~(size_t)15) + (size_t)kGatherWarps * max_ld * 12;
    if (rsmem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(gather_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem);
      if (e != cudaSuccess) return e;
    }
    gather_rows_kernel<<<ctx->n_blocks, kGatherWarps * 32, rsmem, ctx->stream>>>(
        ctx->d_blocks, ctx->d_idx, ctx->d_row_ptr, ctx->d_col, ctx->d_hval, ctx->d_sval, hb, sb, ctx->d_flags, pairs_,
        max_n, max_ld);
    return cudaGetLastError();
  }
  const size_t smem = sizeof(int32_t) * (size_t)max_n;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(gather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int pairs = ctx->opt.chol_precision == NOLSM_CHOL_DF64 || ctx->opt.chol_precision == NOLSM_CHOL_DF64_SIMT;
  gather_kernel<<<ctx->n_blocks, 256, smem, ctx->stream>>>(ctx->d_blocks, ctx->d_idx, ctx->d_row_ptr, ctx->d_col,
                                                           ctx->d_hval, ctx->d_sval, hb, sb, ctx->d_flags, pairs);
  return cudaGetLastError();
}

cudaError_t launch_cholesky_inverse(nolsm_ctx* ctx, double* sb, int mode) {
  // sb holds T_b(S) in FP64 (first sum_sq doubles); the second half is scratch.
  float* s32 = reinterpret_cast<float*>(sb + ctx->sum_sq);   // FP32 factor lives in the scratch half
  cudaError_t e = cudaSuccess;
  if (mode == NOLSM_CHOL_DF64) {
    // blocked by 64-column panels: the 64 x 64 diagonal block and the slices of L11^-1 (FP32 pipe,
    // double-float 32 x 32 pivots), the rows below L21 = A21 L11^-T with their slices, and the
    // trailing update from the slices, both on the tensor cores
    int max_n = 0;
    for (const auto& bd : ctx->h_blocks) max_n = std::max(max_n, bd.n);
    for (int pnl = 0; pnl * kOzPanel < max_n; ++pnl) {
      const int c0 = pnl * kOzPanel;
      if (pnl > 0 && (e = phase_mark(ctx, NOLSM_PHASE_FACTOR)) != cudaSuccess) return e;
      chol_diag64_kernel<<<ctx->n_blocks, kDiagThreads, 0, ctx->stream>>>(ctx->d_blocks, sb, ctx->d_flags, c0, ctx->d_oz_exp,
                                                                 ctx->d_oz_m, ctx->d_oz_f, s32,
                                                                 ctx->cong_simt ? nullptr : ctx->d_linv);
      ctx->n_launches += 1;
      if (c0 + kOzPanel >= max_n) break;
      if ((e = phase_mark(ctx, NOLSM_PHASE_FACTOR_TRSM)) != cudaSuccess) return e;
      if ((e = launch_chol_trsm_tc(ctx, pnl, sb, s32)) != cudaSuccess) return e;
      if ((e = phase_mark(ctx, NOLSM_PHASE_FACTOR_UPDATE)) != cudaSuccess) return e;
      if ((e = launch_chol_update_tc(ctx, pnl, sb)) != cudaSuccess) return e;
    }
    // (the diagonal and TRSM kernels wrote the factor's FP32 rounding beside the pairs)
    if ((e = phase_mark(ctx, NOLSM_PHASE_INVERSE)) != cudaSuccess) return e;
    // mixed paths: the tiled inverse with its off-diagonal blocks on the tensor cores (three TF32
    // passes, the congruence's arithmetic); FP32 path: the SIMT inverse with two-level sums
    if (!ctx->cong_simt) return launch_trinv_tc(ctx, s32, ctx->d_t1);
    trinv_tile_kernel<<<ctx->n_blocks, kInvWarps * 32, 0, ctx->stream>>>(ctx->d_blocks, s32, ctx->d_linv);
  } else if (mode == NOLSM_CHOL_DF64_SIMT) {
    cholesky_df_kernel<<<ctx->n_blocks, kCholWarps * 32, 0, ctx->stream>>>(ctx->d_blocks, sb, s32, ctx->d_flags, 0,
                                                                          1 << 30, nullptr, 1 << 30, nullptr);
    if ((e = phase_mark(ctx, NOLSM_PHASE_INVERSE)) != cudaSuccess) return e;
    trinv_tile_kernel<<<ctx->n_blocks, kInvWarps * 32, 0, ctx->stream>>>(ctx->d_blocks, s32, ctx->d_linv);
  } else if (mode == NOLSM_CHOL_FP64_INV64) {
    cholesky_kernel<double, 4><<<ctx->n_blocks, 128, 0, ctx->stream>>>(ctx->d_blocks, sb, nullptr, ctx->d_flags);
    if ((e = phase_mark(ctx, NOLSM_PHASE_INVERSE)) != cudaSuccess) return e;
    trinv_kernel<double, 4><<<ctx->n_blocks, 128, 0, ctx->stream>>>(ctx->d_blocks, sb, sb + ctx->sum_sq);
    to_f32_kernel<double><<<sq_grid(ctx->n_blocks), 256, 0, ctx->stream>>>(ctx->d_blocks, sb + ctx->sum_sq, ctx->d_linv, 1);
  } else if (mode == NOLSM_CHOL_FP64) {
    cholesky_kernel<double, 4><<<ctx->n_blocks, 128, 0, ctx->stream>>>(ctx->d_blocks, sb, s32, ctx->d_flags);
    if ((e = phase_mark(ctx, NOLSM_PHASE_INVERSE)) != cudaSuccess) return e;
    trinv_tile_kernel<<<ctx->n_blocks, kInvWarps * 32, 0, ctx->stream>>>(ctx->d_blocks, s32, ctx->d_linv);
  } else {
    to_f32_kernel<double><<<sq_grid(ctx->n_blocks), 256, 0, ctx->stream>>>(ctx->d_blocks, sb, s32, 0);
    cholesky_kernel<float, 4><<<ctx->n_blocks, 128, 0, ctx->stream>>>(ctx->d_blocks, s32, nullptr, ctx->d_flags);
    if ((e = phase_mark(ctx, NOLSM_PHASE_INVERSE)) != cudaSuccess) return e;
    trinv_tile_kernel<<<ctx->n_blocks, kInvWarps * 32, 0, ctx->stream>>>(ctx->d_blocks, s32, ctx->d_linv);
  }
  return cudaGetLastError();
}

// The 128 x 128 diagonal blocks of the mixed paths' L^-1 from the 64 x 64 ones the blocked factor
// left in X (L11^-1 of every panel, computed in double-float and rounded):
//   [[A, 0], [B, C]]^-1 = [[A^-1, 0], [-C^-1 B A^-1, C^-1]],
// the off-diagonal quarter by two 64 x 64 x 64 FP32 products (B from the factor's FP32 rounding).
// The CTA writes zeros where the block lies past n (panels past n were never factored) and the
// block's transpose into ypool (Y = X^T, the tiled inverse's second operand); the blocks right of
// the diagonal block stay unwritten (nothing reads them).  Grid: (block,
// diagonal block); 256 threads; dynamic shared memory: A^-1, C^-1, B and B A^-1 (64 x 65 floats
// each, kTrinv128Smem).
constexpr int kTrinv128Smem = 4 * 64 * 65 * (int)sizeof(float);
__global__ void __launch_bounds__(256) trinv128_kernel(const BlockDesc* __restrict__ blocks,
                                                       const float* __restrict__ lpool, float* __restrict__ xpool,
                                                       float* __restrict__ ypool) {
  extern __shared__ float t128_smem[];
  float(*Ai)[65] = reinterpret_cast<float(*)[65]>(t128_smem);
  float(*Ci)[65] = Ai + 64;
  float(*Bq)[65] = Ci + 64;
  float(*Tq)[65] = Bq + 64;
  const BlockDesc bd = blocks[blockIdx.x];
  const int ld = bd.n_pad, n = bd.n;
  const int o = 128 * (int)blockIdx.y;
  if (o >= ld) return;
  const int tid = threadIdx.x;
  float* X = xpool + bd.off_mat;
  const float* L = lpool + bd.off_mat;
  const bool live_a = o < n, live_c = o + 64 < n;   // diagonal 64-blocks that were factored
  // the upper-right quarter inside the diagonal block (the blocks right of it are never read: the
  // products stop their K at the diagonal block, the slabs take the lower triangle only)
  for (int e = tid; e < 4096; e += 256) X[(int64_t)(o + (e >> 6)) * ld + o + 64 + (e & 63)] = 0.f;
  for (int e = tid; e < 4096; e += 256) {
    const int r = e >> 6, c = e & 63;
    Ai[r][c] = live_a ? X[(int64_t)(o + r) * ld + o + c] : 0.f;
    Ci[r][c] = live_c ? X[(int64_t)(o + 64 + r) * ld + o + 64 + c] : 0.f;
    Bq[r][c] = live_c ? L[(int64_t)(o + 64 + r) * ld + o + c] : 0.f;
  }
  __syncthreads();
  // T = B A^-1 (A^-1 lower triangular: k >= c), then the quarter -C^-1 T (C^-1 lower: k <= r)
  for (int e = tid; e < 4096; e += 512) {        // two rows per pass (independent chains)
    const int r = e >> 6, c = e & 63;
    float acc0 = 0.f, acc1 = 0.f;
    for (int k = c; k < 64; ++k) {
      const float a = Ai[k][c];
      acc0 = fmaf(Bq[r][k], a, acc0);
      acc1 = fmaf(Bq[r + 4][k], a, acc1);
    }
    Tq[r][c] = acc0;
    Tq[r + 4][c] = acc1;
  }
  __syncthreads();
  for (int e = tid; e < 4096; e += 512) {        // rows r and r + 4 (row r's sum stops at k = r)
    const int r = e >> 6, c = e & 63;
    float acc0 = 0.f, acc1 = 0.f;
    for (int k = 0; k <= r; ++k) {
      const float t = Tq[k][c];
      acc0 = fmaf(Ci[r][k], t, acc0);
      acc1 = fmaf(Ci[r + 4][k], t, acc1);
    }
    for (int k = r + 1; k <= r + 4; ++k) acc1 = fmaf(Ci[r + 4][k], Tq[k][c], acc1);
    Bq[r][c] = -acc0;                            // the quarter (B is no longer needed)
    Bq[r + 4][c] = -acc1;
    X[(int64_t)(o + 64 + r) * ld + o + c] = -acc0;
    X[(int64_t)(o + 68 + r) * ld + o + c] = -acc1;
  }
  for (int e = tid; e < 4096; e += 256) {
    const int r = e >> 6, c = e & 63;
    if (!live_a) X[(int64_t)(o + r) * ld + o + c] = 0.f;
    if (!live_c) X[(int64_t)(o + 64 + r) * ld + o + 64 + c] = 0.f;
  }
  __syncthreads();
  // Y's diagonal block is X's transposed, written from shared memory: Y[c][r] = X[r][c] with
  // X = [[A^-1, 0], [quarter, C^-1]] (consecutive threads take consecutive r: coalesced rows of Y,
  // conflict-free columns of the 65-wide arrays)
  float* Y = ypool + bd.off_mat + (int64_t)o * ld + o;
  for (int e = tid; e < 128 * 128; e += 256) {
    const int c = e >> 7, r = e & 127;
    float v;
    if (c < 64) v = r < 64 ? Ai[r][c] : Bq[r - 64][c];
    else v = r < 64 ? 0.f : Ci[r - 64][c - 64];
    Y[(int64_t)c * ld + r] = v;
  }
}

// X_ii = L_ii^-1 of every 128 x 128 diagonal block, Y_ii = X_ii^T, strict upper blocks of X zeroed
void trinv_diag_launch(nolsm_ctx* ctx, const float* l32, float* ypool, int max_nb) {
  static bool attr_done = false;
  if (!attr_done &&
      cudaFuncSetAttribute(trinv128_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrinv128Smem) == cudaSuccess)
    attr_done = true;
  trinv128_kernel<<<dim3(ctx->n_blocks, max_nb), 256, kTrinv128Smem, ctx->stream>>>(ctx->d_blocks, l32, ctx->d_linv,
                                                                                    ypool);
  ctx->n_launches += 1;
}

cudaError_t launch_congruence(nolsm_ctx* ctx, float* t1) {
  // T_b(H0) (FP32) sits in A0's pool.  T1 = L^-1 H_b (H symmetric: NT form), A0 = T1 L^-T: on the
  // tensor cores (three TF32 passes) unless the SIMT products are asked for.
  if (!ctx->cong_simt) return launch_congruence_tc(ctx, t1);
  cudaError_t e = launch_sgemm_nt(ctx, ctx->d_linv, ctx->d_a0, t1, /*a_lower=*/1, /*b_lower=*/0, /*sym=*/0);
  if (e != cudaSuccess) return e;
  // A0 is symmetric: upper tiles only, mirrored stores (exactly symmetric, half the work)
  return launch_sgemm_nt(ctx, t1, ctx->d_linv, ctx->d_a0, 0, /*b_lower=*/1, /*sym=*/1);
}

cudaError_t launch_slabs_impl(nolsm_ctx* ctx, const void* lfac, int fp32, const float* t1) {
  if (!fp32)
    slabs_kernel<double><<<ctx->n_blocks, 256, 0, ctx->stream>>>(ctx->d_blocks, ctx->d_own, (const double*)lfac,
                                                                ctx->d_linv, t1, ctx->d_w, ctx->d_z, ctx->d_lc);
  else
    slabs_kernel<float><<<ctx->n_blocks, 256, 0, ctx->stream>>>(ctx->d_blocks, ctx->d_own, (const float*)lfac,
                                                               ctx->d_linv, t1, ctx->d_w, ctx->d_z, ctx->d_lc);
  return cudaGetLastError();
}

cudaError_t launch_own_diag(nolsm_ctx* ctx) {
  own_diag_kernel<<<ctx->n_blocks, 128, 0, ctx->stream>>>(ctx->d_blocks, ctx->d_own, ctx->d_rowd, ctx->d_own_diag);
  return cudaGetLastError();
}

}  // namespace nolsm
