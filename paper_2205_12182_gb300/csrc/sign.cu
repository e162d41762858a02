// The mu-dependent part of the NOLSM step: the Newton-Schulz sign iteration (Eq. 6) on
// every block's A0 - mu I, the iteration control, the own-column slab refinement with the
// block traces of D S and D H0, the density scatter (step 3) and the band energy (Eq. 4).
//
// Matrix products here are the SIMT FP32 path; the tensor-core products live in sign_tc.cu
// and share the control kernels below.
#include "internal.h"

#include <cooperative_groups.h>

#include <cfloat>
#include <type_traits>

namespace nolsm {
namespace {

__device__ __forceinline__ void set_error(DevFlags* f, int code) { atomicCAS(&f->error, 0, code); }

template <typename T> __device__ __forceinline__ float ld_as_float(const T* p);
template <> __device__ __forceinline__ float ld_as_float<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ld_as_float<__half>(const __half* p) { return __half2float(*p); }
template <> __device__ __forceinline__ float ld_as_float<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }

template <typename T> __device__ __forceinline__ T from_float(float v);
template <> __device__ __forceinline__ float from_float<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_float<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_float<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }


// ----------------------------------------------------------------------------------------------
// Grouped SIMT product C = A B^T on 128x128 tiles (both operands row-major, K contiguous).
// MODE 0: plain store.  MODE 1: NS first product T = X X^T (X symmetric), epilogue writes
//   B = 1.5 a I - 0.5 a^3 T and accumulates ||T - I||_F^2 per block.  MODE 2: X+ = X B^T.
// MODE 3: plain store of a product known to be symmetric (upper tiles, mirrored).
// TWO: two-level summation for the FP32 path -- each BK-wide slice of k is summed into fresh
// registers and then added to the running sum, so a length-n dot product carries about
// (BK + n / BK) roundings instead of n (one extra add per slice; twice the accumulator registers,
// one CTA per SM).
constexpr int BM = 128, BN = 128, BK = 16;

template <int MODE, bool TWO>
__global__ void __launch_bounds__(256, TWO ? 1 : 2)
sgemm_nt_kernel(const Tile* __restrict__ tiles, const int32_t* __restrict__ n_tiles_dev, int n_tiles_host,
                const BlockDesc* __restrict__ blocks, const float* __restrict__ a_pool, const float* __restrict__ b_pool,
                float* __restrict__ c_pool, float* __restrict__ x0, float* __restrict__ x1, float* __restrict__ bbuf,
                const NsState* __restrict__ st, float* __restrict__ resacc) {
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int lrow = tid >> 2, lcol = (tid & 3) * 4;
  const int n_tiles = n_tiles_dev ? *n_tiles_dev : n_tiles_host;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const Tile tl = tiles[t];
    const BlockDesc bd = blocks[tl.block];
    const int ld = bd.n_pad;
    const float* A;
    const float* B;
    float* C;
    float c1 = 0.f, c3 = 0.f;
    if (MODE == 0 || MODE == 3) {
      A = a_pool + bd.off_mat; B = b_pool + bd.off_mat; C = c_pool + bd.off_mat;
    } else {
      const NsState s = st[tl.block];
      float* X = s.cur ? x1 : x0;
      A = X + bd.off_mat;
      if (MODE == 1) { B = X + bd.off_mat; C = bbuf + bd.off_mat; c1 = 1.5f * s.a; c3 = 0.5f * s.a * s.a * s.a; }
      else { B = bbuf + bd.off_mat; C = (s.cur ? x0 : x1) + bd.off_mat; }
    }
    const float* Ag = A + (int64_t)(tl.m0 + lrow) * ld + lcol;
    const float* Bg = B + (int64_t)(tl.n0 + lrow) * ld + lcol;
    const int64_t half = (int64_t)64 * ld;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    const int kend = tl.kend;
    float4 ra0 = *reinterpret_cast<const float4*>(Ag);
    float4 ra1 = *reinterpret_cast<const float4*>(Ag + half);
    float4 rb0 = *reinterpret_cast<const float4*>(Bg);
    float4 rb1 = *reinterpret_cast<const float4*>(Bg + half);
    int buf = 0;
    for (int k0 = 0; k0 < kend; k0 += BK) {
      As[buf][lcol + 0][lrow] = ra0.x; As[buf][lcol + 1][lrow] = ra0.y; As[buf][lcol + 2][lrow] = ra0.z; As[buf][lcol + 3][lrow] = ra0.w;
      As[buf][lcol + 0][lrow + 64] = ra1.x; As[buf][lcol + 1][lrow + 64] = ra1.y; As[buf][lcol + 2][lrow + 64] = ra1.z; As[buf][lcol + 3][lrow + 64] = ra1.w;
      Bs[buf][lcol + 0][lrow] = rb0.x; Bs[buf][lcol + 1][lrow] = rb0.y; Bs[buf][lcol + 2][lrow] = rb0.z; Bs[buf][lcol + 3][lrow] = rb0.w;
      Bs[buf][lcol + 0][lrow + 64] = rb1.x; Bs[buf][lcol + 1][lrow + 64] = rb1.y; Bs[buf][lcol + 2][lrow + 64] = rb1.z; Bs[buf][lcol + 3][lrow + 64] = rb1.w;
      __syncthreads();
      if (k0 + BK < kend) {
        ra0 = *reinterpret_cast<const float4*>(Ag + k0 + BK);
        ra1 = *reinterpret_cast<const float4*>(Ag + half + k0 + BK);
        rb0 = *reinterpret_cast<const float4*>(Bg + k0 + BK);
        rb1 = *reinterpret_cast<const float4*>(Bg + half + k0 + BK);
      }
#pragma unroll
      float part[TWO ? 8 : 1][TWO ? 8 : 1];
      if constexpr (TWO) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) part[i][j] = 0.f;
      }
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            if constexpr (TWO) part[i][j] = fmaf(av[i], bv[j], part[i][j]);
            else acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
          }
      }
      if constexpr (TWO) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] += part[i][j];
      }
      buf ^= 1;
    }
    __syncthreads();
    // epilogue.  MODE 0 writes the full tile.  MODE 1/2 tiles lie on or above the block diagonal:
    // entry (r, c) with c > r is written at (r, c) and (c, r), the diagonal once, c < r skipped, so
    // every iterate is exactly symmetric (the products read the transpose of their B operand).
    float rsq = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = tl.m0 + ((i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4));
#pragma unroll
      for (int jh = 0; jh < 2; ++jh) {
        const int c = tl.n0 + jh * 64 + tx * 4;
        float4 v = make_float4(acc[i][jh * 4 + 0], acc[i][jh * 4 + 1], acc[i][jh * 4 + 2], acc[i][jh * 4 + 3]);
        if (MODE == 0) {
          *reinterpret_cast<float4*>(C + (int64_t)r * ld + c) = v;
          continue;
        }
        float* pv = &v.x;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int cq = c + q;
          if (cq < r) continue;
          float o = pv[q];
          if (MODE == 1) {
            const float d = (r == cq) ? 1.f : 0.f;
            const float e = o - d;
            rsq = fmaf((r == cq) ? 1.f : 2.f, e * e, rsq);
            o = c1 * d - c3 * o;
          }
          C[(int64_t)r * ld + cq] = o;
          if (cq > r) C[(int64_t)cq * ld + r] = o;
        }
      }
    }
    if (MODE == 1) {
      for (int o = 16; o; o >>= 1) rsq += __shfl_xor_sync(0xffffffffu, rsq, o);
      if ((tid & 31) == 0) atomicAdd(&resacc[tl.block], rsq);
    }
  }
}

// ----------------------------------------------------------------------------------------------
// Iteration control.

// State at the start of a sign evaluation: alpha from the spectral bounds (Gershgorin, with a
// relative margin) so that ||X_0||_2 < 1; the scaled iteration starts from lower bound l0.
// mode 0: Gershgorin scale, lower bound l0.  mode 1: Lanczos Ritz values widened by the last
// Lanczos coefficient.  mode 2: network predictions (lambda_min, lambda_max, log10 distance of mu to
// the nearest eigenvalue): scale 1.25 x the predicted radius, lower bound half the predicted
// distance.  A scale below the rigorous Gershgorin one starts with one unscaled step, which maps
// any eigenvalue in (0, sqrt 3) into (0, 1]; the Gershgorin scale stays the cap.
// Smallest lower bound a prediction may set (out-of-distribution predictions of the distance to mu
// have been two orders of magnitude low; at l = 1e-3 FP16 iterates then miss the 1e-3 accuracy bar).
constexpr float kPredLowerFloor = 0.01f;

__global__ void ns_state_kernel(int n_blocks, const double* __restrict__ lo, const double* __restrict__ hi,
                                double mu, float margin, float l0, float l_floor, int scaled, int mode,
                                const float* __restrict__ lz, const float* __restrict__ pred,
                                NsState* __restrict__ st, float* __restrict__ resacc, DevFlags* flags) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) { flags->sum_n = 0.0; flags->sum_e = 0.0; flags->queue = 0; }
  if (b >= n_blocks) return;
  const double rad = fmax(fabs(hi[b] - mu), fabs(mu - lo[b]));
  float alpha = (float)(rad * (1.0 + margin));
  if (!(alpha > 0.f)) alpha = 1.f;
  // A scale below the true radius / sqrt(3) would send eigenvalues beyond sqrt(3), which the
  // unscaled first step maps to the wrong sign (and between sqrt(3) and sqrt(5) the iteration still
  // converges, so no residual test sees it).  The Gershgorin scale bounds the radius from above, so
  // no scale goes below it / 1.7.
  const float alpha_floor = alpha / 1.7f;
  float l = l0;
  bool plain_first = false;
  if (mode == 1 && lz) {
    const float w = fabsf(lz[4 * b + 2]);
    float r = fmaxf(lz[4 * b + 1] + w - (float)mu, (float)mu - lz[4 * b + 0] + w) * (1.f + margin);
    r = fmaxf(r, alpha_floor);
    if (r < alpha) { alpha = r; plain_first = true; }
  } else if (mode == 2 && pred) {
    float r = 1.25f * fmaxf(pred[3 * b + 1] - (float)mu, (float)mu - pred[3 * b + 0]);
    r = fmaxf(r, alpha_floor);
    if (r < alpha) { alpha = r; plain_first = true; }
    const float dist = exp10f(fminf(fmaxf(pred[3 * b + 2], -8.f), 1.f));
    // A predicted bound far below the truth is an accuracy hazard, not only a cost: the first
    // scaled step maps the top of the spectrum to about 2.6 l, where the rounding of the iterate's
    // O(1) entries is a large relative error of those components.  Raising l above the truth only
    // costs iterations (eigenvalues below l still grow every step, and the plain tail converges).
    l = fmaxf(0.5f * dist / alpha, kPredLowerFloor);
  }
  NsState s;
  s.alpha = alpha;
  s.l = scaled ? fminf(fmaxf(l, l_floor), 0.9f) : 1.f;
  s.a = plain_first ? 1.f : cc_scale(s.l);
  s.res = FLT_MAX;
  s.res_prev = FLT_MAX;
  s.iters = 0;
  s.status = kActive;
  s.cur = 0;
  s.grow = 0;
  s.restarts = 0;
  st[b] = s;
  resacc[b] = 0.f;
}

// Restart of diverged blocks: X_0 again, with the Gershgorin scale and lower bound l0.
template <typename T>
__global__ void ns_restart_fill_kernel(const BlockDesc* __restrict__ blocks, const float* __restrict__ a0,
                                       const NsState* __restrict__ st, const double* __restrict__ lo,
                                       const double* __restrict__ hi, const double* __restrict__ mu_p, float margin,
                                       T* __restrict__ x0) {
  const int b = blockIdx.x;
  if (st[b].status != kRestart) return;
  const double mu = *mu_p;
  const BlockDesc bd = blocks[b];
  const int n = bd.n, ld = bd.n_pad;
  const float alpha = (float)(fmax(fabs(hi[b] - mu), fabs(mu - lo[b])) * (1.0 + margin));
  const float inv = 1.f / alpha, muf = (float)mu;
  const int64_t total = (int64_t)ld * ld;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
    const int r = (int)(e / ld), c = (int)(e % ld);
    float v;
    if (r < n && c < n) v = (a0[bd.off_mat + e] - (r == c ? muf : 0.f)) * inv;
    else v = (r == c) ? 1.f : 0.f;
    x0[bd.off_mat + e] = from_float<T>(v);
  }
}

__global__ void ns_restart_state_kernel(int n_blocks, const double* __restrict__ lo, const double* __restrict__ hi,
                                        const double* __restrict__ mu_p, float margin, float l0, int scaled,
                                        NsState* __restrict__ st, float* __restrict__ resacc) {
  const double mu = *mu_p;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_blocks) return;
  NsState s = st[b];
  if (s.status != kRestart) return;
  s.alpha = (float)(fmax(fabs(hi[b] - mu), fabs(mu - lo[b])) * (1.0 + margin));
  s.l = scaled ? fminf(l0, 1.f) : 1.f;   // l0 carries the format's floor
  s.a = cc_scale(s.l);
  s.res = FLT_MAX;
  s.res_prev = FLT_MAX;
  s.cur = 0;
  s.grow = 0;
  s.status = kActive;
  st[b] = s;
  resacc[b] = 0.f;
}

// X_0 = (A0 - mu I) / alpha on the n x n part, identity on the padding.
template <typename T>
__global__ void ns_fill_kernel(const BlockDesc* __restrict__ blocks, const float* __restrict__ a0,
                               const NsState* __restrict__ st, double mu, T* __restrict__ x0) {
  const BlockDesc bd = blocks[blockIdx.y];
  const int n = bd.n, ld = bd.n_pad;
  const float inv = 1.f / st[blockIdx.y].alpha;
  const float muf = (float)mu;
  const int64_t total = (int64_t)ld * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ld), c = (int)(e % ld);
    float v;
    if (r < n && c < n) v = (a0[bd.off_mat + e] - (r == c ? muf : 0.f)) * inv;
    else v = (r == c) ? 1.f : 0.f;
    x0[bd.off_mat + e] = from_float<T>(v);
  }
}

// Tile list of the blocks still iterating (single CTA scan); also counts them.
__global__ void __launch_bounds__(1024) ns_tiles_kernel(int n_blocks, const BlockDesc* __restrict__ blocks,
                                                        const NsState* __restrict__ st, int tile_n,
                                                        Tile* __restrict__ tiles, DevFlags* flags) {
  __shared__ int32_t warp_sums[32];
  __shared__ int32_t base;
  __shared__ int32_t active_total;
  if (threadIdx.x == 0) { base = 0; active_total = 0; }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int b0 = 0; b0 < n_blocks; b0 += blockDim.x) {
    const int b = b0 + threadIdx.x;
    int cnt = 0, nm = 0, np = 0;
    if (b < n_blocks && st[b].status == kActive) {
      np = blocks[b].n_pad;
      nm = np / BM;
      // row tile mi covers columns [mi*BM, np): the upper triangle including the diagonal tile
      for (int mi = 0; mi < nm; ++mi) cnt += (np - mi * BM + tile_n - 1) / tile_n;
    }
    // block-wide exclusive scan of cnt
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int w = warp_sums[lane];
      int wi = w;
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += v;
      }
      warp_sums[lane] = wi - w;
    }
    __syncthreads();
    const int off = base + warp_sums[warp] + incl - cnt;
    if (cnt) {
      int k = 0;
      for (int mi = 0; mi < nm; ++mi)
        for (int n0 = mi * BM; n0 < np; n0 += tile_n, ++k) {
          Tile tl;
          tl.block = b; tl.m0 = mi * BM; tl.n0 = n0; tl.kend = np;
          tiles[off + k] = tl;
        }
      atomicAdd(&active_total, 1);
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) base = off + cnt;
    __syncthreads();
  }
  if (threadIdx.x == 0) { flags->n_tiles = base; flags->n_active = active_total; }
}

// After the first product of an iteration: the residual decides convergence.
__global__ void ns_check_kernel(int n_blocks, const BlockDesc* __restrict__ blocks, NsState* __restrict__ st,
                                float* __restrict__ resacc, const float* __restrict__ tol_b, int max_iter,
                                int detect_divergence, DevFlags* flags) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_blocks) return;
  NsState s = st[b];
  if (s.status != kActive) return;
  const float res = sqrtf(resacc[b]);
  resacc[b] = 0.f;
  // after the first step every eigenvalue of a well-scaled iterate lies in [-1, 1], so
  // ||X^2 - I||_F <= sqrt(n_pad); beyond that the scale was too small: restart (once per block)
  if (detect_divergence && s.iters >= 1 && s.restarts == 0 &&
      (!isfinite(res) || res > 1.5f * sqrtf((float)blocks[b].n_pad))) {
    s.status = kRestart;
    s.restarts += 1;
    st[b] = s;
    return;
  }
  if (!isfinite(res)) { s.status = kFailed; s.res = res; st[b] = s; set_error(flags, NOLSM_ENONFINITE); return; }
  s.res_prev = s.res;
  s.res = res;
  const bool plain = s.l >= 1.f;
  if (res <= tol_b[b]) {
    s.status = kConverged;
  } else if (plain && s.iters >= 2 && res < 0.25f && res > 0.5f * s.res_prev) {
    s.status = kConverged;      // rounding floor of the operand format reached
  } else if (s.iters >= max_iter) {
    s.status = kFailed;
    set_error(flags, NOLSM_ENOCONV);
  }
  st[b] = s;
}

// After the second product: the new iterate is in the other buffer.
__global__ void ns_advance_kernel(int n_blocks, NsState* __restrict__ st) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_blocks) return;
  NsState s = st[b];
  if (s.status != kActive) return;
  s.cur ^= 1;
  s.iters += 1;
  s.l = cc_next(s.l, s.a);
  s.a = cc_scale(s.l);
  st[b] = s;
}

// ----------------------------------------------------------------------------------------------
// Own-column slab: G = g(X) W with g = f o ... o f (refine times), f(X) = (3X - X^3)/2, then
// Y = (W - G)/2 = T(D) columns before the back-transform, and the block traces
//   N_b = sum_{j in C_b} (L P L^-1)_jj = <Lc, Y>,   E_b = sum_j (H_b D_b)_jj = <Z, Y>   (FP64 sums).
// One CTA per block; slabs are column-major (ld = n_pad) in global scratch, X rows stream
// through shared memory in 128 x 32 tiles.
// Compensated accumulation (Dot2 of Ogita, Rump & Oishi 2005): the rounding error of each
// product (by FMA) and of each addition (TwoSum) is summed on the side; the FP32 path uses it for
// the slab products and the back-transform, where the error budget is tightest.
struct Acc2 {
  float s = 0.f, e = 0.f;
  __device__ __forceinline__ void add_prod(float x, float y) {
    const float p = x * y;
    const float pe = fmaf(x, y, -p);
    const float t = s + p;
    const float z = t - s;
    e += ((s - (t - z)) + (p - z)) + pe;
    s = t;
  }
  __device__ __forceinline__ float value() const { return s + e; }
};

template <bool COMP>
struct AccSel;
template <> struct AccSel<false> {
  float s = 0.f;
  __device__ __forceinline__ void add_prod(float x, float y) { s = fmaf(x, y, s); }
  __device__ __forceinline__ float value() const { return s; }
};
template <> struct AccSel<true> : Acc2 {};

template <typename T>
__device__ void slab_product(const T* __restrict__ X, int ld, int c, const float* __restrict__ V,
                             float* __restrict__ P, float (*Xs)[33], float (*Vs)[8]) {
  constexpr bool COMP = std::is_same<T, float>::value;
  const int tid = threadIdx.x;
  const int row = tid >> 1, cb = (tid & 1) * 4;
  for (int r0 = 0; r0 < ld; r0 += 128) {
    for (int c0 = 0; c0 < c; c0 += 8) {
      AccSel<COMP> acc[4];
      for (int k0 = 0; k0 < ld; k0 += 32) {
        {   // 16 independent loads per thread in flight (blockDim.x == 256)
          float xv[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int e = tid + j * 256;
            xv[j] = ld_as_float<T>(X + (int64_t)(r0 + (e >> 5)) * ld + k0 + (e & 31));
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int e = tid + j * 256;
            Xs[e >> 5][e & 31] = xv[j];
          }
        }
        {
          const int kk = tid >> 3, cc = tid & 7;   // 256 threads = 32 x 8
          Vs[kk][cc] = (c0 + cc < c) ? V[(int64_t)(c0 + cc) * ld + k0 + kk] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
          const float x = Xs[row][kk];
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q].add_prod(x, Vs[kk][cb + q]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c0 + cb + q < c) P[(int64_t)(c0 + cb + q) * ld + r0 + row] = acc[q].value();
    }
  }
  __syncthreads();
}

__device__ void slab_axpby(float alpha, const float* __restrict__ a, float beta, const float* __restrict__ b,
                           float* __restrict__ out, int64_t len) {
  for (int64_t i = threadIdx.x; i < len; i += blockDim.x) out[i] = alpha * a[i] + beta * b[i];
  __syncthreads();
}

template <typename T>
__device__ void slab_f(const T* X, int ld, int c, const float* V, float* out, float* t1, float* t2, float* t3,
                       float (*Xs)[33], float (*Vs)[8]) {
  slab_product<T>(X, ld, c, V, t1, Xs, Vs);
  slab_product<T>(X, ld, c, t1, t2, Xs, Vs);
  slab_product<T>(X, ld, c, t2, t3, Xs, Vs);
  slab_axpby(1.5f, t1, -0.5f, t3, out, (int64_t)ld * c);
}

// ---- Own-column slab with X resident in shared memory: one cluster of kSlabCluster CTAs per
// block.  CTA q holds rows [qR, qR + R) of X (R = n_pad / kSlabCluster, a contiguous range of the
// row-major block, copied once with cp.async).  Every product X V (V: n_pad x 8, all columns of a
// group of up to 8 own columns) is computed slice by slice; each CTA writes its rows of the result
// into every CTA's copy of the next V through distributed shared memory, and a cluster barrier
// separates the products.  X is read from HBM once per evaluation instead of once per product.
// Within a CTA, thread (rp, ks) = (tid / 8, tid % 8) forms the row pair 2rp, 2rp + 1 over the
// 16-byte k-chunks ks, ks + 8, ...; a butterfly over the 8 lanes of a group leaves the sums in all
// of them, and lane ks then writes the rows to cluster rank ks.
constexpr int kSlabCluster = 8;
constexpr size_t kSmemOptin = 227 * 1024;

template <typename T>
__host__ __device__ inline size_t slab_cluster_smem(int n_pad) {
  const size_t R = (size_t)n_pad / kSlabCluster, ck = 16 / sizeof(T);
  return R * n_pad * sizeof(T)                          // this CTA's rows of X
         + 2 * ((size_t)n_pad / ck) * (ck * 8 + 4) * 4  // two full slabs of 8 columns (padded chunks)
         + 4 * R * 8 * 4;                               // local rows: W, t1, t3 / F, F1
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename T> __device__ __forceinline__ void ld_chunk(const T* p, float* out);
template <> __device__ __forceinline__ void ld_chunk<float>(const float* p, float* out) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
template <> __device__ __forceinline__ void ld_chunk<__half>(const __half* p, float* out) {
  const uint4 v = *reinterpret_cast<const uint4*>(p);
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[i]));
    out[2 * i] = f.x; out[2 * i + 1] = f.y;
  }
}
template <> __device__ __forceinline__ void ld_chunk<__nv_bfloat16>(const __nv_bfloat16* p, float* out) {
  const uint4 v = *reinterpret_cast<const uint4*>(p);
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[i]));
    out[2 * i] = f.x; out[2 * i + 1] = f.y;
  }
}

// Rows 2 rpi, 2 rpi + 1 of Xs V (8 columns), reduced over the 8 k-slices of the lane group.
template <typename T>
__device__ __forceinline__ void slab_rowpair(const T* __restrict__ Xs, int ld, const float* __restrict__ V, int rpi,
                                             int ks, float (&out)[2][8]) {
  constexpr bool COMP = std::is_same<T, float>::value;
  constexpr int CK = 16 / (int)sizeof(T);
  constexpr int VS = CK * 8 + 4;
  AccSel<COMP> acc[2][8];
  const T* x0 = Xs + (size_t)(2 * rpi) * ld;
  const T* x1 = x0 + ld;
  const int nch = ld / CK;
  for (int g = ks; g < nch; g += 8) {
    float a0[CK], a1[CK];
    ld_chunk<T>(x0 + g * CK, a0);
    ld_chunk<T>(x1 + g * CK, a1);
    const float* v = V + g * VS;
#pragma unroll
    for (int kk = 0; kk < CK; ++kk) {
      const float4 va = *reinterpret_cast<const float4*>(v + kk * 8);
      const float4 vb = *reinterpret_cast<const float4*>(v + kk * 8 + 4);
      const float vv[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        acc[0][cc].add_prod(a0[kk], vv[cc]);
        acc[1][cc].add_prod(a1[kk], vv[cc]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      if constexpr (COMP) {
        // compensated butterfly: TwoSum of the leading parts, the errors summed on the side
        float s = acc[i][cc].s, e = acc[i][cc].e;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
          const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
          const float e2 = __shfl_xor_sync(0xffffffffu, e, o);
          const float t = s + s2;
          const float z = t - s;
          const float err = (s - (t - z)) + (s2 - z);
          s = t;
          e = (e + e2) + err;
        }
        out[i][cc] = s + e;
      } else {
        float s = acc[i][cc].s;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        out[i][cc] = s;
      }
    }
}

template <typename T>
__global__ void __cluster_dims__(kSlabCluster, 1, 1) __launch_bounds__(256)
    slab_cluster_kernel(const BlockDesc* __restrict__ blocks, const NsState* __restrict__ st, const T* __restrict__ x0,
                        const T* __restrict__ x1, const float* __restrict__ w, const float* __restrict__ z,
                        const float* __restrict__ lc, float* __restrict__ y, int refine, size_t cluster_cap,
                        double* __restrict__ bn, double* __restrict__ be) {
  namespace cg = cooperative_groups;
  constexpr int CK = 16 / (int)sizeof(T);
  constexpr int VS = CK * 8 + 4;
  extern __shared__ __align__(16) uint8_t slab_smem[];
  __shared__ double wred[8][2];
  __shared__ double cred[kSlabCluster][2];
  cg::cluster_group cluster = cg::this_cluster();
  const int b = blockIdx.x / kSlabCluster;
  const int q = (int)cluster.block_rank();
  const BlockDesc bd = blocks[b];
  const int ld = bd.n_pad;
  if (slab_cluster_smem<T>(ld) > cluster_cap) return;   // the whole cluster: handled by slab_traces_kernel
  const int R = ld / kSlabCluster;
  const int tid = threadIdx.x, ks = tid & 7, rp = tid >> 3;
  T* Xs = reinterpret_cast<T*>(slab_smem);
  const int vlen = (ld / CK) * VS;
  float* const Vb0 = reinterpret_cast<float*>(slab_smem + (size_t)R * ld * sizeof(T));
  auto vb = [&](int i) { return Vb0 + i * vlen; };
  float* Wl = Vb0 + 2 * vlen;
  float* T1 = Wl + R * 8;
  float* T3 = T1 + R * 8;
  float* F1 = T3 + R * 8;

  const NsState s = st[b];
  {
    const T* X = (s.cur ? x1 : x0) + bd.off_mat + (int64_t)q * R * ld;
    const int nvec = (int)((size_t)R * ld * sizeof(T) / 16);
    for (int i = tid; i < nvec; i += blockDim.x)
      cp_async16(reinterpret_cast<uint8_t*>(Xs) + (size_t)i * 16, reinterpret_cast<const uint8_t*>(X) + (size_t)i * 16);
  }
  auto vpos = [&](int k) { return (k / CK) * VS + (k % CK) * 8; };
  // rows of X_q Vin -> local rows (Lout) and/or every rank's copy of Vout
  auto product = [&](const float* Vin, float* Lout, float* Vout) {
    for (int rpi = rp; rpi < R / 2; rpi += 32) {
      float o[2][8];
      slab_rowpair<T>(Xs, ld, Vin, rpi, ks, o);
      if (Lout && ks == 0) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          float4* d = reinterpret_cast<float4*>(Lout + (2 * rpi + i) * 8);
          d[0] = make_float4(o[i][0], o[i][1], o[i][2], o[i][3]);
          d[1] = make_float4(o[i][4], o[i][5], o[i][6], o[i][7]);
        }
      }
      if (Vout) {
        float* dst = cluster.map_shared_rank(Vout, (unsigned)ks);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          float4* d = reinterpret_cast<float4*>(dst + vpos(q * R + 2 * rpi + i));
          d[0] = make_float4(o[i][0], o[i][1], o[i][2], o[i][3]);
          d[1] = make_float4(o[i][4], o[i][5], o[i][6], o[i][7]);
        }
      }
    }
  };
  // local rows (R x 8) -> every rank's copy of Vout
  auto broadcast_rows = [&](const float* Lsrc, float* Vout) {
    for (int e = tid; e < R * 8 * kSlabCluster; e += blockDim.x) {
      const int rank = e / (R * 8), le = e % (R * 8);
      float* dst = cluster.map_shared_rank(Vout, (unsigned)rank);
      dst[vpos(q * R + (le >> 3)) + (le & 7)] = Lsrc[le];
    }
  };
  cp_async_wait_all();
  __syncthreads();

  double sn = 0.0, se = 0.0;
  for (int c0 = 0; c0 < bd.c; c0 += 8) {
    const int cw = min(8, bd.c - c0);
    for (int e = tid; e < R * 8; e += blockDim.x) {
      const int cc = e & 7;
      Wl[e] = (cc < cw) ? w[bd.off_slab + (int64_t)(c0 + cc) * ld + q * R + (e >> 3)] : 0.f;
    }
    __syncthreads();
    broadcast_rows(Wl, vb(0));
    cluster.sync();
    const float* G;
    if (refine <= 0) {
      product(vb(0), T1, nullptr);
      __syncthreads();
      G = T1;
    } else {
      // f(X) V = 1.5 X V - 0.5 X (X (X V)); refine >= 2 evaluates g = f o f as 1.5 F1 - 0.5 F3
      // with F1 = f(X) W, F2 = f(X) F1, F3 = f(X) F2
      const int nf = refine >= 2 ? 3 : 1;
      int cur = 0;
      for (int f = 0; f < nf; ++f) {
        product(vb(cur), T1, vb(cur ^ 1));
        cluster.sync();
        product(vb(cur ^ 1), nullptr, vb(cur));
        cluster.sync();
        product(vb(cur), T3, nullptr);
        __syncthreads();
        for (int e = tid; e < R * 8; e += blockDim.x) {
          const float v = 1.5f * T1[e] + -0.5f * T3[e];
          T3[e] = v;
          if (f == 0) F1[e] = v;
        }
        __syncthreads();
        if (f + 1 < nf) {
          broadcast_rows(T3, vb(cur ^ 1));
          cluster.sync();
          cur ^= 1;
        }
      }
      if (nf > 1) {
        for (int e = tid; e < R * 8; e += blockDim.x) T3[e] = 1.5f * F1[e] + -0.5f * T3[e];
        __syncthreads();
      }
      G = T3;
    }
    for (int e = tid; e < R * 8; e += blockDim.x) {
      const int cc = e & 7;
      if (cc >= cw) continue;
      const int64_t o = bd.off_slab + (int64_t)(c0 + cc) * ld + q * R + (e >> 3);
      const float yv = 0.5f * (Wl[e] - G[e]);
      y[o] = yv;
      sn += (double)lc[o] * (double)yv;
      se += (double)z[o] * (double)yv;
    }
    cluster.sync();   // every rank is done with both slab copies before the next group overwrites them
  }
  for (int o = 16; o; o >>= 1) {
    sn += __shfl_xor_sync(0xffffffffu, sn, o);
    se += __shfl_xor_sync(0xffffffffu, se, o);
  }
  if ((tid & 31) == 0) { wred[tid >> 5][0] = sn; wred[tid >> 5][1] = se; }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, c2 = 0.0;
    for (int i = 0; i < 8; ++i) { a += wred[i][0]; c2 += wred[i][1]; }
    double* dst = cluster.map_shared_rank(&cred[0][0], 0u);
    dst[2 * q] = a;
    dst[2 * q + 1] = c2;
  }
  cluster.sync();
  if (q == 0 && tid == 0) {
    double a = 0.0, c2 = 0.0;
    for (int i = 0; i < kSlabCluster; ++i) { a += cred[i][0]; c2 += cred[i][1]; }
    bn[b] = a;
    be[b] = c2;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) slab_traces_kernel(const BlockDesc* __restrict__ blocks,
                                                          const NsState* __restrict__ st, const T* __restrict__ x0,
                                                          const T* __restrict__ x1, const float* __restrict__ w,
                                                          const float* __restrict__ z, const float* __restrict__ lc,
                                                          float* __restrict__ y, float* __restrict__ tmp,
                                                          int64_t slab_total, int refine, size_t cluster_cap,
                                                          double* __restrict__ bn, double* __restrict__ be) {
  __shared__ float Xs[128][33];
  __shared__ float Vs[32][8];
  __shared__ double red[2][8];
  const BlockDesc bd = blocks[blockIdx.x];
  const int ld = bd.n_pad, c = bd.c;
  if (slab_cluster_smem<T>(ld) <= cluster_cap) return;   // resident in a cluster (slab_cluster_kernel)
  const NsState s = st[blockIdx.x];
  const T* X = (s.cur ? x1 : x0) + bd.off_mat;
  const int64_t len = (int64_t)ld * c;
  const float* W = w + bd.off_slab;
  float* t1 = tmp + bd.off_slab;
  float* t2 = t1 + slab_total;
  float* t3 = t2 + slab_total;
  float* f1 = t3 + slab_total;
  float* f2 = f1 + slab_total;
  float* f3 = f2 + slab_total;
  float* G;
  if (refine <= 0) {
    slab_product<T>(X, ld, c, W, f1, Xs, Vs);
    G = f1;
  } else if (refine == 1) {
    slab_f<T>(X, ld, c, W, f1, t1, t2, t3, Xs, Vs);
    G = f1;
  } else {
    // g = f o f: G = 1.5 F1 - 0.5 F3 with F1 = f(X)W, F2 = f(X)F1, F3 = f(X)F2
    slab_f<T>(X, ld, c, W, f1, t1, t2, t3, Xs, Vs);
    slab_f<T>(X, ld, c, f1, f2, t1, t2, t3, Xs, Vs);
    slab_f<T>(X, ld, c, f2, f3, t1, t2, t3, Xs, Vs);
    slab_axpby(1.5f, f1, -0.5f, f3, f2, len);
    G = f2;
  }
  float* Y = y + bd.off_slab;
  const float* Lc = lc + bd.off_slab;
  const float* Z = z + bd.off_slab;
  double sn = 0.0, se = 0.0;
  for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
    const float yv = 0.5f * (W[i] - G[i]);
    Y[i] = yv;
    sn += (double)Lc[i] * (double)yv;
    se += (double)Z[i] * (double)yv;
  }
  for (int o = 16; o; o >>= 1) {
    sn += __shfl_xor_sync(0xffffffffu, sn, o);
    se += __shfl_xor_sync(0xffffffffu, se, o);
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[0][warp] = sn; red[1][warp] = se; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b2 = 0.0;
    for (int i = 0; i < 8; ++i) { a += red[0][i]; b2 += red[1][i]; }
    bn[blockIdx.x] = a;
    be[blockIdx.x] = b2;
  }
}

// Deterministic FP64 sum of the per-block traces (single CTA).
__global__ void __launch_bounds__(1024) sum_traces_kernel(int n_blocks, const double* __restrict__ bn,
                                                          const double* __restrict__ be, DevFlags* flags) {
  __shared__ double r0[32], r1[32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n_blocks; i += blockDim.x) { a += bn[i]; b += be[i]; }
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) { r0[threadIdx.x >> 5] = a; r1[threadIdx.x >> 5] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { x += r0[i]; y += r1[i]; }
    flags->sum_n = x;
    flags->sum_e = y;
  }
}

// ----------------------------------------------------------------------------------------------
// Step 3: D_b[:, C_b] = L^-T Y, then every stored entry (r, c) of an own column c is written to
// its CSR position transpose[e] (e = the entry (c, r) of row c; the pattern is symmetric).
__device__ __forceinline__ int lower_bound_g(const int32_t* a, int n, int32_t key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// D_b[:, C_b] = L^-T Y into the slab scratch: grid (128-row tile, block), each CTA one row tile for
// every own column (L^-1[k, i] = 0 for k < i, so the sum over k starts at the tile).
template <bool COMP>
__global__ void __launch_bounds__(256) density_slab_kernel(const BlockDesc* __restrict__ blocks,
                                                           const float* __restrict__ linv, const float* __restrict__ y,
                                                           float* __restrict__ dslab) {
  __shared__ float Ls[32][129];
  __shared__ float Vs[32][8];
  const BlockDesc bd = blocks[blockIdx.y];
  const int ld = bd.n_pad, c = bd.c;
  const int r0 = blockIdx.x * 128;
  if (r0 >= ld) return;
  const float* Li = linv + bd.off_mat;
  const float* Y = y + bd.off_slab;
  float* Dsl = dslab + bd.off_slab;
  const int tid = threadIdx.x;
  const int row = tid >> 1, cb = (tid & 1) * 4;
  // a thread's sixteen L^-1 loads of a 32-row step (one 128-byte row segment per warp and load) and
  // its Y load are issued one step ahead, before the current step's products
  auto load_step = [&](int k0, int c0, float (&lv)[16], float& yv) {
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int e = tid + 256 * t;
      lv[t] = Li[(int64_t)(k0 + (e >> 7)) * ld + r0 + (e & 127)];
    }
    const int kk = tid >> 3, cc = tid & 7;
    yv = (c0 + cc < c) ? Y[(int64_t)(c0 + cc) * ld + k0 + kk] : 0.f;
  };
  for (int c0 = 0; c0 < c; c0 += 8) {
    AccSel<COMP> acc[4];
    float lv[16], yv;
    load_step(r0, c0, lv, yv);
    for (int k0 = r0; k0 < ld; k0 += 32) {
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int e = tid + 256 * t;
        Ls[e >> 7][e & 127] = lv[t];
      }
      Vs[tid >> 3][tid & 7] = yv;
      __syncthreads();
      if (k0 + 32 < ld) load_step(k0 + 32, c0, lv, yv);
#pragma unroll 8
      for (int kk = 0; kk < 32; ++kk) {
        const float l = Ls[kk][row];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q].add_prod(l, Vs[kk][cb + q]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (c0 + cb + q < c) Dsl[(int64_t)(c0 + cb + q) * ld + r0 + row] = acc[q].value();
  }
}

// The same back-transform for blocks with many own columns on the mixed paths: a CTA takes 128
// rows x 64 columns of D_b[:, C_b] (grid: row tiles, 64-column tiles, blocks), each thread an 8 x 4
// piece in registers, so L^-1 is read once per 64 columns instead of once per 8 and a step of k
// costs three 16-byte shared loads for 32 FMAs.  Every output takes its terms in ascending k with
// one FMA each, as density_slab_kernel<false> does: the results are the same bit for bit.
__global__ void __launch_bounds__(256) density_slab_wide_kernel(const BlockDesc* __restrict__ blocks,
                                                                const float* __restrict__ linv,
                                                                const float* __restrict__ y,
                                                                float* __restrict__ dslab) {
  __shared__ __align__(16) float Ls[32][128];   // L^-1[k0 + kk][r0 + i]
  __shared__ __align__(16) float Ys[32][64];    // Y[k0 + kk][c0 + j]
  const BlockDesc bd = blocks[blockIdx.z];
  const int ld = bd.n_pad, c = bd.c;
  const int r0 = blockIdx.x * 128, c0 = blockIdx.y * 64;
  if (r0 >= ld || c0 >= c) return;
  const float* Li = linv + bd.off_mat;
  const float* Y = y + bd.off_slab;
  float* Dsl = dslab + bd.off_slab;
  const int tid = threadIdx.x;
  const int rg = tid & 15, cg = tid >> 4;        // rows rg*8 .. +8, columns cg*4 .. +4
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = r0; k0 < ld; k0 += 32) {
    // L^-1 rows k0 .. k0+31, columns r0 .. r0+127: 1,024 float4, four per thread (coalesced rows)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = tid + 256 * t;
      const int kk = e >> 5, i4 = (e & 31) * 4;
      *reinterpret_cast<float4*>(&Ls[kk][i4]) =
          *reinterpret_cast<const float4*>(Li + (int64_t)(k0 + kk) * ld + r0 + i4);
    }
    // Y columns c0 .. c0+63, rows k0 .. k0+31 (column-major slab): 512 float4 along k, two per thread
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int e = tid + 256 * t;
      const int j = e >> 3, k4 = (e & 7) * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (c0 + j < c) v = *reinterpret_cast<const float4*>(Y + (int64_t)(c0 + j) * ld + k0 + k4);
      Ys[k4][j] = v.x;
      Ys[k4 + 1][j] = v.y;
      Ys[k4 + 2][j] = v.z;
      Ys[k4 + 3][j] = v.w;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&Ls[kk][rg * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&Ls[kk][rg * 8 + 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Ys[kk][cg * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int cc = c0 + cg * 4 + j;
    if (cc >= c) continue;
    float* out = Dsl + (int64_t)cc * ld + r0 + rg * 8;
    *reinterpret_cast<float4*>(out) = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
    *reinterpret_cast<float4*>(out + 4) = make_float4(acc[4][j], acc[5][j], acc[6][j], acc[7][j]);
  }
}

// Step 3: every stored entry (r, c) of an own column c is written to its CSR position transpose[e]
// (e = the entry (c, r) of row c; the pattern is symmetric) from the block's D slab.
__global__ void __launch_bounds__(256) density_scatter_kernel(const BlockDesc* __restrict__ blocks,
                                                              const int32_t* __restrict__ idx_pool,
                                                              const int32_t* __restrict__ blk_cols,
                                                              const float* __restrict__ dslab,
                                                              const int64_t* __restrict__ row_ptr,
                                                              const int32_t* __restrict__ col,
                                                              const int64_t* __restrict__ transpose,
                                                              double* __restrict__ dval, DevFlags* flags) {
  const BlockDesc bd = blocks[blockIdx.x];
  const int ld = bd.n_pad, c = bd.c, n = bd.n;
  const float* Dsl = dslab + bd.off_slab;
  const int32_t* I = idx_pool + bd.off_idx;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = warp; j < c; j += 8) {
    const int32_t cg = blk_cols[bd.col0 + j];
    const int64_t e0 = row_ptr[cg], e1 = row_ptr[cg + 1];
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      const int32_t r = col[e];
      const int p = lower_bound_g(I, n, r);
      if (p < n && I[p] == r) dval[transpose[e]] = (double)Dsl[(int64_t)j * ld + p];
      else set_error(flags, NOLSM_EINVAL);
    }
  }
}

// E = sum_e D[e] * H[e]  (H symmetric on a symmetric pattern: H_ji = H_ij), FP64, two passes.
__global__ void __launch_bounds__(256) dot_kernel(int64_t nnz, const double* __restrict__ a, const double* __restrict__ b,
                                                  double* __restrict__ partial) {
  __shared__ double red[8];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    partial[blockIdx.x] = t;
  }
}

__global__ void sum_partials_kernel(int n, const double* __restrict__ partial, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += partial[i];
    *out = s;
  }
}

}  // namespace

// ------------------------------------------------------------------------------------------------ launchers

cudaError_t launch_sgemm_nt(nolsm_ctx* ctx, const float* a, const float* b, float* c, int a_lower, int b_lower,
                            int sym) {
  // host-built tile list over all blocks (build phase only)
  std::vector<Tile> tl;
  for (int32_t i = 0; i < ctx->n_blocks; ++i) {
    const BlockDesc& bd = ctx->h_blocks[i];
    for (int m0 = 0; m0 < bd.n_pad; m0 += BM)
      for (int n0 = sym ? m0 : 0; n0 < bd.n_pad; n0 += BN) {
        int kend = bd.n_pad;
        if (a_lower) kend = std::min(kend, m0 + BM);
        if (b_lower) kend = std::min(kend, n0 + BN);
        tl.push_back(Tile{i, m0, n0, kend});
      }
  }
  if ((int64_t)tl.size() > ctx->max_tiles) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemcpyAsync(ctx->d_tiles, tl.data(), tl.size() * sizeof(Tile), cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(ctx->stream);   // tl is a host temporary
  if (e != cudaSuccess) return e;
  const bool two = ctx->opt.precision == NOLSM_PREC_FP32;
  const int grid = ctx->num_sms * (two ? 1 : 2);   // persistent: one wave of resident CTAs
  if (sym && two)
    sgemm_nt_kernel<3, true><<<grid, 256, 0, ctx->stream>>>(ctx->d_tiles, nullptr, (int)tl.size(), ctx->d_blocks, a,
                                                            b, c, nullptr, nullptr, nullptr, nullptr, nullptr);
  else if (sym)
    sgemm_nt_kernel<3, false><<<grid, 256, 0, ctx->stream>>>(ctx->d_tiles, nullptr, (int)tl.size(), ctx->d_blocks, a,
                                                             b, c, nullptr, nullptr, nullptr, nullptr, nullptr);
  else if (two)
    sgemm_nt_kernel<0, true><<<grid, 256, 0, ctx->stream>>>(ctx->d_tiles, nullptr, (int)tl.size(), ctx->d_blocks, a,
                                                            b, c, nullptr, nullptr, nullptr, nullptr, nullptr);
  else
    sgemm_nt_kernel<0, false><<<grid, 256, 0, ctx->stream>>>(ctx->d_tiles, nullptr, (int)tl.size(), ctx->d_blocks, a,
                                                             b, c, nullptr, nullptr, nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_ns_init(nolsm_ctx* ctx, double mu, int half, int mode, const float* lz, const float* pred,
                           bool fill) {
  const float l_floor = scaled_l_floor(ctx);
  const float l0 = std::max((float)ctx->opt.lower_bound, l_floor);
  ns_state_kernel<<<(ctx->n_blocks + 255) / 256, 256, 0, ctx->stream>>>(
      ctx->n_blocks, ctx->d_lo, ctx->d_hi, mu, (float)ctx->opt.alpha_margin, l0, l_floor, ctx->opt.scaled, mode, lz, pred,
      ctx->d_state, ctx->d_resacc, ctx->d_flags);
  if (!fill) return cudaGetLastError();   // the persistent product kernel forms X_0 itself
  const dim3 g(64, ctx->n_blocks);
  if (half == 0)
    ns_fill_kernel<float><<<g, 256, 0, ctx->stream>>>(ctx->d_blocks, ctx->d_a0, ctx->d_state, mu, (float*)ctx->d_x[0]);
  else if (half == 1)
    ns_fill_kernel<__half><<<g, 256, 0, ctx->stream>>>(ctx->d_blocks, ctx->d_a0, ctx->d_state, mu, (__half*)ctx->d_x[0]);
  else
    ns_fill_kernel<__nv_bfloat16><<<g, 256, 0, ctx->stream>>>(ctx->d_blocks, ctx->d_a0, ctx->d_state, mu,
                                                              (__nv_bfloat16*)ctx->d_x[0]);
  return cudaGetLastError();
}

cudaError_t launch_ns_tiles_n(nolsm_ctx* ctx, int tile_n) {
  ns_tiles_kernel<<<1, 1024, 0, ctx->stream>>>(ctx->n_blocks, ctx->d_blocks, ctx->d_state, tile_n, ctx->d_tiles,
                                               ctx->d_flags);
  return cudaGetLastError();
}

cudaError_t launch_ns_tiles(nolsm_ctx* ctx) { return launch_ns_tiles_n(ctx, BN); }

cudaError_t launch_ns_check_impl(nolsm_ctx* ctx, const float* tol_b, int detect_divergence) {
  ns_check_kernel<<<(ctx->n_blocks + 255) / 256, 256, 0, ctx->stream>>>(ctx->n_blocks, ctx->d_blocks, ctx->d_state,
                                                                        ctx->d_resacc, tol_b, ctx->opt.max_iter,
                                                                        detect_divergence, ctx->d_flags);
  return cudaGetLastError();
}

cudaError_t launch_ns_check_impl(nolsm_ctx* ctx, const float* tol_b) { return launch_ns_check_impl(ctx, tol_b, 0); }

// mu is read on the device from DevFlags::mu (set_loop_mu), so that the launches also serve a captured
// iteration graph whatever the chemical potential
cudaError_t launch_ns_restart(nolsm_ctx* ctx, int half) {
  const dim3 g(ctx->n_blocks);
  const float margin = (float)ctx->opt.alpha_margin;
  const double* mu = &ctx->d_flags->mu;
  if (half == 0)
    ns_restart_fill_kernel<float><<<g, 256, 0, ctx->stream>>>(ctx->d_blocks, ctx->d_a0, ctx->d_state, ctx->d_lo,
                                                              ctx->d_hi, mu, margin, (float*)ctx->d_x[0]);
  else if (half == 1)
    ns_restart_fill_kernel<__half><<<g, 256, 0, ctx->stream>>>(ctx->d_blocks, ctx->d_a0, ctx->d_state, ctx->d_lo,
                                                               ctx->d_hi, mu, margin, (__half*)ctx->d_x[0]);
  else
    ns_restart_fill_kernel<__nv_bfloat16><<<g, 256, 0, ctx->stream>>>(ctx->d_blocks, ctx->d_a0, ctx->d_state,
                                                                      ctx->d_lo, ctx->d_hi, mu, margin,
                                                                      (__nv_bfloat16*)ctx->d_x[0]);
  ns_restart_state_kernel<<<(ctx->n_blocks + 255) / 256, 256, 0, ctx->stream>>>(
      ctx->n_blocks, ctx->d_lo, ctx->d_hi, mu, margin, std::max((float)ctx->opt.lower_bound, scaled_l_floor(ctx)),
      ctx->opt.scaled, ctx->d_state,
      ctx->d_resacc);
  return cudaGetLastError();
}

cudaError_t launch_ns_advance(nolsm_ctx* ctx) {
  ns_advance_kernel<<<(ctx->n_blocks + 255) / 256, 256, 0, ctx->stream>>>(ctx->n_blocks, ctx->d_state);
  return cudaGetLastError();
}

cudaError_t launch_gemm_f32(nolsm_ctx* ctx, int phase) {
  const int grid = ctx->num_sms;   // one resident CTA per SM (two-level summation)
  const int32_t* nt = &ctx->d_flags->n_tiles;
  if (phase == 1)
    sgemm_nt_kernel<1, true><<<grid, 256, 0, ctx->stream>>>(ctx->d_tiles, nt, 0, ctx->d_blocks, nullptr, nullptr, nullptr,
                                                      (float*)ctx->d_x[0], (float*)ctx->d_x[1], (float*)ctx->d_b,
                                                      ctx->d_state, ctx->d_resacc);
  else
    sgemm_nt_kernel<2, true><<<grid, 256, 0, ctx->stream>>>(ctx->d_tiles, nt, 0, ctx->d_blocks, nullptr, nullptr, nullptr,
                                                      (float*)ctx->d_x[0], (float*)ctx->d_x[1], (float*)ctx->d_b,
                                                      ctx->d_state, ctx->d_resacc);
  return cudaGetLastError();
}

namespace {
template <typename T>
cudaError_t slab_launch(nolsm_ctx* ctx) {
  const int r = ctx->opt.refine_iters;
  // dynamic shared memory of the cluster kernel: the largest resident block that fits
  size_t cap = 0;
  bool any_big = false;
  for (const BlockDesc& bd : ctx->h_blocks) {
    const size_t need = slab_cluster_smem<T>(bd.n_pad);
    if (need <= kSmemOptin) cap = std::max(cap, need);
    else any_big = true;
  }
  const T* x0 = (const T*)ctx->d_x[0];
  const T* x1 = (const T*)ctx->d_x[1];
  if (cap > 0) {
    cudaError_t e = cudaFuncSetAttribute(slab_cluster_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
    if (e != cudaSuccess) return e;
    slab_cluster_kernel<T><<<ctx->n_blocks * kSlabCluster, 256, cap, ctx->stream>>>(
        ctx->d_blocks, ctx->d_state, x0, x1, ctx->d_w, ctx->d_z, ctx->d_lc, ctx->d_y, r, cap, ctx->d_bn, ctx->d_be);
    ctx->n_launches += 1;
  }
  if (any_big) {
    slab_traces_kernel<T><<<ctx->n_blocks, 256, 0, ctx->stream>>>(ctx->d_blocks, ctx->d_state, x0, x1, ctx->d_w,
                                                                 ctx->d_z, ctx->d_lc, ctx->d_y, ctx->d_tmp,
                                                                 ctx->sum_slab, r, cap, ctx->d_bn, ctx->d_be);
    ctx->n_launches += 1;
  }
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_slab_traces(nolsm_ctx* ctx, int half) {
  const bool tc = half != 0 && ctx->opt.refine_path == NOLSM_REFINE_TENSOR;
  cudaError_t e = tc ? launch_slab_tc(ctx)
                     : half == 0 ? slab_launch<float>(ctx)
                                 : half == 1 ? slab_launch<__half>(ctx) : slab_launch<__nv_bfloat16>(ctx);
  if (e != cudaSuccess) return e;
  // per-block traces, or per own-column piece on the tensor-core path
  const int n = tc ? ctx->n_units_narrow + ctx->n_units_wide : ctx->n_blocks;
  ctx->traces_per_unit = tc;
  sum_traces_kernel<<<1, 1024, 0, ctx->stream>>>(n, ctx->d_bn, ctx->d_be, ctx->d_flags);
  return cudaGetLastError();
}

cudaError_t launch_density(nolsm_ctx* ctx) {
  // the chunked solve scatters every chunk into the caller's D, cleared once per pass
  double* dst = ctx->d_dval_target ? ctx->d_dval_target : ctx->d_dval;
  if (!ctx->d_dval_target) {
    cudaError_t e = cudaMemsetAsync(ctx->d_dval, 0, sizeof(double) * ctx->nnz, ctx->stream);
    if (e != cudaSuccess) return e;
  }
  int max_pad = 0, max_c = 0;
  for (const auto& bd : ctx->h_blocks) {
    max_pad = std::max(max_pad, bd.n_pad);
    max_c = std::max(max_c, bd.c);
  }
  const dim3 g(max_pad / 128, ctx->n_blocks);
  if (ctx->opt.precision == NOLSM_PREC_FP32)
    density_slab_kernel<true><<<g, 256, 0, ctx->stream>>>(ctx->d_blocks, ctx->d_linv, ctx->d_y, ctx->d_tmp);
  else if (max_c >= 32)   // many own columns: 64-column tiles (same results as the narrow kernel)
    density_slab_wide_kernel<<<dim3(max_pad / 128, (max_c + 63) / 64, ctx->n_blocks), 256, 0, ctx->stream>>>(
        ctx->d_blocks, ctx->d_linv, ctx->d_y, ctx->d_tmp);
  else
    density_slab_kernel<false><<<g, 256, 0, ctx->stream>>>(ctx->d_blocks, ctx->d_linv, ctx->d_y, ctx->d_tmp);
  density_scatter_kernel<<<ctx->n_blocks, 256, 0, ctx->stream>>>(ctx->d_blocks, ctx->d_idx, ctx->d_blk_cols, ctx->d_tmp,
                                                                 ctx->d_row_ptr, ctx->d_col, ctx->d_transpose,
                                                                 dst, ctx->d_flags);
  ctx->n_launches += 1;   // the second of the two (the caller counts one)
  return cudaGetLastError();
}

cudaError_t launch_band_energy(nolsm_ctx* ctx) {
  const int grid = 1024;
  double* partial = reinterpret_cast<double*>(ctx->d_tmp);   // scratch: grid doubles
  const double* d = ctx->d_dval_target ? ctx->d_dval_target : ctx->d_dval;
  dot_kernel<<<grid, 256, 0, ctx->stream>>>(ctx->nnz, d, ctx->d_hval, partial);
  sum_partials_kernel<<<1, 32, 0, ctx->stream>>>(grid, partial, &ctx->d_flags->energy);
  return cudaGetLastError();
}


namespace {
__global__ void set_loop_mu_kernel(DevFlags* f, double mu) { f->mu = mu; }

// End of one captured iteration: run the next while no error is recorded, some block was still
// iterating at this iteration's start and the iteration budget is not spent.
__global__ void loop_cond_kernel(cudaGraphConditionalHandle h, DevFlags* f, int max_iter) {
  const int it = ++f->loop_iter;
  cudaGraphSetConditional(h, (f->error == 0 && f->n_active > 0 && it <= max_iter) ? 1u : 0u);
}
__global__ void loop_reset_kernel(DevFlags* f) { f->loop_iter = 0; }
}  // namespace

cudaError_t launch_set_loop_mu(nolsm_ctx* ctx, double mu) {
  set_loop_mu_kernel<<<1, 1, 0, ctx->stream>>>(ctx->d_flags, mu);
  return cudaGetLastError();
}
cudaError_t launch_loop_cond(nolsm_ctx* ctx, cudaGraphConditionalHandle h) {
  loop_cond_kernel<<<1, 1, 0, ctx->stream>>>(h, ctx->d_flags, ctx->opt.max_iter);
  return cudaGetLastError();
}
cudaError_t launch_loop_reset(nolsm_ctx* ctx) {
  loop_reset_kernel<<<1, 1, 0, ctx->stream>>>(ctx->d_flags);
  return cudaGetLastError();
}

}  // namespace nolsm
