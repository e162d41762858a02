// Spectral bounds beyond Gershgorin, and the learned predictor that sets the sign iteration's
// scaling: per-block features, Lanczos on A0 or on |A0 - mu|, and the kernels of a small
// network 32 -> 128 -> 128 -> 3 (GELU) -- its gradient (forward + backward), Adam, and inference
// with BF16 weights and FP32 accumulation.
//
// Outputs of the network for block b at chemical potential mu: lambda_min(A0), lambda_max(A0),
// and log10 of the distance from mu to the nearest eigenvalue of A0.  The first two tighten the
// scale alpha of X_0 = (A0 - mu)/alpha, the third the lower bound l of the scaled iteration.
#include "internal.h"

#include <cfloat>

namespace nolsm {

constexpr int NI = 32, NH = 128, NO = 3;
constexpr int OFF_W1 = 0, OFF_B1 = NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH,
              OFF_B3 = OFF_W3 + NO * NH, N_PARAMS = OFF_B3 + NO;
constexpr int N_NORM = 2 * NI + 2 * NO;     // x mean, x std, y mean, y std
constexpr int SPC = 32;                     // samples per CTA

namespace {

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__device__ __forceinline__ float block_sum(float v, float* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  float t = 0.f;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

// ------------------------------------------------------------------------------------------ features
// 32 numbers per block, all O(n^2) from A0 and mu (see the list in nolsm_block_features).
// The same pass over A0 also yields the Gershgorin bounds [min_i a_ii - R_i, max_i a_ii + R_i] of the
// real n x n part (FP32 sums, each radius rounded up by a relative n 2^-23 so that the discs stay
// enclosing; written to glo / ghi) and the per-row diagonal and radius; the features take those bounds.
__global__ void __launch_bounds__(256) features_kernel(const BlockDesc* __restrict__ blocks, const float* __restrict__ a0,
                                                       double* __restrict__ glo, double* __restrict__ ghi,
                                                       double mu, float margin, float* __restrict__ feat,
                                                       float* __restrict__ row_diag, float* __restrict__ row_rad,
                                                       DevFlags* flags) {
  __shared__ float red[8];
  const BlockDesc bd = blocks[blockIdx.x];
  const int n = bd.n, ld = bd.n_pad;
  const float* A = a0 + bd.off_mat;
  const float m = (float)mu;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float s_d = 0, s_d2 = 0, s_d3 = 0, s_d4 = 0, mn_d = FLT_MAX, mx_d = -FLT_MAX;
  float s_off2 = 0, s_r = 0, s_r2 = 0, mx_r = 0, s_abs = 0, mx_abs = 0;
  float below = 0, near05 = 0, near1 = 0, mn_dist = FLT_MAX, in_disc = 0, s_edge = 0, mn_edge = FLT_MAX;
  float wlo = FLT_MAX, whi = -FLT_MAX;
  const float up = 1.f + (float)n * 1.2e-7f;   // Gershgorin radius rounded up by a relative n 2^-23
  for (int r = warp; r < n; r += 8) {
    float rad = 0.f, off2 = 0.f, mabs = 0.f, dg = 0.f;
    // 16-byte loads, four in flight per lane; the padding columns of A0 are zero and add nothing
    const float4* Ar = reinterpret_cast<const float4*>(A + (int64_t)r * ld);
    for (int c4 = lane; c4 < ld / 4; c4 += 4 * 32) {
      float4 v4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v4[u] = c4 + 32 * u < ld / 4 ? __ldg(Ar + c4 + 32 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float vv[4] = {v4[u].x, v4[u].y, v4[u].z, v4[u].w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = 4 * (c4 + 32 * u) + j;
          const float v = vv[j];
          if (c == r) dg = v;
          else { rad += fabsf(v); off2 += v * v; mabs = fmaxf(mabs, fabsf(v)); }
        }
      }
    }
    for (int o = 16; o; o >>= 1) {
      rad += __shfl_xor_sync(0xffffffffu, rad, o);
      off2 += __shfl_xor_sync(0xffffffffu, off2, o);
      dg += __shfl_xor_sync(0xffffffffu, dg, o);
      mabs = fmaxf(mabs, __shfl_xor_sync(0xffffffffu, mabs, o));
    }
    if (lane == 0) {
      row_diag[bd.off_idx + r] = dg;      // per-row data for features at any mu (index-set stride)
      row_rad[bd.off_idx + r] = rad;
      const float ru = rad * up;
      wlo = fminf(wlo, dg - ru);
      whi = fmaxf(whi, dg + ru);
    }
    if (lane == 0) {
      s_d += dg; s_d2 += dg * dg; s_d3 += dg * dg * dg; s_d4 += dg * dg * dg * dg;
      mn_d = fminf(mn_d, dg); mx_d = fmaxf(mx_d, dg);
      s_off2 += off2; s_r += rad; s_r2 += rad * rad; mx_r = fmaxf(mx_r, rad);
      s_abs += rad; mx_abs = fmaxf(mx_abs, mabs);
      const float dm = dg - m;
      below += (dm < 0.f); near05 += (fabsf(dm) < 0.05f); near1 += (fabsf(dm) < 0.1f);
      mn_dist = fminf(mn_dist, fabsf(dm));
      in_disc += (fabsf(dm) <= rad);
      const float edge = fabsf(dm) - rad;
      s_edge += edge; mn_edge = fminf(mn_edge, edge);
    }
  }
  // reductions (lane 0 of each warp holds partial values)
  __shared__ float part[24][8];
  if (lane == 0) {
    const float v[24] = {s_d, s_d2, s_d3, s_d4, -mn_d, mx_d, s_off2, s_r, s_r2, mx_r, s_abs, mx_abs,
                         below, near05, near1, -mn_dist, in_disc, s_edge, -mn_edge, -wlo, whi, 0, 0, 0};
    for (int i = 0; i < 24; ++i) part[i][warp] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < 24) {
    const int i = threadIdx.x;
    const bool is_max = (i == 4 || i == 5 || i == 9 || i == 11 || i == 15 || i == 18 || i == 19 || i == 20);
    float t = is_max ? -FLT_MAX : 0.f;
    for (int w = 0; w < 8; ++w) t = is_max ? fmaxf(t, part[i][w]) : t + part[i][w];
    part[i][0] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const float nf = (float)n;
    const float md = part[0][0] / nf, vd = fmaxf(part[1][0] / nf - md * md, 0.f), sd = sqrtf(vd);
    const float m3 = part[2][0] / nf - 3 * md * part[1][0] / nf + 2 * md * md * md;
    const float m4 = part[3][0] / nf - 4 * md * part[2][0] / nf + 6 * md * md * part[1][0] / nf - 3 * md * md * md * md;
    const float tr2 = (part[1][0] + part[6][0]) / nf;     // Tr(A0^2)/n
    const float lo = -part[19][0], hi = part[20][0];
    if (!isfinite(lo) || !isfinite(hi)) atomicCAS(&flags->error, 0, (int)NOLSM_ENONFINITE);
    glo[blockIdx.x] = lo;
    ghi[blockIdx.x] = hi;
    const float alpha_g = fmaxf(fabsf(hi - m), fabsf(m - lo)) * (1.f + margin);
    const float mr = part[7][0] / nf;
    float* f = feat + (int64_t)blockIdx.x * NI;
    f[0] = nf / 512.f;
    f[1] = (float)bd.c / nf;
    f[2] = m;
    f[3] = lo;
    f[4] = hi;
    f[5] = md;
    f[6] = sd;
    f[7] = -part[4][0];
    f[8] = part[5][0];
    f[9] = sqrtf(part[6][0] / nf);
    f[10] = mr;
    f[11] = part[9][0];
    f[12] = sqrtf(fmaxf(part[8][0] / nf - mr * mr, 0.f));
    f[13] = tr2;
    f[14] = md;
    f[15] = sqrtf(fmaxf(tr2 - md * md, 0.f));
    f[16] = md - m;
    f[17] = -part[15][0];
    f[18] = part[12][0] / nf;
    f[19] = part[13][0] / nf;
    f[20] = part[14][0] / nf;
    f[21] = part[10][0] / (nf * fmaxf(nf - 1.f, 1.f));
    f[22] = part[11][0];
    f[23] = (sd > 0.f) ? m3 / (sd * sd * sd) : 0.f;
    f[24] = (vd > 0.f) ? m4 / (vd * vd) : 0.f;
    f[25] = part[16][0] / nf;
    f[26] = -part[18][0];
    f[27] = part[17][0] / nf;
    f[28] = (hi > lo) ? (m - lo) / (hi - lo) : 0.5f;
    f[29] = log10f(fmaxf(alpha_g, 1e-6f));
    f[30] = (float)bd.c / 100.f;
    f[31] = 1.f;
  }
}

// Features at a new mu from the mu-independent ones (computed once per build) and the per-row
// diagonal and Gershgorin radius: O(n) per block instead of O(n^2).
__global__ void __launch_bounds__(128) features_mu_kernel(const BlockDesc* __restrict__ blocks,
                                                          const float* __restrict__ fstatic,
                                                          const float* __restrict__ row_diag,
                                                          const float* __restrict__ row_rad, double mu, float margin,
                                                          float* __restrict__ feat) {
  __shared__ float red[4];
  const BlockDesc bd = blocks[blockIdx.x];
  const int n = bd.n;
  const float m = (float)mu;
  const float* D = row_diag + bd.off_idx;
  const float* R = row_rad + bd.off_idx;
  float mn = FLT_MAX, below = 0, n05 = 0, n1 = 0, disc = 0, medge = FLT_MAX, sedge = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float dm = D[i] - m, ad = fabsf(dm), e = ad - R[i];
    mn = fminf(mn, ad);
    below += (dm < 0.f);
    n05 += (ad < 0.05f);
    n1 += (ad < 0.1f);
    disc += (ad <= R[i]);
    medge = fminf(medge, e);
    sedge += e;
  }
  for (int o = 16; o; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    medge = fminf(medge, __shfl_xor_sync(0xffffffffu, medge, o));
  }
  below = block_sum(below, red);
  n05 = block_sum(n05, red);
  n1 = block_sum(n1, red);
  disc = block_sum(disc, red);
  sedge = block_sum(sedge, red);
  __shared__ float smn[4], sme[4];
  if ((threadIdx.x & 31) == 0) { smn[threadIdx.x >> 5] = mn; sme[threadIdx.x >> 5] = medge; }
  __syncthreads();
  const float* fs = fstatic + (int64_t)blockIdx.x * NI;
  float* f = feat + (int64_t)blockIdx.x * NI;
  if (threadIdx.x < NI) f[threadIdx.x] = fs[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    const float nf = (float)n;
    float mn_all = FLT_MAX, me_all = FLT_MAX;
    for (int w = 0; w < 4; ++w) { mn_all = fminf(mn_all, smn[w]); me_all = fminf(me_all, sme[w]); }
    const float lo = fs[3], hi = fs[4];
    f[2] = m;
    f[16] = fs[5] - m;
    f[17] = mn_all;
    f[18] = below / nf;
    f[19] = n05 / nf;
    f[20] = n1 / nf;
    f[25] = disc / nf;
    f[26] = me_all;
    f[27] = sedge / nf;
    f[28] = (hi > lo) ? (m - lo) / (hi - lo) : 0.5f;
    f[29] = log10f(fmaxf(fmaxf(fabsf(hi - m), fabsf(m - lo)) * (1.f + margin), 1e-6f));
  }
}

// ------------------------------------------------------------------------------------------ Lanczos
// One CTA per block; k steps with full (twice-repeated classical Gram-Schmidt) reorthogonalisation
// against the stored basis.  op 0: v -> A0 v.  op 1: v -> X (A0 - mu) v with X the converged sign
// iterate (|A0 - mu| = sign(A0 - mu)(A0 - mu) for commuting symmetric factors).  Extreme Ritz values
// of the tridiagonal matrix by Sturm-count bisection.  out[4b..]: theta_min, theta_max, last beta,
// steps taken.
template <typename TX>
__device__ float ld_x(const TX* p);
template <> __device__ float ld_x<float>(const float* p) { return *p; }
template <> __device__ float ld_x<__half>(const __half* p) { return __half2float(*p); }
template <> __device__ float ld_x<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }

__device__ int sturm_below(const float* al, const float* be, int k, float x) {
  // number of eigenvalues of the k x k tridiagonal (al, be) below x
  int cnt = 0;
  float d = al[0] - x;
  if (d < 0.f) ++cnt;
  for (int i = 1; i < k; ++i) {
    const float dd = (fabsf(d) < 1e-30f) ? 1e-30f : d;
    d = al[i] - x - be[i] * be[i] / dd;
    if (d < 0.f) ++cnt;
  }
  return cnt;
}

template <typename TX>
__global__ void __launch_bounds__(256) lanczos_kernel(const BlockDesc* __restrict__ blocks, const float* __restrict__ a0,
                                                      const NsState* __restrict__ st, const TX* __restrict__ x0,
                                                      const TX* __restrict__ x1, double mu, int op, int k,
                                                      float* __restrict__ basis, int64_t basis_stride,
                                                      float* __restrict__ out) {
  extern __shared__ float sv[];          // v (n_pad) | u (n_pad)
  __shared__ float red[8];
  __shared__ float al[64], be[65];
  const BlockDesc bd = blocks[blockIdx.x];
  const int n = bd.n, ld = bd.n_pad;
  const float* A = a0 + bd.off_mat;
  const TX* X = (st[blockIdx.x].cur ? x1 : x0) + bd.off_mat;
  float* V = basis + (int64_t)blockIdx.x * basis_stride;    // k+1 vectors of length ld
  float* v = sv;
  float* u = sv + ld;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float m = (float)mu;
  // start vector: deterministic, non-zero in every component
  float nrm = 0.f;
  for (int i = threadIdx.x; i < ld; i += blockDim.x) {
    const float val = (i < n) ? 1.f + 0.5f * sinf(0.7f * (float)i + 1.3f) : 0.f;
    v[i] = val;
    nrm += val * val;
  }
  nrm = sqrtf(block_sum(nrm, red));
  for (int i = threadIdx.x; i < ld; i += blockDim.x) { v[i] /= nrm; V[i] = v[i]; }
  __syncthreads();
  if (threadIdx.x == 0) be[0] = 0.f;
  int steps = 0;
  for (int j = 0; j < k; ++j) {
    // u = Op v
    for (int r = warp; r < ld; r += 8) {
      float acc = 0.f;
      if (r < n)
        for (int c = lane; c < n; c += 32) acc += A[(int64_t)r * ld + c] * v[c];
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) u[r] = (r < n) ? acc - (op == 1 ? m * v[r] : 0.f) : 0.f;
    }
    __syncthreads();
    if (op == 1) {
      // u <- X u (X symmetric, identity on the padding which u does not touch)
      float* w = V + (int64_t)(j + 1) * ld;                 // temporary: next basis slot
      for (int r = warp; r < ld; r += 8) {
        float acc = 0.f;
        if (r < n)
          for (int c = lane; c < n; c += 32) acc += ld_x<TX>(X + (int64_t)r * ld + c) * u[c];
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) w[r] = (r < n) ? acc : 0.f;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < ld; i += blockDim.x) u[i] = w[i];
      __syncthreads();
    }
    float a = 0.f;
    for (int i = threadIdx.x; i < ld; i += blockDim.x) a += u[i] * v[i];
    a = block_sum(a, red);
    // orthogonalise against the whole basis, twice
    for (int pass = 0; pass < 2; ++pass)
      for (int q = 0; q <= j; ++q) {
        const float* Vq = V + (int64_t)q * ld;
        float c = 0.f;
        for (int i = threadIdx.x; i < ld; i += blockDim.x) c += u[i] * Vq[i];
        c = block_sum(c, red);
        for (int i = threadIdx.x; i < ld; i += blockDim.x) u[i] -= c * Vq[i];
        __syncthreads();
      }
    float b = 0.f;
    for (int i = threadIdx.x; i < ld; i += blockDim.x) b += u[i] * u[i];
    b = sqrtf(block_sum(b, red));
    if (threadIdx.x == 0) { al[j] = a; be[j + 1] = b; }
    steps = j + 1;
    if (!(b > 1e-6f * fabsf(a) + 1e-20f) || j + 1 == k) break;
    for (int i = threadIdx.x; i < ld; i += blockDim.x) {
      v[i] = u[i] / b;
      V[(int64_t)(j + 1) * ld + i] = v[i];
    }
    __syncthreads();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // Gershgorin interval of T, then bisection for the smallest and largest eigenvalues
    float lo = FLT_MAX, hi = -FLT_MAX;
    for (int i = 0; i < steps; ++i) {
      const float r = fabsf(be[i]) * (i > 0) + (i + 1 < steps ? fabsf(be[i + 1]) : 0.f);
      lo = fminf(lo, al[i] - r);
      hi = fmaxf(hi, al[i] + r);
    }
    float a1 = lo, b1 = hi, a2 = lo, b2 = hi;
    for (int it = 0; it < 60; ++it) {
      const float mid1 = 0.5f * (a1 + b1);
      if (sturm_below(al, be, steps, mid1) >= 1) b1 = mid1; else a1 = mid1;
      const float mid2 = 0.5f * (a2 + b2);
      if (sturm_below(al, be, steps, mid2) >= steps) b2 = mid2; else a2 = mid2;
    }
    float* o = out + (int64_t)blockIdx.x * 4;
    o[0] = 0.5f * (a1 + b1);
    o[1] = 0.5f * (a2 + b2);
    o[2] = be[steps];
    o[3] = (float)steps;
  }
}

// ------------------------------------------------------------------------------------------ network
// Gradient of the mean weighted squared error over B samples (normalised inputs and targets).
// One CTA of 128 threads per SPC samples; thread j owns hidden unit j.  Weights and the CTA's
// gradient sums live in shared memory with row strides 33 / 129 so that row and column accesses
// are both free of bank conflicts; sums go to the global gradient with one atomicAdd per entry.
__global__ void __launch_bounds__(128) mlp_grad_kernel(const float* __restrict__ P, const float* __restrict__ norm,
                                                       const float* __restrict__ X, const float* __restrict__ T,
                                                       float lw0, float lw1, float lw2, int B,
                                                       float* __restrict__ grad, double* __restrict__ loss) {
  extern __shared__ float sm[];
  float* W1 = sm;                  // [128][33]
  float* W2 = W1 + NH * 33;        // [128][129]
  float* W3 = W2 + NH * 129;       // [3][128]
  float* G1 = W3 + NO * NH;        // [128][33]
  float* G2 = G1 + NH * 33;        // [128][129]
  float* G3 = G2 + NH * 129;       // [3][128]
  float* xs = G3 + NO * NH;        // 32
  float* a1 = xs + NI;             // 128
  float* a2 = a1 + NH;             // 128
  float* d2 = a2 + NH;             // 128
  float* yv = d2 + NH;             // 4
  float* dy = yv + 4;              // 4
  const int j = threadIdx.x, lane = j & 31, warp = j >> 5;
  for (int e = j; e < NH * NI; e += NH) { W1[(e / NI) * 33 + e % NI] = P[OFF_W1 + e]; G1[(e / NI) * 33 + e % NI] = 0.f; }
  for (int e = j; e < NH * NH; e += NH) { W2[(e / NH) * 129 + e % NH] = P[OFF_W2 + e]; G2[(e / NH) * 129 + e % NH] = 0.f; }
  for (int e = j; e < NO * NH; e += NH) { W3[e] = P[OFF_W3 + e]; G3[e] = 0.f; }
  const float b1 = P[OFF_B1 + j], b2 = P[OFF_B2 + j];
  const float lw[3] = {lw0, lw1, lw2};
  float gb1 = 0.f, gb2 = 0.f, gb3 = 0.f;
  double lsum = 0.0;
  __syncthreads();
  const int s0 = blockIdx.x * SPC, s1 = min(s0 + SPC, B);
  for (int s = s0; s < s1; ++s) {
    if (j < NI) xs[j] = (X[(int64_t)s * NI + j] - norm[j]) / norm[NI + j];
    __syncthreads();
    float h1 = b1;
    for (int i = 0; i < NI; ++i) h1 = fmaf(W1[j * 33 + i], xs[i], h1);
    a1[j] = gelu(h1);
    __syncthreads();
    float h2 = b2;
    for (int i = 0; i < NH; ++i) h2 = fmaf(W2[j * 129 + i], a1[i], h2);
    a2[j] = gelu(h2);
    __syncthreads();
    if (warp < NO) {
      float acc = 0.f;
      for (int i = lane; i < NH; i += 32) acc = fmaf(W3[warp * NH + i], a2[i], acc);
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) yv[warp] = acc + P[OFF_B3 + warp];
    }
    __syncthreads();
    if (j < NO) {
      const float tn = (T[(int64_t)s * NO + j] - norm[2 * NI + j]) / norm[2 * NI + NO + j];
      const float e = yv[j] - tn;
      dy[j] = lw[j] * e / (float)B;
      lsum += 0.5 * lw[j] * (double)e * e / B;
      gb3 += dy[j];
    }
    __syncthreads();
    const float dy0 = dy[0], dy1 = dy[1], dy2 = dy[2];
    const float a2j = a2[j];
    G3[j] += dy0 * a2j;
    G3[NH + j] += dy1 * a2j;
    G3[2 * NH + j] += dy2 * a2j;
    const float da2 = W3[j] * dy0 + W3[NH + j] * dy1 + W3[2 * NH + j] * dy2;
    const float dh2 = da2 * gelu_grad(h2);
    d2[j] = dh2;
    gb2 += dh2;
    __syncthreads();
    for (int i = 0; i < NH; ++i) G2[j * 129 + i] = fmaf(dh2, a1[i], G2[j * 129 + i]);
    float da1 = 0.f;
    for (int i = 0; i < NH; ++i) da1 = fmaf(W2[i * 129 + j], d2[i], da1);
    const float dh1 = da1 * gelu_grad(h1);
    gb1 += dh1;
    for (int i = 0; i < NI; ++i) G1[j * 33 + i] = fmaf(dh1, xs[i], G1[j * 33 + i]);
    __syncthreads();
  }
  for (int e = j; e < NH * NI; e += NH) atomicAdd(&grad[OFF_W1 + e], G1[(e / NI) * 33 + e % NI]);
  for (int e = j; e < NH * NH; e += NH) atomicAdd(&grad[OFF_W2 + e], G2[(e / NH) * 129 + e % NH]);
  for (int e = j; e < NO * NH; e += NH) atomicAdd(&grad[OFF_W3 + e], G3[e]);
  atomicAdd(&grad[OFF_B1 + j], gb1);
  atomicAdd(&grad[OFF_B2 + j], gb2);
  if (j < NO) {
    atomicAdd(&grad[OFF_B3 + j], gb3);
    atomicAdd(loss, lsum);
  }
}

__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2,
                            __nv_bfloat16* __restrict__ pb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float p = P[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  P[i] = p;
  pb[i] = __float2bfloat16_rn(p);
}

__global__ void to_bf16_kernel(const float* __restrict__ P, __nv_bfloat16* __restrict__ pb, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) pb[i] = __float2bfloat16_rn(P[i]);
}

// Inference: BF16 weights (converted to FP32 in shared memory), FP32 accumulation.
__global__ void __launch_bounds__(128) mlp_predict_kernel(const __nv_bfloat16* __restrict__ P,
                                                          const float* __restrict__ norm, const float* __restrict__ X,
                                                          int B, float* __restrict__ Y) {
  extern __shared__ float sm[];
  float* W1 = sm;
  float* W2 = W1 + NH * 33;
  float* W3 = W2 + NH * 129;
  float* xs = W3 + NO * NH;
  float* a1 = xs + NI;
  float* a2 = a1 + NH;
  const int j = threadIdx.x, lane = j & 31, warp = j >> 5;
  for (int e = j; e < NH * NI; e += NH) W1[(e / NI) * 33 + e % NI] = __bfloat162float(P[OFF_W1 + e]);
  for (int e = j; e < NH * NH; e += NH) W2[(e / NH) * 129 + e % NH] = __bfloat162float(P[OFF_W2 + e]);
  for (int e = j; e < NO * NH; e += NH) W3[e] = __bfloat162float(P[OFF_W3 + e]);
  const float b1 = __bfloat162float(P[OFF_B1 + j]), b2 = __bfloat162float(P[OFF_B2 + j]);
  __syncthreads();
  const int s0 = blockIdx.x * SPC, s1 = min(s0 + SPC, B);
  for (int s = s0; s < s1; ++s) {
    if (j < NI) xs[j] = (X[(int64_t)s * NI + j] - norm[j]) / norm[NI + j];
    __syncthreads();
    float h1 = b1;
    for (int i = 0; i < NI; ++i) h1 = fmaf(W1[j * 33 + i], xs[i], h1);
    a1[j] = gelu(h1);
    __syncthreads();
    float h2 = b2;
    for (int i = 0; i < NH; ++i) h2 = fmaf(W2[j * 129 + i], a1[i], h2);
    a2[j] = gelu(h2);
    __syncthreads();
    if (warp < NO) {
      float acc = 0.f;
      for (int i = lane; i < NH; i += 32) acc = fmaf(W3[warp * NH + i], a2[i], acc);
      for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0)
        Y[(int64_t)s * NO + warp] = (acc + __bfloat162float(P[OFF_B3 + warp])) * norm[2 * NI + NO + warp] + norm[2 * NI + warp];
    }
    __syncthreads();
  }
}

constexpr size_t GRAD_SMEM = sizeof(float) * (2 * (NH * 33 + NH * 129 + NO * NH) + NI + 3 * NH + 8);
constexpr size_t PRED_SMEM = sizeof(float) * (NH * 33 + NH * 129 + NO * NH + NI + 2 * NH);

}  // namespace

// ------------------------------------------------------------------------------------------ launchers

// One pass over A0 for the Gershgorin bounds, the per-row diagonal and radius and the mu-independent
// features (at mu = 0) of every block.
cudaError_t launch_bounds_features(nolsm_ctx* ctx, float* feat) {
  features_kernel<<<ctx->n_blocks, 256, 0, ctx->stream>>>(ctx->d_blocks, ctx->d_a0, ctx->d_lo, ctx->d_hi, 0.0,
                                                                (float)ctx->opt.alpha_margin, feat, ctx->d_rowd,
                                                                ctx->d_rowr, ctx->d_flags);
  return cudaGetLastError();
}

cudaError_t launch_features_mu(nolsm_ctx* ctx, double mu, float* feat) {
  features_mu_kernel<<<ctx->n_blocks, 128, 0, ctx->stream>>>(ctx->d_blocks, ctx->d_feat_static, ctx->d_rowd,
                                                             ctx->d_rowr, mu, (float)ctx->opt.alpha_margin, feat);
  return cudaGetLastError();
}

// Kept bounds for the next geometry: (smallest and largest Ritz value of A0, log10 of the smallest
// Ritz value of |A0 - mu|) per block, the layout of the network's predictions.
__global__ void given_from_lanczos_kernel(int n_blocks, const float* __restrict__ lz_a0, const float* __restrict__ lz_abs,
                                          float* __restrict__ given) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_blocks) return;
  given[3 * b + 0] = lz_a0[4 * b + 0];
  given[3 * b + 1] = lz_a0[4 * b + 1];
  given[3 * b + 2] = log10f(fmaxf(lz_abs[4 * b + 0], 1e-8f));
}

cudaError_t launch_given_from_lanczos(nolsm_ctx* ctx, const float* lz_a0, const float* lz_abs, float* given) {
  given_from_lanczos_kernel<<<(ctx->n_blocks + 255) / 256, 256, 0, ctx->stream>>>(ctx->n_blocks, lz_a0, lz_abs, given);
  return cudaGetLastError();
}

cudaError_t launch_lanczos(nolsm_ctx* ctx, double mu, int op, int k, float* basis, int64_t stride, float* out) {
  int max_pad = 128;
  for (const auto& b : ctx->h_blocks) max_pad = std::max(max_pad, b.n_pad);
  const size_t smem = sizeof(float) * 2 * (size_t)max_pad;
  const int hk = (ctx->opt.precision == NOLSM_PREC_MIXED_FP16) ? 1 : (ctx->opt.precision == NOLSM_PREC_MIXED_BF16 ? 2 : 0);
  if (smem > 48 * 1024) {   // blocks above n_pad 6144
    cudaError_t e = hk == 0 ? cudaFuncSetAttribute(lanczos_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                  : hk == 1 ? cudaFuncSetAttribute(lanczos_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                            : cudaFuncSetAttribute(lanczos_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (hk == 0)
    lanczos_kernel<float><<<ctx->n_blocks, 256, smem, ctx->stream>>>(ctx->d_blocks, ctx->d_a0, ctx->d_state,
                                                                     (const float*)ctx->d_x[0], (const float*)ctx->d_x[1],
                                                                     mu, op, k, basis, stride, out);
  else if (hk == 1)
    lanczos_kernel<__half><<<ctx->n_blocks, 256, smem, ctx->stream>>>(ctx->d_blocks, ctx->d_a0, ctx->d_state,
                                                                      (const __half*)ctx->d_x[0], (const __half*)ctx->d_x[1],
                                                                      mu, op, k, basis, stride, out);
  else
    lanczos_kernel<__nv_bfloat16><<<ctx->n_blocks, 256, smem, ctx->stream>>>(
        ctx->d_blocks, ctx->d_a0, ctx->d_state, (const __nv_bfloat16*)ctx->d_x[0], (const __nv_bfloat16*)ctx->d_x[1], mu,
        op, k, basis, stride, out);
  return cudaGetLastError();
}

}  // namespace nolsm

// ------------------------------------------------------------------------------------------ the network object

struct nolsm_mlp {
  cudaStream_t stream = nullptr;
  float* p = nullptr;        // FP32 master parameters
  __nv_bfloat16* pb = nullptr;
  float* g = nullptr;        // gradient of the last nolsm_mlp_gradient
  float* m = nullptr;
  float* v = nullptr;
  float* norm = nullptr;     // x mean, x std, y mean, y std
  double* d_loss = nullptr;
  int t = 0;                 // Adam steps taken
};

using namespace nolsm;

extern "C" {

nolsm_status nolsm_mlp_create(nolsm_mlp** out, const float* params, const float* norm, void* cuda_stream) {
  if (!out || !norm) return NOLSM_EINVAL;
  *out = nullptr;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GRAD_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(mlp_predict_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PRED_SMEM) !=
            cudaSuccess)
      return NOLSM_ECUDA;
    attr = true;
  }
  nolsm_mlp* m = new (std::nothrow) nolsm_mlp();
  if (!m) return NOLSM_ENOMEM;
  m->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaMalloc(&m->p, sizeof(float) * N_PARAMS);
  if (e == cudaSuccess) e = cudaMalloc(&m->pb, sizeof(__nv_bfloat16) * N_PARAMS);
  if (e == cudaSuccess) e = cudaMalloc(&m->g, sizeof(float) * N_PARAMS);
  if (e == cudaSuccess) e = cudaMalloc(&m->m, sizeof(float) * N_PARAMS);
  if (e == cudaSuccess) e = cudaMalloc(&m->v, sizeof(float) * N_PARAMS);
  if (e == cudaSuccess) e = cudaMalloc(&m->norm, sizeof(float) * N_NORM);
  if (e == cudaSuccess) e = cudaMalloc(&m->d_loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, sizeof(float) * N_PARAMS, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, sizeof(float) * N_PARAMS, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->g, 0, sizeof(float) * N_PARAMS, m->stream);
  if (e == cudaSuccess) {
    if (params) e = cudaMemcpyAsync(m->p, params, sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice, m->stream);
    else e = cudaMemsetAsync(m->p, 0, sizeof(float) * N_PARAMS, m->stream);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->norm, norm, sizeof(float) * N_NORM, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) {
    to_bf16_kernel<<<(N_PARAMS + 255) / 256, 256, 0, m->stream>>>(m->p, m->pb, N_PARAMS);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    nolsm_mlp_destroy(m);
    return e == cudaErrorMemoryAllocation ? NOLSM_ENOMEM : NOLSM_ECUDA;
  }
  *out = m;
  return NOLSM_OK;
}

void nolsm_mlp_destroy(nolsm_mlp* m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  cudaFree(m->p);
  cudaFree(m->pb);
  cudaFree(m->g);
  cudaFree(m->m);
  cudaFree(m->v);
  cudaFree(m->norm);
  cudaFree(m->d_loss);
  delete m;
}

nolsm_status nolsm_mlp_get_params(const nolsm_mlp* m, float* params) {
  if (!m || !params) return NOLSM_EINVAL;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return NOLSM_ECUDA;
  return cudaMemcpy(params, m->p, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost) == cudaSuccess ? NOLSM_OK : NOLSM_ECUDA;
}

nolsm_status nolsm_mlp_gradient(nolsm_mlp* m, const float* x, const float* t, int32_t n, const float* loss_w,
                                float* grad_out, double* loss_out) {
  if (!m || !x || !t || n <= 0 || !loss_w) return NOLSM_EINVAL;
  if (cudaMemsetAsync(m->g, 0, sizeof(float) * N_PARAMS, m->stream) != cudaSuccess) return NOLSM_ECUDA;
  if (cudaMemsetAsync(m->d_loss, 0, sizeof(double), m->stream) != cudaSuccess) return NOLSM_ECUDA;
  mlp_grad_kernel<<<(n + SPC - 1) / SPC, NH, GRAD_SMEM, m->stream>>>(m->p, m->norm, x, t, loss_w[0], loss_w[1],
                                                                     loss_w[2], n, m->g, m->d_loss);
  if (cudaGetLastError() != cudaSuccess) return NOLSM_ECUDA;
  if (grad_out && cudaMemcpyAsync(grad_out, m->g, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToDevice, m->stream) !=
                      cudaSuccess)
    return NOLSM_ECUDA;
  if (loss_out) {
    if (cudaMemcpyAsync(loss_out, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
      return NOLSM_ECUDA;
  }
  return NOLSM_OK;
}

nolsm_status nolsm_mlp_adam(nolsm_mlp* m, float lr, float beta1, float beta2, float eps) {
  if (!m || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0)) return NOLSM_EINVAL;
  m->t += 1;
  const float c1 = 1.f - powf(beta1, (float)m->t), c2 = 1.f - powf(beta2, (float)m->t);
  adam_kernel<<<(N_PARAMS + 255) / 256, 256, 0, m->stream>>>(m->p, m->g, m->m, m->v, N_PARAMS, lr, beta1, beta2, eps,
                                                             c1, c2, m->pb);
  return cudaGetLastError() == cudaSuccess ? NOLSM_OK : NOLSM_ECUDA;
}

nolsm_status nolsm_mlp_predict(const nolsm_mlp* m, const float* x, int32_t n, float* y) {
  if (!m || !x || !y || n <= 0) return NOLSM_EINVAL;
  mlp_predict_kernel<<<(n + SPC - 1) / SPC, NH, PRED_SMEM, m->stream>>>(m->pb, m->norm, x, n, y);
  return cudaGetLastError() == cudaSuccess ? NOLSM_OK : NOLSM_ECUDA;
}

}  // extern "C"

// internal access for the context (api.cu)
namespace nolsm {
cudaError_t mlp_predict_on(const nolsm_mlp* m, cudaStream_t s, const float* x, int n, float* y) {
  mlp_predict_kernel<<<(n + SPC - 1) / SPC, NH, PRED_SMEM, s>>>(m->pb, m->norm, x, n, y);
  return cudaGetLastError();
}
}  // namespace nolsm
