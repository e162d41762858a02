// The whole density step for systems whose blocks do not fit in device memory at once: the
// submatrix method's blocks are independent (Section II), so they can be streamed through the
// context's pools in chunks while the CSR of H0, S and D stays resident.  One pass builds every
// chunk in turn (gather, factor, inverse, congruence, bounds), evaluates its sign at the pass's
// chemical potential, adds its terms of N(mu) = Tr(D S) and Tr(D H0), and scatters its columns of D
// into the caller's D.  The chemical potential follows nolsm_set_mu's bisection, one pass per
// evaluation (Section V-A); the D of the last pass is the D at the returned mu.
#include "internal.h"

#include <cmath>
#include <limits>
#include <numeric>

using namespace nolsm;

namespace {

// Restores the context's chunked-mode fields on every exit path.
struct ChunkedMode {
  nolsm_ctx* ctx;
  explicit ChunkedMode(nolsm_ctx* c, double* target) : ctx(c) {
    ctx->chunked = true;
    ctx->transpose_ready = false;
    ctx->d_dval_target = target;
  }
  ~ChunkedMode() {
    ctx->chunked = false;
    ctx->transpose_ready = false;
    ctx->d_dval_target = nullptr;
    ctx->have_density = false;
  }
};

// Midpoint of the k-th and (k+1)-th smallest entries (nolsm_set_mu's Aufbau estimate), NaN when k
// is out of range.
double aufbau(std::vector<float> d, int64_t k) {
  if (k < 1 || k >= (int64_t)d.size()) return std::numeric_limits<double>::quiet_NaN();
  std::nth_element(d.begin(), d.begin() + k, d.end());
  const float above = d[(size_t)k];
  const float below = *std::max_element(d.begin(), d.begin() + k);
  return 0.5 * ((double)below + (double)above);
}

// Device bytes the context's pools need for one block of dimension at most n (square pools of
// n_pad^2: A0, L^-1, T1 in FP32, S and its factor in 2 x FP64, three iterate buffers of 2 or 4
// bytes; slabs, per-row tables and the factor's slice planes are small beside them).
double block_bytes(int64_t n, int64_t cols, bool mixed) {
  const double np = (double)pad_dim((int)std::min<int64_t>(n, kMaxDimLarge));
  const double sq = np * np;
  return sq * (3 * 4 + 16 + 3 * (mixed ? 2 : 4)) + np * (double)cols * 4 * 10 + 3.0 * kMaxDim * 4 +
         7.0 * 64 * 2 * np + 64.0 * 1024;
}

}  // namespace

extern "C" nolsm_status nolsm_solve_chunked(nolsm_ctx* ctx, const nolsm_csr* H, const nolsm_csr* S,
                                            int32_t n_blocks, const int32_t* blk_ptr, const int32_t* blk_cols,
                                            const int32_t* extra_ptr, const int32_t* extra_idx, int32_t chunk_blocks,
                                            double n_electrons, double tol_n, int32_t max_passes, double* d_val,
                                            double* block_n, double* block_e, nolsm_chunked_stats* out) {
  if (!ctx) return NOLSM_EINVAL;
  if (!H || !S || !blk_ptr || !blk_cols || !d_val || n_blocks <= 0)
    return fail(ctx, NOLSM_EINVAL, "null argument or no blocks");
  if (H->memory != NOLSM_MEM_DEVICE || S->memory != NOLSM_MEM_DEVICE)
    return fail(ctx, NOLSM_EINVAL, "the chunked solve needs the CSR in device memory");
  if (!(n_electrons > 0) || !(tol_n >= 0) || max_passes <= 0)
    return fail(ctx, NOLSM_EINVAL, "bad bisection arguments");
  if ((extra_ptr == nullptr) != (extra_idx == nullptr)) return fail(ctx, NOLSM_EINVAL, "extra_ptr and extra_idx go together");
  if (blk_ptr[0] != 0 || (extra_ptr && extra_ptr[0] != 0)) return fail(ctx, NOLSM_EINVAL, "blk_ptr[0] and extra_ptr[0] must be 0");
  for (int32_t b = 0; b < n_blocks; ++b)
    if (blk_ptr[b + 1] <= blk_ptr[b] || (extra_ptr && extra_ptr[b + 1] < extra_ptr[b]))
      return fail(ctx, NOLSM_EINVAL, "blk_ptr / extra_ptr not increasing");
  const bool mixed = ctx->opt.precision != NOLSM_PREC_FP32;
  const int64_t N = H->n, nnz = H->nnz;
  if (N <= 0 || nnz <= 0 || S->n != N || S->nnz != nnz) return fail(ctx, NOLSM_EINVAL, "H and S must share the pattern");

  // ---- chunks: consecutive blocks, either chunk_blocks at a time or as many as fit within 60 % of
  // the free device memory (plus the context's own pools, which the chunks reuse).  The pool bytes of
  // a block are estimated from a bound on its dimension (its own rows' entries plus its extra list)
  // scaled by the largest ratio of actual to estimated bytes among the blocks built so far, so the
  // first chunk is sized conservatively and the later ones from the measured dimensions.  The cuts
  // of the first pass are kept for the later ones.
  std::vector<int32_t> cut{0};
  std::vector<double> est;
  double budget = 0.0, ratio = 1.0;   // estimate scale; 1 until the first chunk has been built
  bool measured = false;
  if (chunk_blocks > 0) {
    for (int32_t b = chunk_blocks; b < n_blocks; b += chunk_blocks) cut.push_back(b);
    cut.push_back(n_blocks);
  } else {
    std::vector<int64_t> rp((size_t)N + 1);
    if (cudaMemcpy(rp.data(), H->row_ptr, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(ctx, NOLSM_ECUDA, "row pointers");
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(ctx, NOLSM_ECUDA, "cudaMemGetInfo");
    double held = 0.0;
    for (const auto& c : ctx->caps) held += (double)c.second;
    budget = 0.6 * ((double)free_b + held);
    est.resize((size_t)n_blocks);
    for (int32_t b = 0; b < n_blocks; ++b) {
      int64_t m = extra_ptr ? extra_ptr[b + 1] - extra_ptr[b] : 0;
      for (int32_t k = blk_ptr[b]; k < blk_ptr[b + 1]; ++k) {
        const int32_t c = blk_cols[k];
        if (c < 0 || c >= N) return fail(ctx, NOLSM_EINVAL, "block column out of range");
        m += rp[c + 1] - rp[c];
      }
      est[b] = block_bytes(m, blk_ptr[b + 1] - blk_ptr[b], mixed);
    }
  }
  // end of the chunk that starts at b0 (first pass, automatic sizing)
  auto next_cut = [&](int32_t b0) {
    double used = 0.0;
    int32_t b = b0;
    while (b < n_blocks && (b == b0 || used + ratio * est[b] <= budget)) used += ratio * est[b++];
    return b;
  };
  ChunkedMode mode(ctx, d_val);
  const int64_t total_cols = blk_ptr[n_blocks];
  const double n_occ = n_electrons / ctx->opt.spin_factor;
  double mu = std::numeric_limits<double>::quiet_NaN();
  double lo = std::numeric_limits<double>::infinity(), hi = -lo, lo0 = 0, hi0 = 0;
  double n_mu = 0.0, e_tr = 0.0;
  std::vector<float> own_diag;
  own_diag.reserve((size_t)total_cols);
  nolsm_chunked_stats st{};
  std::vector<int32_t> bp, ep;
  std::vector<double> bn, be;
  cudaEvent_t t0 = nullptr, t1 = nullptr, tp = nullptr;
  if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess || cudaEventCreate(&tp) != cudaSuccess)
    return fail(ctx, NOLSM_ECUDA, "events");
  struct Ev { cudaEvent_t* e; ~Ev() { for (int i = 0; i < 3; ++i) if (e[i]) cudaEventDestroy(e[i]); } };
  cudaEvent_t evs[3] = {t0, t1, tp};
  Ev ev_guard{evs};
  cudaEventRecord(t0, ctx->stream);
  int pass = 0;
  for (; pass < max_passes; ++pass) {
    cudaEventRecord(tp, ctx->stream);
    if (cudaMemsetAsync(d_val, 0, sizeof(double) * nnz, ctx->stream) != cudaSuccess)
      return fail(ctx, NOLSM_ECUDA, "clearing D");
    n_mu = 0.0;
    e_tr = 0.0;
    int64_t it_sum = 0;
    int32_t it_max = 0;
    double fp = 0.0, fe = 0.0, fu = 0.0;
    for (int c = 0; c + 1 < (int)cut.size() || (chunk_blocks <= 0 && pass == 0 && cut.back() < n_blocks); ++c) {
      if (c + 1 >= (int)cut.size()) cut.push_back(next_cut(cut.back()));
      const int32_t b0 = cut[c], b1 = cut[c + 1], nb = b1 - b0;
      bp.resize((size_t)nb + 1);
      for (int32_t b = 0; b <= nb; ++b) bp[b] = blk_ptr[b0 + b] - blk_ptr[b0];
      const int32_t* ep_c = nullptr;
      const int32_t* ei_c = nullptr;
      if (extra_ptr) {
        ep.resize((size_t)nb + 1);
        for (int32_t b = 0; b <= nb; ++b) ep[b] = extra_ptr[b0 + b] - extra_ptr[b0];
        ep_c = ep.data();
        ei_c = extra_idx + extra_ptr[b0];
      }
      nolsm_status s = nolsm_build_submatrices(ctx, H, S, nb, bp.data(), blk_cols + blk_ptr[b0], ep_c, ei_c);
      if (s != NOLSM_OK) return s;
      if (chunk_blocks <= 0 && pass == 0) {
        double r = 0.0;
        for (int32_t b = 0; b < nb; ++b)
          r = std::max(r, 1.1 * block_bytes(ctx->h_blocks[b].n, bp[b + 1] - bp[b], mixed) / est[b0 + b]);
        ratio = measured ? std::max(ratio, r) : r;
        measured = true;
      }
      if (pass == 0) {
        lo = std::min(lo, *std::min_element(ctx->h_lo.begin(), ctx->h_lo.end()));
        hi = std::max(hi, *std::max_element(ctx->h_hi.begin(), ctx->h_hi.end()));
        own_diag.insert(own_diag.end(), ctx->h_own_diag.begin(), ctx->h_own_diag.end());
        if (c == 0) {
          // first point: the Aufbau estimate of the first chunk with its share of the occupied
          // orbitals (the global estimate needs every chunk's A0; it is the second point)
          const int64_t k0 = std::llround(n_occ * (double)ctx->h_own_diag.size() / (double)total_cols);
          mu = aufbau(ctx->h_own_diag, k0);
          if (!std::isfinite(mu)) mu = 0.5 * (ctx->h_lo[0] + ctx->h_hi[0]);
        }
      }
      nolsm_sign_stats ss{};
      s = nolsm_sign_batch(ctx, mu, &ss);
      if (s != NOLSM_OK) return s;
      n_mu += ss.n_electrons;
      e_tr += ss.band_energy;
      it_sum += (int64_t)std::llround(ss.iters_avg * nb);
      it_max = std::max(it_max, ss.iters_max);
      fp += ss.flops_paper;
      fe += ss.flops_executed;
      for (int32_t b = 0; b < nb; ++b) {   // n_b^2 (n_b + 1) per symmetric product, 2 i_b + 1 products
        const double n = ctx->h_blocks[b].n;
        fu += (2.0 * ctx->h_iters[b] + 1.0) * n * n * (n + 1.0);
      }
      if (block_n || block_e) {
        bn.resize((size_t)nb);
        be.resize((size_t)nb);
        s = nolsm_block_traces(ctx, bn.data(), be.data());
        if (s != NOLSM_OK) return s;
        if (block_n) std::copy(bn.begin(), bn.end(), block_n + b0);
        if (block_e) std::copy(be.begin(), be.end(), block_e + b0);
      }
      if (phase_mark(ctx, NOLSM_PHASE_DENSITY) != cudaSuccess || launch_density(ctx) != cudaSuccess ||
          phase_mark(ctx, -1) != cudaSuccess)
        return fail(ctx, NOLSM_ECUDA, "density scatter");
      ctx->n_launches += 1;
    }
    cudaEventRecord(t1, ctx->stream);
    if (cudaEventSynchronize(t1) != cudaSuccess) return fail(ctx, NOLSM_ECUDA, "pass");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, tp, t1);
    st.ms_last_pass = ms;
    st.iters_avg = (double)it_sum / n_blocks;
    st.iters_max = it_max;
    st.flops_paper = fp;
    st.flops_executed = fe;
    st.flops_useful = fu;
    if (pass == 0) {
      lo0 = lo;
      hi0 = hi;
    }
    if (std::fabs(n_mu - n_electrons) <= tol_n * n_electrons) { ++pass; break; }
    if (pass + 1 >= max_passes || hi - lo < 1e-10) { ++pass; break; }
    if (n_mu < n_electrons) lo = mu; else hi = mu;
    const double g = pass == 0 ? aufbau(own_diag, (int64_t)std::floor(n_occ)) : std::numeric_limits<double>::quiet_NaN();
    mu = (std::isfinite(g) && g > lo && g < hi) ? g : 0.5 * (lo + hi);
  }
  if (std::fabs(n_mu - n_electrons) > tol_n * n_electrons && (mu - lo0 < 1e-9 || hi0 - mu < 1e-9))
    return fail(ctx, NOLSM_EBRACKET, "N(mu) does not bracket the electron count");
  // E = spin Tr(D H0) over the assembled D (the last pass)
  if (phase_mark(ctx, NOLSM_PHASE_ENERGY) != cudaSuccess || launch_band_energy(ctx) != cudaSuccess ||
      phase_mark(ctx, -1) != cudaSuccess)
    return fail(ctx, NOLSM_ECUDA, "band energy");
  ctx->n_launches += 2;
  cudaEventRecord(t1, ctx->stream);
  if (cudaEventSynchronize(t1) != cudaSuccess) return fail(ctx, NOLSM_ECUDA, "band energy");
  if (cudaMemcpy(ctx->h_flags, ctx->d_flags, sizeof(DevFlags), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(ctx, NOLSM_ECUDA, "flags");
  if (ctx->h_flags->error != 0) return fail(ctx, (nolsm_status)ctx->h_flags->error, "device error");
  harvest_phases(ctx);
  float ms_all = 0.f;
  cudaEventElapsedTime(&ms_all, t0, t1);
  st.mu = mu;
  st.n_electrons = n_mu;
  st.band_energy = ctx->opt.spin_factor * ctx->h_flags->energy;
  st.band_energy_traces = e_tr;
  st.passes = pass;
  st.chunks = (int32_t)cut.size() - 1;
  st.n_blocks = n_blocks;
  st.max_chunk_blocks = 0;
  for (size_t c = 0; c + 1 < cut.size(); ++c) st.max_chunk_blocks = std::max(st.max_chunk_blocks, cut[c + 1] - cut[c]);
  st.ms_total = ms_all;
  if (out) *out = st;
  return NOLSM_OK;
}
