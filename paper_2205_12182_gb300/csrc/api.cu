// C ABI of libnolsm.so: context life cycle, the build of the submatrices (host-side index sets,
// size bins and memory layout), the sign evaluation loop, the chemical-potential bisection, the
// density scatter and the band energy.  See include/nolsm.h for the contract of every call.
#include "internal.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>

using namespace nolsm;

namespace nolsm {

nolsm_status fail(nolsm_ctx* ctx, nolsm_status st, const std::string& msg) {
  if (ctx) {
    if (ctx->sticky == NOLSM_OK) {
      ctx->sticky = st;
      ctx->last_error = msg;
    }
  }
  return st;
}

nolsm_status cuda_fail(nolsm_ctx* ctx, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(ctx, e == cudaErrorMemoryAllocation ? NOLSM_ENOMEM : NOLSM_ECUDA, m);
}

double unit_roundoff(const nolsm_ctx* ctx) {
  switch (ctx->opt.precision) {
    case NOLSM_PREC_MIXED_FP16: return std::ldexp(1.0, -11);
    case NOLSM_PREC_MIXED_BF16: return std::ldexp(1.0, -8);
    default: return std::ldexp(1.0, -24);
  }
}

cudaError_t phase_mark(nolsm_ctx* ctx, int phase) {
  cudaEvent_t ev;
  if (!ctx->ev_free.empty()) {
    ev = ctx->ev_free.back();
    ctx->ev_free.pop_back();
  } else {
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaEventRecord(ev, ctx->stream);
  if (e != cudaSuccess) return e;
  if (ctx->ph_open >= 0) ctx->ph_pending.push_back({ctx->ph_open, ctx->ph_open_ev, ev});
  if (phase >= 0) {
    ctx->ph_open = phase;
    ctx->ph_open_ev = ev;
  } else {
    ctx->ph_open = -1;
    ctx->ph_open_ev = nullptr;
    if (ctx->ph_pending.empty()) ctx->ev_free.push_back(ev);
  }
  return cudaSuccess;
}

// The stream has drained: accumulate every closed interval and recycle its events (an event that
// closes one interval and opens the next is recycled once).
void harvest_phases(nolsm_ctx* ctx) {
  std::vector<cudaEvent_t> done;
  for (const auto& r : ctx->ph_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) ctx->phase_ms[r.phase] += ms;
    done.push_back(r.a);
    done.push_back(r.b);
  }
  ctx->ph_pending.clear();
  std::sort(done.begin(), done.end());
  done.erase(std::unique(done.begin(), done.end()), done.end());
  for (cudaEvent_t ev : done)
    if (ev != ctx->ph_open_ev) ctx->ev_free.push_back(ev);
}

}  // namespace nolsm

#define CK(call)                                                  \
  do {                                                            \
    cudaError_t _e = (call);                                      \
    if (_e != cudaSuccess) return nolsm::cuda_fail(ctx, _e, #call); \
  } while (0)

namespace {

void dfree(void* p) {
  if (p) cudaFree(p);
}

// Make *p hold at least count elements; a pool keeps its allocation across builds and only
// grows (rebuilding the same system allocates nothing).
template <typename T>
cudaError_t dalloc(nolsm_ctx* ctx, T** p, size_t count) {
  if (count == 0) count = 1;
  const size_t bytes = count * sizeof(T);
  void** key = reinterpret_cast<void**>(p);
  for (auto& kv : ctx->caps)
    if (kv.first == key) {
      if (kv.second >= bytes && *p) return cudaSuccess;
      dfree(*p);
      *p = nullptr;
      cudaError_t e = cudaMalloc(key, bytes);
      kv.second = (e == cudaSuccess) ? bytes : 0;
      return e;
    }
  dfree(*p);
  *p = nullptr;
  cudaError_t e = cudaMalloc(key, bytes);
  ctx->caps.emplace_back(key, e == cudaSuccess ? bytes : 0);
  return e;
}

// The captured per-product iteration (its kernels' arguments name the context's pools).
void release_loop_graph(nolsm_ctx* ctx) {
  if (ctx->loop_exec) cudaGraphExecDestroy(ctx->loop_exec);
  if (ctx->loop_graph) cudaGraphDestroy(ctx->loop_graph);
  ctx->loop_exec = nullptr;
  ctx->loop_graph = nullptr;
  for (auto& k : ctx->loop_key) k = -1;
}

void release_pools(nolsm_ctx* ctx) {
  dfree(ctx->d_blocks); ctx->d_blocks = nullptr;
  dfree(ctx->d_idx); ctx->d_idx = nullptr;
  dfree(ctx->d_own); ctx->d_own = nullptr;
  dfree(ctx->d_blk_cols); ctx->d_blk_cols = nullptr;
  dfree(ctx->d_a0); ctx->d_a0 = nullptr;
  dfree(ctx->d_linv); ctx->d_linv = nullptr;
  dfree(ctx->d_x[0]); ctx->d_x[0] = nullptr;
  dfree(ctx->d_x[1]); ctx->d_x[1] = nullptr;
  dfree(ctx->d_b); ctx->d_b = nullptr;
  dfree(ctx->d_w); ctx->d_w = nullptr;
  dfree(ctx->d_z); ctx->d_z = nullptr;
  dfree(ctx->d_lc); ctx->d_lc = nullptr;
  dfree(ctx->d_y); ctx->d_y = nullptr;
  dfree(ctx->d_tmp); ctx->d_tmp = nullptr;
  dfree(ctx->d_lo); ctx->d_lo = nullptr;
  dfree(ctx->d_hi); ctx->d_hi = nullptr;
  dfree(ctx->d_bn); ctx->d_bn = nullptr;
  dfree(ctx->d_be); ctx->d_be = nullptr;
  dfree(ctx->d_slab_units); ctx->d_slab_units = nullptr;
  dfree(ctx->d_oz_exp); ctx->d_oz_exp = nullptr;
  dfree(ctx->d_oz_planes); ctx->d_oz_planes = nullptr;
  dfree(ctx->d_oz_items); ctx->d_oz_items = nullptr;
  dfree(ctx->d_oz_tmaps); ctx->d_oz_tmaps = nullptr;
  dfree(ctx->d_oz_m); ctx->d_oz_m = nullptr;
  dfree(ctx->d_oz_f); ctx->d_oz_f = nullptr;
  dfree(ctx->d_tr_items); ctx->d_tr_items = nullptr;
  dfree(ctx->d_own_diag); ctx->d_own_diag = nullptr;
  dfree(ctx->d_resacc); ctx->d_resacc = nullptr;
  dfree(ctx->d_tol); ctx->d_tol = nullptr;
  dfree(ctx->d_state); ctx->d_state = nullptr;
  dfree(ctx->d_tiles); ctx->d_tiles = nullptr;
  dfree(ctx->d_cg_kbeg); ctx->d_cg_kbeg = nullptr;
  dfree(ctx->d_bt); ctx->d_bt = nullptr;
  ctx->bt_dev = ctx->bt_kdev = nullptr;
  ctx->bt_layout.clear();
  dfree(ctx->d_transpose); ctx->d_transpose = nullptr;
  dfree(ctx->d_dval); ctx->d_dval = nullptr;
  dfree(ctx->d_csr_own); ctx->d_csr_own = nullptr;
  dfree(ctx->d_bptr); ctx->d_bptr = nullptr;
  dfree(ctx->d_extra); ctx->d_extra = nullptr;
  dfree(ctx->d_nb); ctx->d_nb = nullptr;
  dfree(ctx->d_tmaps); ctx->d_tmaps = nullptr;
  ctx->tmap_cap = 0;
  dfree(ctx->d_cg_tmaps); ctx->d_cg_tmaps = nullptr;
  ctx->cg_tmap_cap = 0;
  ctx->cg_maps_gen = -1;
  dfree(ctx->d_sb); ctx->d_sb = nullptr;
  dfree(ctx->d_feat); ctx->d_feat = nullptr;
  dfree(ctx->d_pred); ctx->d_pred = nullptr;
  dfree(ctx->d_lz); ctx->d_lz = nullptr;
  dfree(ctx->d_lz1); ctx->d_lz1 = nullptr;
  dfree(ctx->d_given); ctx->d_given = nullptr;
  dfree(ctx->d_lz_basis); ctx->d_lz_basis = nullptr;
  dfree(ctx->d_t1); ctx->d_t1 = nullptr;
  ctx->caps.clear();
  release_loop_graph(ctx);
  ctx->built = ctx->have_sign = ctx->have_density = false;
}

bool is_mixed(const nolsm_ctx* ctx) {
  return ctx->opt.precision == NOLSM_PREC_MIXED_FP16 || ctx->opt.precision == NOLSM_PREC_MIXED_BF16;
}

int half_kind(const nolsm_ctx* ctx) {
  if (ctx->opt.precision == NOLSM_PREC_MIXED_FP16) return 1;
  if (ctx->opt.precision == NOLSM_PREC_MIXED_BF16) return 2;
  return 0;
}


nolsm_status check_device_flags(nolsm_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, sizeof(DevFlags), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const int e = ctx->h_flags->error;
  if (e != 0) {
    const char* what = "device error";
    switch (e) {
      case NOLSM_ENOTPD: what = "a submatrix T_b(S) is not positive definite"; break;
      case NOLSM_ENOCONV: what = "sign iteration did not reach the tolerance within max_iter"; break;
      case NOLSM_ETIMEOUT: what = "a bounded device wait ran out"; break;
      case NOLSM_ENONFINITE: what = "non-finite value in the inputs or an iterate"; break;
      case NOLSM_EINVAL: what = "an own-column pattern entry is missing from its index set"; break;
      default: break;
    }
    return fail(ctx, (nolsm_status)e, what);
  }
  return NOLSM_OK;
}

// Lanczos on every block into out (device n_blocks x 4), or into the context's d_lz when out is NULL.
nolsm_status run_lanczos(nolsm_ctx* ctx, double mu, int op, int steps, float* out) {
  int max_pad = kTile;
  for (const auto& b : ctx->h_blocks) max_pad = std::max(max_pad, b.n_pad);
  const int64_t stride = (int64_t)(steps + 1) * max_pad;
  CK(dalloc(ctx, &ctx->d_lz_basis, (size_t)stride * ctx->n_blocks));
  if (!out) {
    CK(dalloc(ctx, &ctx->d_lz, (size_t)4 * ctx->n_blocks));
    out = ctx->d_lz;
  }
  CK(launch_lanczos(ctx, mu, op, steps, ctx->d_lz_basis, stride, out));
  ctx->n_launches += 1;
  CK(cudaStreamSynchronize(ctx->stream));
  return NOLSM_OK;
}

}  // namespace

extern "C" {

nolsm_status nolsm_default_options(nolsm_options* opt) {
  if (!opt) return NOLSM_EINVAL;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = NOLSM_PREC_MIXED_FP16;
  opt->bounds = NOLSM_BOUNDS_GERSHGORIN;
  opt->chol_precision = NOLSM_CHOL_DF64;
  opt->scaled = 1;
  opt->sign_tol = 0.0;
  opt->max_iter = 100;
  opt->refine_iters = 2;
  opt->spin_factor = 2.0;
  opt->lower_bound = 0.02;
  opt->alpha_margin = 0.02;
  opt->wait_budget = 1LL << 22;
  opt->lanczos_steps = 24;
  opt->schedule = NOLSM_SCHEDULE_AUTO;
  opt->refine_path = NOLSM_REFINE_TENSOR;
  opt->fp8_iters = 0;
  opt->mu_first = NOLSM_MU_FIRST_AUFBAU;
  opt->loop = NOLSM_LOOP_GRAPH;
  return NOLSM_OK;
}

nolsm_status nolsm_create(nolsm_ctx** out, const nolsm_options* opt, void* cuda_stream) {
  if (!out) return NOLSM_EINVAL;
  *out = nullptr;
  nolsm_ctx* ctx = new (std::nothrow) nolsm_ctx();
  if (!ctx) return NOLSM_ENOMEM;
  if (opt) ctx->opt = *opt; else nolsm_default_options(&ctx->opt);
  if (ctx->opt.precision < NOLSM_PREC_FP32 || ctx->opt.precision > NOLSM_PREC_MIXED_BF16 || ctx->opt.max_iter <= 0 ||
      ctx->opt.refine_iters < 0 || ctx->opt.refine_iters > 3 || !(ctx->opt.spin_factor > 0) ||
      ctx->opt.wait_budget <= 0 || ctx->opt.alpha_margin < 0 || ctx->opt.chol_precision < 0 ||
      ctx->opt.chol_precision > NOLSM_CHOL_DF64_SIMT || ctx->opt.bounds < NOLSM_BOUNDS_GERSHGORIN ||
      ctx->opt.bounds > NOLSM_BOUNDS_GIVEN || ctx->opt.lanczos_steps < 1 || ctx->opt.lanczos_steps > 64 ||
      ctx->opt.schedule < NOLSM_SCHEDULE_PERSISTENT || ctx->opt.schedule > NOLSM_SCHEDULE_PERSISTENT_INTERLEAVED ||
      ctx->opt.refine_path < NOLSM_REFINE_TENSOR || ctx->opt.refine_path > NOLSM_REFINE_SIMT ||
      ctx->opt.fp8_iters < 0 || ctx->opt.fp8_iters > ctx->opt.max_iter || ctx->opt.loop < NOLSM_LOOP_GRAPH ||
      ctx->opt.loop > NOLSM_LOOP_HOST) {
    delete ctx;
    return NOLSM_EINVAL;
  }
  ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&ctx->d_flags), sizeof(DevFlags));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&ctx->h_flags), sizeof(DevFlags));
  if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
  if (e != cudaSuccess) {
    if (ctx->d_flags) cudaFree(ctx->d_flags);
    if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
    delete ctx;
    return e == cudaErrorMemoryAllocation ? NOLSM_ENOMEM : NOLSM_ECUDA;
  }
  *out = ctx;
  return NOLSM_OK;
}

void nolsm_destroy(nolsm_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream); else cudaDeviceSynchronize();
  release_pools(ctx);
  if (ctx->d_flags) cudaFree(ctx->d_flags);
  if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  for (auto e : ctx->gemm_ev) cudaEventDestroy(e);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

const char* nolsm_last_error(const nolsm_ctx* ctx) {
  if (!ctx) return "";
  return ctx->last_error.c_str();
}

nolsm_status nolsm_build_submatrices(nolsm_ctx* ctx, const nolsm_csr* H, const nolsm_csr* S, int32_t n_blocks,
                                     const int32_t* blk_ptr, const int32_t* blk_cols, const int32_t* extra_ptr,
                                     const int32_t* extra_idx) {
  if (!ctx) return NOLSM_EINVAL;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  ctx->sticky = NOLSM_OK;   // a new build clears the sticky error
  ctx->last_error.clear();
  ctx->built = ctx->have_sign = ctx->have_density = false;
  ctx->build_gen += 1;      // a captured iteration graph names the previous build's pools
  if (!H || !S || !blk_ptr || !blk_cols || n_blocks <= 0) return fail(ctx, NOLSM_EINVAL, "null argument or no blocks");
  if (H->n != S->n || H->nnz != S->nnz || H->n <= 0 || H->nnz <= 0 || H->memory != S->memory ||
      H->n > INT32_MAX)
    return fail(ctx, NOLSM_EINVAL, "H and S must share dimension, pattern and memory kind");
  if ((extra_ptr == nullptr) != (extra_idx == nullptr)) return fail(ctx, NOLSM_EINVAL, "extra_ptr and extra_idx go together");
  const int64_t N = H->n, nnz = H->nnz;
  ctx->n = N;
  ctx->nnz = nnz;
  ctx->n_blocks = n_blocks;
  if (blk_ptr[0] != 0) return fail(ctx, NOLSM_EINVAL, "blk_ptr[0] must be 0");
  for (int32_t b = 0; b < n_blocks; ++b) {
    if (blk_ptr[b + 1] <= blk_ptr[b]) return fail(ctx, NOLSM_EINVAL, "every block needs at least one column");
    if (extra_ptr && extra_ptr[b + 1] < extra_ptr[b]) return fail(ctx, NOLSM_EINVAL, "extra_ptr not monotone");
  }
  if (extra_ptr && extra_ptr[0] != 0) return fail(ctx, NOLSM_EINVAL, "extra_ptr[0] must be 0");
  const int64_t n_cols = blk_ptr[n_blocks];
  const int64_t n_extra = extra_ptr ? extra_ptr[n_blocks] : 0;
  ctx->h_blk_cols.assign(blk_cols, blk_cols + n_cols);
  for (int64_t k = 0; k < n_cols; ++k)
    if (blk_cols[k] < 0 || blk_cols[k] >= N) return fail(ctx, NOLSM_EINVAL, "block column out of range");

  // ---- CSR on the device (staged when host-resident); the row pointers also on the host
  std::vector<int64_t> rp((size_t)N + 1);
  if (H->memory == NOLSM_MEM_HOST) {
    std::memcpy(rp.data(), H->row_ptr, sizeof(int64_t) * (N + 1));
    const size_t bytes = sizeof(int64_t) * (N + 1) + sizeof(int32_t) * nnz + 2 * sizeof(double) * nnz + 64;
    CK(dalloc(ctx, reinterpret_cast<uint8_t**>(&ctx->d_csr_own), bytes));
    uint8_t* base = reinterpret_cast<uint8_t*>(ctx->d_csr_own);
    double* hv = reinterpret_cast<double*>(base);
    double* sv = hv + nnz;
    int64_t* rpd = reinterpret_cast<int64_t*>(sv + nnz);
    int32_t* cld = reinterpret_cast<int32_t*>(rpd + N + 1);
    CK(cudaMemcpyAsync(hv, H->val, sizeof(double) * nnz, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(sv, S->val, sizeof(double) * nnz, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(rpd, H->row_ptr, sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(cld, H->col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, ctx->stream));
    ctx->d_hval = hv; ctx->d_sval = sv; ctx->d_row_ptr = rpd; ctx->d_col = cld;
  } else {
    CK(cudaMemcpyAsync(rp.data(), H->row_ptr, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToHost, ctx->stream));
    ctx->d_hval = H->val; ctx->d_sval = S->val; ctx->d_row_ptr = H->row_ptr; ctx->d_col = H->col;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  if (rp[0] != 0 || rp[N] != nnz) return fail(ctx, NOLSM_EINVAL, "row_ptr must start at 0 and end at nnz");
  // candidates of each block's index set: the own columns' row counts plus its extra list
  int64_t max_cand = 1;
  for (int32_t b = 0; b < n_blocks; ++b) {
    int64_t m = extra_ptr ? (extra_ptr[b + 1] - extra_ptr[b]) : 0;
    for (int32_t k = blk_ptr[b]; k < blk_ptr[b + 1]; ++k) m += rp[blk_cols[k] + 1] - rp[blk_cols[k]];
    max_cand = std::max(max_cand, m);
  }
  // the index-set kernel sorts in shared memory: up to kMaxCandidates entries, compacted to the
  // distinct rows whenever the next column would overflow (so one column may hold up to
  // kMaxCandidates - kMaxDim rows)
  int cap = 256;
  while (cap < max_cand && cap < kMaxCandidates) cap <<= 1;
  int64_t max_deg = 0;
  for (int64_t r = 0; r < N; ++r) max_deg = std::max<int64_t>(max_deg, rp[r + 1] - rp[r]);
  if (max_cand > cap && max_deg > cap - kMaxDim)
    return fail(ctx, NOLSM_EINVAL, "a row of the pattern holds more than 28672 entries");
  ctx->idx_stride = kMaxDim;

  // ---- transpose positions, pattern checks and index sets on the device
  CK(dalloc(ctx, &ctx->d_transpose, (size_t)nnz));
  CK(dalloc(ctx, &ctx->d_idx, (size_t)n_blocks * ctx->idx_stride));
  CK(dalloc(ctx, &ctx->d_own, (size_t)n_cols));
  CK(dalloc(ctx, &ctx->d_blk_cols, (size_t)n_cols));
  CK(dalloc(ctx, &ctx->d_bptr, (size_t)(2 * (n_blocks + 1))));
  CK(dalloc(ctx, &ctx->d_extra, (size_t)std::max<int64_t>(n_extra, 1)));
  CK(dalloc(ctx, &ctx->d_nb, (size_t)n_blocks));
  CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(DevFlags), ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_blk_cols, blk_cols, sizeof(int32_t) * n_cols, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_bptr, blk_ptr, sizeof(int32_t) * (n_blocks + 1), cudaMemcpyHostToDevice, ctx->stream));
  if (extra_ptr) {
    CK(cudaMemcpyAsync(ctx->d_bptr + n_blocks + 1, extra_ptr, sizeof(int32_t) * (n_blocks + 1), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_extra, extra_idx, sizeof(int32_t) * n_extra, cudaMemcpyHostToDevice, ctx->stream));
  }
  if (!(ctx->chunked && ctx->transpose_ready)) CK(launch_transpose(ctx));
  ctx->transpose_ready = ctx->chunked;
  CK(launch_index_sets(ctx, ctx->d_bptr, extra_ptr ? ctx->d_bptr + n_blocks + 1 : nullptr,
                       extra_ptr ? ctx->d_extra : nullptr, ctx->d_nb, cap, ctx->idx_stride));
  ctx->n_launches += 2;
  {
    nolsm_status st0 = check_device_flags(ctx);
    if (st0 == NOLSM_OK && ctx->h_flags->oversize > 0) {
      // some index set holds more than 4096 rows: every block again with the wide stride (blocks up
      // to 16384; larger ones are an EINVAL error of the kernel)
      ctx->idx_stride = kMaxDimLarge;
      cap = kMaxCandidates;
      CK(dalloc(ctx, &ctx->d_idx, (size_t)n_blocks * ctx->idx_stride));
      CK(cudaMemsetAsync(ctx->d_flags, 0, sizeof(DevFlags), ctx->stream));
      CK(launch_index_sets(ctx, ctx->d_bptr, extra_ptr ? ctx->d_bptr + n_blocks + 1 : nullptr,
                           extra_ptr ? ctx->d_extra : nullptr, ctx->d_nb, cap, ctx->idx_stride));
      ctx->n_launches += 1;
      st0 = check_device_flags(ctx);
    }
    if (st0 != NOLSM_OK) {
      ctx->last_error = "pattern not symmetric / columns out of order or range / missing diagonal, or a "
                        "submatrix dimension above 16384";
      return st0;
    }
  }
  std::vector<int32_t> nb((size_t)n_blocks);
  CK(cudaMemcpy(nb.data(), ctx->d_nb, sizeof(int32_t) * n_blocks, cudaMemcpyDeviceToHost));

  // ---- layout: bins of equal n_pad stored contiguously (tensor maps stack a bin's matrices)
  ctx->h_blocks.assign((size_t)n_blocks, BlockDesc{});
  std::vector<int32_t> order((size_t)n_blocks);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return pad_dim(nb[a]) < pad_dim(nb[b]); });
  int64_t off_mat = 0, off_slab = 0;
  int bin = -1, pos = 0, last_pad = -1, slab_row = 0;
  ctx->sum_pad = 0;
  ctx->flops_paper_iter = ctx->flops_exec_iter = 0.0;
  for (int32_t b = 0; b < n_blocks; ++b) {
    BlockDesc& bd = ctx->h_blocks[b];
    bd.n = nb[b];
    bd.n_pad = pad_dim(bd.n);
    bd.c = blk_ptr[b + 1] - blk_ptr[b];
    bd.col0 = blk_ptr[b];
    bd.off_idx = (int64_t)b * ctx->idx_stride;
    bd.off_own = blk_ptr[b];
    ctx->flops_paper_iter += 2.0 * 2.0 * (double)bd.n * bd.n * bd.n;
    ctx->flops_exec_iter += 2.0 * (double)bd.n_pad * bd.n_pad * (bd.n_pad + kTile);
  }
  for (int32_t b : order) {
    BlockDesc& bd = ctx->h_blocks[b];
    if (bd.n_pad != last_pad) { ++bin; pos = 0; slab_row = 0; last_pad = bd.n_pad; }
    bd.bin = bin;
    bd.pos = pos++;
    bd.slab_row = slab_row;
    slab_row += bd.c;
    bd.row_off = (int32_t)ctx->sum_pad;
    ctx->sum_pad += bd.n_pad;
    bd.off_mat = off_mat;
    bd.off_slab = off_slab;
    off_mat += (int64_t)bd.n_pad * bd.n_pad;
    off_slab += (int64_t)bd.n_pad * bd.c;
  }
  ctx->sum_sq = off_mat;
  ctx->sum_slab = off_slab;
  ctx->sum_idx = (int64_t)n_blocks * ctx->idx_stride;
  ctx->sum_own = n_cols;
  int64_t tiles_max = 0;
  for (const auto& bd : ctx->h_blocks) tiles_max += (int64_t)(bd.n_pad / kTile) * (bd.n_pad / kTile);
  ctx->max_tiles = tiles_max;
  ctx->max_tiles_tc = 0;
  for (const auto& bd : ctx->h_blocks)
    for (int m0 = 0; m0 < bd.n_pad; m0 += kTile) ctx->max_tiles_tc += (bd.n_pad - m0 + 255) / 256;
  // pieces of the own columns for the tensor-core refinement (block, first column, width)
  std::vector<int32_t> units_n, units_w;
  {
    std::vector<int32_t> by_size(order.rbegin(), order.rend());   // largest n_pad first
    for (int32_t b : by_size) {
      const BlockDesc& bd = ctx->h_blocks[b];
      for (int c0 = 0; c0 < bd.c; c0 += kSlabWide) {
        const int cw = std::min(kSlabWide, bd.c - c0);
        std::vector<int32_t>& dst = cw <= kSlabNarrow ? units_n : units_w;
        dst.insert(dst.end(), {b, c0, cw, 0});
      }
    }
  }
  ctx->n_units_narrow = (int32_t)(units_n.size() / 4);
  ctx->n_units_wide = (int32_t)(units_w.size() / 4);
  units_n.insert(units_n.end(), units_w.begin(), units_w.end());
  ctx->h_slab_units.swap(units_n);
  const int64_t n_units = std::max<int64_t>((int64_t)ctx->h_slab_units.size() / 4, 1);

  // ---- device pools
  const bool mixed = is_mixed(ctx);
  const size_t xbytes = mixed ? 2 : 4;
  CK(dalloc(ctx, &ctx->d_blocks, (size_t)n_blocks));
  CK(dalloc(ctx, &ctx->d_a0, (size_t)ctx->sum_sq));
  CK(dalloc(ctx, &ctx->d_linv, (size_t)ctx->sum_sq));
  CK(dalloc(ctx, reinterpret_cast<uint8_t**>(&ctx->d_x[0]), xbytes * (size_t)ctx->sum_sq));
  CK(dalloc(ctx, reinterpret_cast<uint8_t**>(&ctx->d_x[1]), xbytes * (size_t)ctx->sum_sq));
  CK(dalloc(ctx, reinterpret_cast<uint8_t**>(&ctx->d_b), xbytes * (size_t)ctx->sum_sq));
  CK(dalloc(ctx, &ctx->d_w, (size_t)ctx->sum_slab));
  CK(dalloc(ctx, &ctx->d_z, (size_t)ctx->sum_slab));
  CK(dalloc(ctx, &ctx->d_lc, (size_t)ctx->sum_slab));
  CK(dalloc(ctx, &ctx->d_y, (size_t)ctx->sum_slab));
  CK(dalloc(ctx, &ctx->d_tmp, (size_t)std::max<int64_t>(6 * ctx->sum_slab, 4096)));
  CK(dalloc(ctx, &ctx->d_lo, (size_t)n_blocks));
  CK(dalloc(ctx, &ctx->d_hi, (size_t)n_blocks));
  CK(dalloc(ctx, &ctx->d_bn, (size_t)std::max<int64_t>(n_blocks, n_units)));
  CK(dalloc(ctx, &ctx->d_be, (size_t)std::max<int64_t>(n_blocks, n_units)));
  CK(dalloc(ctx, &ctx->d_slab_units, (size_t)(4 * n_units)));
  CK(dalloc(ctx, &ctx->d_resacc, (size_t)n_blocks));
  CK(dalloc(ctx, &ctx->d_tol, (size_t)n_blocks));
  CK(dalloc(ctx, &ctx->d_state, (size_t)n_blocks));
  CK(dalloc(ctx, &ctx->d_tiles, (size_t)tiles_max));
  // the build's product tile lists: congruence passes (all 128 x 128 tiles, then those on or above
  // the diagonal) and the tiled inverse (two launches per block row i >= 1, i tiles each)
  ctx->bt_cap = 0;
  for (const auto& bd : ctx->h_blocks) {
    const int64_t q = bd.n_pad / kTile;
    ctx->bt_cap += q * q + q * (q + 1) / 2 + q * (q - 1);
  }
  CK(dalloc(ctx, &ctx->d_bt, (size_t)ctx->bt_cap));
  CK(dalloc(ctx, &ctx->d_cg_kbeg, (size_t)ctx->bt_cap));
  if (!ctx->chunked) CK(dalloc(ctx, &ctx->d_dval, (size_t)nnz));
  CK(cudaMemcpyAsync(ctx->d_blocks, ctx->h_blocks.data(), sizeof(BlockDesc) * n_blocks, cudaMemcpyHostToDevice, ctx->stream));
  if (!ctx->h_slab_units.empty())
    CK(cudaMemcpyAsync(ctx->d_slab_units, ctx->h_slab_units.data(), sizeof(int32_t) * ctx->h_slab_units.size(),
                       cudaMemcpyHostToDevice, ctx->stream));
  {
    // Full-matrix iterations stop once the own-column refinement can finish the job: an
    // eigenvalue 1 - delta of X goes to about 1 - 1.5 delta^2 under one step of Eq. 6, so r
    // refinement steps need ||X^2 - I||_F ~ 2 delta no smaller than 0.02 (r >= 2: 3.4 delta^4 is
    // FP32 rounding for delta = 0.01) or 4e-4 (r = 1); never below the operand format's floor
    // 8 u sqrt(n) and never above 0.05.  Each further full iteration only adds rounding.
    std::vector<float>& tol = ctx->h_tol;   // the upload's source, kept until the next build
    tol.assign((size_t)n_blocks, 0.f);
    const double u = unit_roundoff(ctx);
    const int r = ctx->opt.refine_iters;
    const double t_refine = r >= 2 ? 0.02 : r == 1 ? 4e-4 : 0.0;
    for (int32_t b = 0; b < n_blocks; ++b) {
      const double d = 8.0 * u * std::sqrt((double)ctx->h_blocks[b].n);
      tol[b] = (float)(ctx->opt.sign_tol > 0 ? ctx->opt.sign_tol : std::min(0.05, std::max(d, t_refine)));
    }
    CK(cudaMemcpyAsync(ctx->d_tol, tol.data(), sizeof(float) * n_blocks, cudaMemcpyHostToDevice, ctx->stream));
  }

  // ---- gather (H FP32 into A0's pool, S FP64), factor, inverse, congruence, slabs, bounds
  CK(dalloc(ctx, &ctx->d_sb, (size_t)(2 * ctx->sum_sq)));
  CK(dalloc(ctx, &ctx->d_t1, (size_t)ctx->sum_sq));
  double* sb = ctx->d_sb;
  ctx->n_launches += 8;   // gather, factor, inverse (+conversion), two products, slabs, bounds
  CK(phase_mark(ctx, NOLSM_PHASE_GATHER));
  CK(launch_gather(ctx, ctx->d_a0, sb));
  const int chol_mode = ctx->opt.chol_precision;
  const int chol32 = chol_mode == NOLSM_CHOL_FP32;
  if (chol_mode == NOLSM_CHOL_DF64) {
    // slicing exponents, slice planes of one panel, work items of every panel's trailing update
    int64_t items = 0;
    for (const auto& bd : ctx->h_blocks) items += (int64_t)(bd.n_pad / kOzPanel + 1) * (bd.n_pad / 32 + 1);
    CK(dalloc(ctx, &ctx->d_oz_exp, (size_t)ctx->sum_pad));
    CK(dalloc(ctx, &ctx->d_oz_planes, (size_t)(kOzSlices * kOzPanel) * (size_t)ctx->sum_pad));
    CK(dalloc(ctx, &ctx->d_oz_items, (size_t)(2 * items)));
    int n_bins = 0;
    for (const auto& bd : ctx->h_blocks) n_bins = std::max(n_bins, bd.bin + 1);
    CK(dalloc(ctx, &ctx->d_oz_tmaps, (size_t)128 * (size_t)(3 + 2 * n_bins)));   // CUtensorMap: 128 bytes
    CK(dalloc(ctx, &ctx->d_oz_m, (size_t)kOzSlices * 4096 * (size_t)n_blocks));
    CK(dalloc(ctx, &ctx->d_oz_f, (size_t)68 * (size_t)n_blocks));
    int64_t tr_items = 0;
    for (const auto& bd : ctx->h_blocks) tr_items += (int64_t)(bd.n_pad / kOzPanel + 1) * (bd.n_pad / 128 + 1);
    CK(dalloc(ctx, &ctx->d_tr_items, (size_t)tr_items));
    CK(oz_prepare(ctx));
  }
  // FP32 path: SIMT inverse and congruence products with two-level sums; mixed: tensor cores (3 x TF32)
  ctx->cong_simt = !mixed;
  CK(phase_mark(ctx, NOLSM_PHASE_FACTOR));
  CK(launch_cholesky_inverse(ctx, sb, chol_mode));   // marks the inverse stage between its launches
  CK(phase_mark(ctx, NOLSM_PHASE_CONGRUENCE));
  CK(launch_congruence(ctx, ctx->d_t1));
  CK(phase_mark(ctx, NOLSM_PHASE_BUILD_REST));
  // the trace slab takes the factor's FP32 rounding (FP32 and double-float modes) or the FP64 factor
  const int l32 = chol32 || chol_mode == NOLSM_CHOL_DF64 || chol_mode == NOLSM_CHOL_DF64_SIMT;
  CK(launch_slabs_impl(ctx, l32 ? (const void*)(sb + ctx->sum_sq) : (const void*)sb, l32, ctx->d_t1));
  CK(dalloc(ctx, &ctx->d_rowd, (size_t)ctx->n_blocks * ctx->idx_stride));
  CK(dalloc(ctx, &ctx->d_rowr, (size_t)ctx->n_blocks * ctx->idx_stride));
  // the Gershgorin bounds and the mu-independent features in one pass over A0 (the mu-dependent
  // features are refreshed in O(n) per evaluation)
  CK(dalloc(ctx, &ctx->d_feat_static, (size_t)32 * ctx->n_blocks));
  CK(launch_bounds_features(ctx, ctx->d_feat_static));
  CK(dalloc(ctx, &ctx->d_own_diag, (size_t)std::max<int64_t>(ctx->sum_own, 1)));
  CK(launch_own_diag(ctx));
  ctx->n_launches += 1;
  if (ctx->opt.bounds == NOLSM_BOUNDS_LANCZOS) {
    nolsm_status st_l = run_lanczos(ctx, 0.0, 0, ctx->opt.lanczos_steps, nullptr);
    if (st_l != NOLSM_OK) return st_l;
  }
  CK(phase_mark(ctx, -1));
  // the products' tensor maps are encoded on the host while the build's kernels still run (the
  // upload follows them on the stream)
  if (mixed) CK(tc_prepare(ctx));
  nolsm_status st = check_device_flags(ctx);
  harvest_phases(ctx);
  if (st != NOLSM_OK) return st;
  ctx->h_lo.resize((size_t)n_blocks);
  ctx->h_hi.resize((size_t)n_blocks);
  CK(cudaMemcpy(ctx->h_lo.data(), ctx->d_lo, sizeof(double) * n_blocks, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(ctx->h_hi.data(), ctx->d_hi, sizeof(double) * n_blocks, cudaMemcpyDeviceToHost));
  ctx->h_own_diag.resize((size_t)ctx->sum_own);
  CK(cudaMemcpy(ctx->h_own_diag.data(), ctx->d_own_diag, sizeof(float) * ctx->sum_own, cudaMemcpyDeviceToHost));
  ctx->built = true;
  return NOLSM_OK;
}

namespace {

// Event pair around one matrix-product launch (recorded on the context stream).
// phase 1 / 2: one grouped product; phase 0: the persistent kernel (mixed paths only).
cudaError_t gemm_timed(nolsm_ctx* ctx, bool mixed, int phase, double mu) {
  const int k = ctx->gemm_ev_used;
  if ((int)ctx->gemm_ev.size() < 2 * (k + 1)) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) return e;
    ctx->gemm_ev.push_back(a);
    ctx->gemm_ev.push_back(b);
  }
  cudaError_t e = cudaEventRecord(ctx->gemm_ev[2 * k], ctx->stream);
  if (e != cudaSuccess) return e;
  e = phase == 0 ? launch_ns_pair(ctx, mu, ctx->pair_interleaved) : mixed ? launch_gemm_tc(ctx, phase)
                                                                     : launch_gemm_f32(ctx, phase);
  if (e != cudaSuccess) return e;
  ctx->gemm_ev_used = k + 1;
  ctx->n_launches += 1;
  ctx->n_gemm += 1;
  return cudaEventRecord(ctx->gemm_ev[2 * k + 1], ctx->stream);
}

// Sum the recorded product durations (the stream has been synchronised).
void harvest_gemm_events(nolsm_ctx* ctx) {
  for (int k = 0; k < ctx->gemm_ev_used; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->gemm_ev[2 * k], ctx->gemm_ev[2 * k + 1]) == cudaSuccess) ctx->gemm_ms += ms;
  }
  ctx->gemm_ev_used = 0;
}

}  // namespace

nolsm_status nolsm_sign_batch(nolsm_ctx* ctx, double mu, nolsm_sign_stats* out) {
  if (!ctx) return NOLSM_EINVAL;
  if (ctx->sticky != NOLSM_OK) return ctx->sticky;
  if (!ctx->built) return fail(ctx, NOLSM_ENOTBUILT, "nolsm_build_submatrices has not succeeded");
  if (!std::isfinite(mu)) return fail(ctx, NOLSM_EINVAL, "mu is not finite");
  const bool mixed = is_mixed(ctx);
  const int hk = half_kind(ctx);
  CK(cudaEventRecord(ctx->ev0, ctx->stream));
  CK(phase_mark(ctx, NOLSM_PHASE_SIGN_SETUP));
  int mode = ctx->opt.bounds;
  const float* pred = nullptr;
  if (mode == NOLSM_BOUNDS_GIVEN) {
    // kept or given bounds enter as the network's predictions do; none yet: Gershgorin
    if (ctx->given_blocks == ctx->n_blocks) {
      pred = ctx->d_given;
      mode = NOLSM_BOUNDS_LEARNED;
    } else {
      mode = NOLSM_BOUNDS_GERSHGORIN;
    }
  } else if (mode == NOLSM_BOUNDS_LEARNED) {
    if (!ctx->predictor) return fail(ctx, NOLSM_EINVAL, "learned bounds need nolsm_set_predictor");
    CK(dalloc(ctx, &ctx->d_feat, (size_t)32 * ctx->n_blocks));
    CK(dalloc(ctx, &ctx->d_pred, (size_t)3 * ctx->n_blocks));
    CK(launch_features_mu(ctx, mu, ctx->d_feat));
    CK(mlp_predict_on(ctx->predictor, ctx->stream, ctx->d_feat, ctx->n_blocks, ctx->d_pred));
    ctx->n_launches += 2;
    pred = ctx->d_pred;
  }
  // Schedule of every block.  The persistent kernels hold a product's tile list per CTA for n_pad <=
  // 4096; larger blocks always run per-product launches.  AUTO takes the measured table
  // (nolsm_set_schedule_table) when one is set, else the built-in rule (persistent while every
  // n_pad < 1024).  Blocks that prefer a persistent schedule form the queue of one persistent launch;
  // the others follow in per-product launches (a split evaluation).
  int max_pad = 0;
  for (const auto& bd : ctx->h_blocks) max_pad = std::max(max_pad, bd.n_pad);
  std::vector<int32_t> queue;
  bool interleaved = ctx->opt.schedule == NOLSM_SCHEDULE_PERSISTENT_INTERLEAVED;
  if (mixed) {
    const int sch = ctx->opt.schedule;
    if (sch == NOLSM_SCHEDULE_PERSISTENT || sch == NOLSM_SCHEDULE_PERSISTENT_INTERLEAVED) {
      if (max_pad <= kMaxDim)
        for (int32_t b = 0; b < ctx->n_blocks; ++b) queue.push_back(b);
    } else if (sch == NOLSM_SCHEDULE_AUTO && ctx->sched_pad.empty()) {
      if (max_pad < 1024)
        for (int32_t b = 0; b < ctx->n_blocks; ++b) queue.push_back(b);
    } else if (sch == NOLSM_SCHEDULE_AUTO) {
      // per block the entry of the smallest tabulated n_pad >= its own (the last one beyond); the
      // persistent variant is the one preferred by the larger share of the queue's n_pad^3
      double w_plain = 0.0, w_inter = 0.0;
      std::vector<size_t> entry((size_t)ctx->n_blocks);
      for (int32_t b = 0; b < ctx->n_blocks; ++b) {
        const int np = ctx->h_blocks[b].n_pad;
        size_t k = 0;
        while (k + 1 < ctx->sched_pad.size() && ctx->sched_pad[k] < np) ++k;
        entry[b] = k;
        const int kind = ctx->sched_kind[k];
        if (np > kMaxDim || kind == NOLSM_SCHEDULE_PER_PRODUCT) continue;
        queue.push_back(b);
        (kind == NOLSM_SCHEDULE_PERSISTENT_INTERLEAVED ? w_inter : w_plain) += (double)np * np * np;
      }
      interleaved = w_inter > w_plain;
      if (!ctx->sched_ms.empty() && !queue.empty()) {
        // With measured times: predicted products time of the batch under each single schedule (the
        // sum of the blocks' per-block times, measured in full batches) and under the split (each
        // block at its entry's best, plus the tail of the persistent launch: its last block runs on
        // one cluster while the others idle, about that block's time on the whole GPU times the
        // clusters).  The smallest prediction decides.
        const auto ms = [&](int32_t b, int s) { return ctx->sched_ms[3 * entry[b] + s]; };
        const int ncl = std::max(1, ctx->pair_clusters > 0 ? ctx->pair_clusters : ctx->num_sms / 2);
        double t_p = 0.0, t_pp = 0.0, t_i = 0.0, t_split = 0.0, tail = 0.0;
        std::vector<char> in_q((size_t)ctx->n_blocks, 0);
        for (int32_t b : queue) in_q[b] = 1;
        for (int32_t b = 0; b < ctx->n_blocks; ++b) {
          t_p += ms(b, 0);
          t_pp += ms(b, 1);
          t_i += ms(b, 2);
          const int qs = interleaved ? 2 : 0;
          t_split += in_q[b] ? ms(b, qs) : ms(b, 1);
          if (in_q[b]) tail = std::max(tail, ms(b, qs) * ncl);
        }
        const bool all_fit = max_pad <= kMaxDim;
        const double best_single = all_fit ? std::min(t_pp, std::min(t_p, t_i)) : t_pp;
        if ((int32_t)queue.size() < ctx->n_blocks && t_split + tail < best_single) {
          // keep the split
        } else {
          queue.clear();
          if (all_fit && best_single < t_pp) {
            interleaved = t_i < t_p;
            for (int32_t b = 0; b < ctx->n_blocks; ++b) queue.push_back(b);
          }
        }
      }
      // largest blocks first: the queue's tail is then made of short jobs
      std::stable_sort(queue.begin(), queue.end(),
                       [&](int32_t a, int32_t c) { return ctx->h_blocks[a].n_pad > ctx->h_blocks[c].n_pad; });
    }
  }
  const bool persistent = !queue.empty() && (int32_t)queue.size() == ctx->n_blocks;
  const bool split = !queue.empty() && !persistent;
  ctx->pair_interleaved = interleaved;
  ctx->n_queue = (int32_t)queue.size();
  ctx->last_schedule = persistent ? (interleaved ? NOLSM_SCHEDULE_PERSISTENT_INTERLEAVED : NOLSM_SCHEDULE_PERSISTENT)
                                  : split ? -2 : NOLSM_SCHEDULE_PER_PRODUCT;
  if (split) {
    CK(dalloc(ctx, &ctx->d_queue, queue.size()));
    CK(cudaMemcpyAsync(ctx->d_queue, queue.data(), sizeof(int32_t) * queue.size(), cudaMemcpyHostToDevice,
                       ctx->stream));
  }
  if (ctx->opt.fp8_iters > 0 && (!persistent || ctx->pair_interleaved))
    return fail(ctx, NOLSM_EINVAL, "fp8_iters needs a mixed-precision path on the persistent schedule");
  // X_0 of the per-product blocks (in a split evaluation every block's; the persistent kernel forms
  // its own blocks' X_0 again)
  CK(launch_ns_init(ctx, mu, hk, mode, mode == NOLSM_BOUNDS_LANCZOS ? ctx->d_lz : nullptr, pred, !persistent));
  ctx->n_launches += persistent ? 1 : 2;
  const int tile_n = mixed ? tc_tile_n() : kTile;
  const int check_every = 4;
  ctx->gemm_ev_used = 0;
  CK(phase_mark(ctx, NOLSM_PHASE_PRODUCTS));
  // the whole iteration of the queued blocks, on the device; the per-product loop below then sees
  // them converged (or failed) and runs the remaining blocks
  if (!queue.empty()) CK(gemm_timed(ctx, mixed, 0, mu));
  CK(launch_set_loop_mu(ctx, mu));   // the restart kernels read mu on the device
  const bool restart = mode != NOLSM_BOUNDS_GERSHGORIN;
  if (!persistent && ctx->opt.loop == NOLSM_LOOP_GRAPH) {
    // the whole per-product iteration as one graph launch: a while node whose body is one iteration
    // and whose condition the body's last kernel sets on the device (no host round trip)
    const int64_t key[6] = {ctx->build_gen, ctx->opt.precision, restart ? 1 : 0, tile_n, ctx->opt.max_iter,
                            ctx->opt.wait_budget};
    if (!ctx->loop_exec || !std::equal(key, key + 6, ctx->loop_key)) {
      release_loop_graph(ctx);
      cudaGraph_t g = nullptr, body = nullptr;
      cudaGraphConditionalHandle h;
      CK(cudaGraphCreate(&g, 0));
      ctx->loop_graph = g;
      CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
      body = np.conditional.phGraph_out[0];
      // captured on a stream of the context's own (the caller's may be the legacy default stream, which
      // cannot be captured); the launchers below issue to ctx->stream, so it points there meanwhile
      if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
      cudaStream_t user_stream = ctx->stream;
      CK(cudaStreamBeginCaptureToGraph(ctx->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      ctx->stream = ctx->cap_stream;
      cudaError_t ce = launch_ns_tiles_n(ctx, tile_n);
      if (ce == cudaSuccess) ce = mixed ? launch_gemm_tc(ctx, 1) : launch_gemm_f32(ctx, 1);
      if (ce == cudaSuccess) ce = launch_ns_check_impl(ctx, ctx->d_tol, restart);
      if (ce == cudaSuccess) ce = launch_ns_tiles_n(ctx, tile_n);
      if (ce == cudaSuccess) ce = mixed ? launch_gemm_tc(ctx, 2) : launch_gemm_f32(ctx, 2);
      if (ce == cudaSuccess) ce = launch_ns_advance(ctx);
      if (ce == cudaSuccess && restart) ce = launch_ns_restart(ctx, hk);
      if (ce == cudaSuccess) ce = launch_loop_cond(ctx, h);
      cudaGraph_t captured = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream, &captured);
      ctx->stream = user_stream;
      CK(ce);
      CK(ee);
      CK(cudaGraphInstantiate(&ctx->loop_exec, g, 0));
      std::copy(key, key + 6, ctx->loop_key);
    }
    CK(launch_loop_reset(ctx));
    const int k = ctx->gemm_ev_used;   // the products' interval is the graph's
    if ((int)ctx->gemm_ev.size() < 2 * (k + 1)) {
      cudaEvent_t a, b;
      CK(cudaEventCreate(&a));
      CK(cudaEventCreate(&b));
      ctx->gemm_ev.push_back(a);
      ctx->gemm_ev.push_back(b);
    }
    CK(cudaEventRecord(ctx->gemm_ev[2 * k], ctx->stream));
    CK(cudaGraphLaunch(ctx->loop_exec, ctx->stream));
    CK(cudaEventRecord(ctx->gemm_ev[2 * k + 1], ctx->stream));
    ctx->gemm_ev_used = k + 1;
    ctx->n_launches += 3;
    ctx->n_gemm += 1;
  }
  for (int it = 0; !persistent && ctx->opt.loop != NOLSM_LOOP_GRAPH && it <= ctx->opt.max_iter; ++it) {
    CK(launch_ns_tiles_n(ctx, tile_n));
    CK(gemm_timed(ctx, mixed, 1, mu));
    CK(launch_ns_check_impl(ctx, ctx->d_tol, restart));
    CK(launch_ns_tiles_n(ctx, tile_n));
    CK(gemm_timed(ctx, mixed, 2, mu));
    CK(launch_ns_advance(ctx));
    ctx->n_launches += 4;
    if (restart) {
      CK(launch_ns_restart(ctx, hk));
      ctx->n_launches += 2;
    }
    if (it % check_every == check_every - 1 || it == ctx->opt.max_iter) {
      CK(cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, sizeof(DevFlags), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      harvest_gemm_events(ctx);
      if (ctx->h_flags->error != 0 || ctx->h_flags->n_active == 0) break;
    }
  }
  CK(phase_mark(ctx, NOLSM_PHASE_SLAB));
  CK(launch_slab_traces(ctx, hk));
  ctx->n_launches += 1;   // sum_traces (the slab launches count themselves)
  CK(phase_mark(ctx, -1));
  CK(cudaEventRecord(ctx->ev1, ctx->stream));
  nolsm_status st = check_device_flags(ctx);
  harvest_gemm_events(ctx);
  harvest_phases(ctx);
  if (st != NOLSM_OK) return st;
  ctx->last_mu = mu;
  ctx->have_sign = true;
  ctx->have_density = false;
  {
    // executed product flops of this evaluation (counters), from the per-block iteration counts
    std::vector<NsState> hs((size_t)ctx->n_blocks);
    CK(cudaMemcpy(hs.data(), ctx->d_state, sizeof(NsState) * ctx->n_blocks, cudaMemcpyDeviceToHost));
    double fe = 0.0;
    for (int32_t b = 0; b < ctx->n_blocks; ++b) {
      const double np = ctx->h_blocks[b].n_pad;
      fe += (2.0 * hs[b].iters + 1.0) * np * np * (np + kTile);
    }
    ctx->gemm_flops += fe;
  }
  nolsm_sign_stats s{};
  s.mu = mu;
  s.n_electrons = ctx->opt.spin_factor * ctx->h_flags->sum_n;
  s.band_energy = ctx->opt.spin_factor * ctx->h_flags->sum_e;
  s.n_blocks = ctx->n_blocks;
  if (out) {
    std::vector<NsState> hs((size_t)ctx->n_blocks);
    CK(cudaMemcpy(hs.data(), ctx->d_state, sizeof(NsState) * ctx->n_blocks, cudaMemcpyDeviceToHost));
    ctx->h_iters.resize((size_t)ctx->n_blocks);
    int64_t sum_it = 0;
    s.iters_min = INT32_MAX;
    s.iters_max = 0;
    double fp = 0.0, fe = 0.0;
    for (int32_t b = 0; b < ctx->n_blocks; ++b) {
      const int it = hs[b].iters;
      ctx->h_iters[b] = it;
      sum_it += it;
      s.iters_min = std::min(s.iters_min, it);
      s.iters_max = std::max(s.iters_max, it);
      s.max_residual = std::max(s.max_residual, (double)hs[b].res);
      s.n_restarted += hs[b].restarts > 0;
      const double n = ctx->h_blocks[b].n, np = ctx->h_blocks[b].n_pad;
      // it full iterations (2 products) plus the first product of the converged check
      fp += (2.0 * it + 1.0) * 2.0 * n * n * n;
      // executed: upper-triangular 128-row tiles only, np^2 (np + 128) per product
      fe += (2.0 * it + 1.0) * np * np * (np + kTile);
    }
    s.iters_avg = (double)sum_it / ctx->n_blocks;
    s.flops_paper = fp;
    s.flops_executed = fe;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    s.ms = ms;
    *out = s;
  }
  ctx->last_stats = s;
  return NOLSM_OK;
}

nolsm_status nolsm_set_mu(nolsm_ctx* ctx, double n_electrons, double mu_lo, double mu_hi, double tol_n,
                          int32_t max_steps, double* mu_out, double* n_out, int32_t* steps_out) {
  if (!ctx) return NOLSM_EINVAL;
  if (ctx->sticky != NOLSM_OK) return ctx->sticky;
  if (!ctx->built) return fail(ctx, NOLSM_ENOTBUILT, "nolsm_build_submatrices has not succeeded");
  if (!(n_electrons > 0) || !(tol_n >= 0) || max_steps <= 0) return fail(ctx, NOLSM_EINVAL, "bad bisection arguments");
  double lo = mu_lo, hi = mu_hi;
  const double total = ctx->opt.spin_factor * (double)ctx->sum_own;   // N(mu) above every eigenvalue
  if (!(lo < hi)) {
    lo = *std::min_element(ctx->h_lo.begin(), ctx->h_lo.end());
    hi = *std::max_element(ctx->h_hi.begin(), ctx->h_hi.end());
    if (!(n_electrons < total)) return fail(ctx, NOLSM_EBRACKET, "electron count not below the number of own columns");
  }
  const double lo0 = lo, hi0 = hi;
  double mu = 0.5 * (lo + hi), n_mu = 0.0;
  {
    // Aufbau first point: between the k-th and (k+1)-th smallest own-column diagonal entries of A0
    const int64_t k = (int64_t)std::floor(n_electrons / ctx->opt.spin_factor);
    std::vector<float> d = ctx->h_own_diag;
    if (ctx->opt.mu_first == NOLSM_MU_FIRST_AUFBAU && k >= 1 && k < (int64_t)d.size()) {
      std::nth_element(d.begin(), d.begin() + k, d.end());
      const float above = d[(size_t)k];
      const float below = *std::max_element(d.begin(), d.begin() + k);
      const double guess = 0.5 * ((double)below + (double)above);
      if (guess > lo && guess < hi) mu = guess;
    }
  }
  int steps = 0;
  nolsm_sign_stats s;
  while (true) {
    nolsm_status st = nolsm_sign_batch(ctx, mu, &s);
    if (st != NOLSM_OK) return st;
    ++steps;
    n_mu = s.n_electrons;
    if (std::fabs(n_mu - n_electrons) <= tol_n * n_electrons) break;
    if (steps >= max_steps || hi - lo < 1e-10) break;
    if (n_mu < n_electrons) lo = mu; else hi = mu;
    mu = 0.5 * (lo + hi);
  }
  if (std::fabs(n_mu - n_electrons) > tol_n * n_electrons && (mu - lo0 < 1e-9 || hi0 - mu < 1e-9))
    return fail(ctx, NOLSM_EBRACKET, "N(mu) does not bracket the electron count in [mu_lo, mu_hi]");
  if (mu_out) *mu_out = mu;
  if (n_out) *n_out = n_mu;
  if (steps_out) *steps_out = steps;
  return NOLSM_OK;
}

nolsm_status nolsm_density(nolsm_ctx* ctx, double* d_val, int32_t memory) {
  if (!ctx) return NOLSM_EINVAL;
  if (ctx->sticky != NOLSM_OK) return ctx->sticky;
  if (!ctx->have_sign) return fail(ctx, NOLSM_ENOTBUILT, "nolsm_sign_batch has not run");
  if (memory != NOLSM_MEM_DEVICE && memory != NOLSM_MEM_HOST) return fail(ctx, NOLSM_EINVAL, "bad memory kind");
  CK(phase_mark(ctx, NOLSM_PHASE_DENSITY));
  CK(launch_density(ctx));
  CK(phase_mark(ctx, -1));
  ctx->n_launches += 1;
  if (d_val) {
    CK(cudaMemcpyAsync(d_val, ctx->d_dval, sizeof(double) * ctx->nnz,
                       memory == NOLSM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, ctx->stream));
    if (memory == NOLSM_MEM_HOST) {
      nolsm_status st = check_device_flags(ctx);
      if (st != NOLSM_OK) return st;
    }
  }
  ctx->have_density = true;
  return NOLSM_OK;
}

nolsm_status nolsm_band_energy(nolsm_ctx* ctx, double* e_out) {
  if (!ctx || !e_out) return NOLSM_EINVAL;
  if (ctx->sticky != NOLSM_OK) return ctx->sticky;
  if (!ctx->have_density) return fail(ctx, NOLSM_ENOTBUILT, "nolsm_density has not run");
  CK(phase_mark(ctx, NOLSM_PHASE_ENERGY));
  CK(launch_band_energy(ctx));
  CK(phase_mark(ctx, -1));
  ctx->n_launches += 2;
  nolsm_status st = check_device_flags(ctx);
  harvest_phases(ctx);
  if (st != NOLSM_OK) return st;
  *e_out = ctx->opt.spin_factor * ctx->h_flags->energy;
  return NOLSM_OK;
}

nolsm_status nolsm_block_traces(const nolsm_ctx* ctx, double* n_out, double* e_out) {
  if (!ctx || !ctx->have_sign) return NOLSM_ENOTBUILT;
  if (!n_out && !e_out) return NOLSM_EINVAL;
  const int64_t nb = ctx->n_blocks;
  const int64_t n = ctx->traces_per_unit ? (int64_t)ctx->h_slab_units.size() / 4 : nb;
  std::vector<double> bn((size_t)n), be((size_t)n);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess ||
      cudaMemcpy(bn.data(), ctx->d_bn, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(be.data(), ctx->d_be, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return NOLSM_ECUDA;
  std::vector<double> sn((size_t)nb, 0.0), se((size_t)nb, 0.0);
  for (int64_t u = 0; u < n; ++u) {
    const int32_t b = ctx->traces_per_unit ? ctx->h_slab_units[(size_t)(4 * u)] : (int32_t)u;
    sn[b] += bn[u];
    se[b] += be[u];
  }
  for (int64_t b = 0; b < nb; ++b) {
    if (n_out) n_out[b] = ctx->opt.spin_factor * sn[b];
    if (e_out) e_out[b] = ctx->opt.spin_factor * se[b];
  }
  return NOLSM_OK;
}

nolsm_status nolsm_own_diagonal(const nolsm_ctx* ctx, int64_t* count, float* out) {
  if (!ctx || !ctx->built || !count) return NOLSM_EINVAL;
  *count = (int64_t)ctx->h_own_diag.size();
  if (out) std::copy(ctx->h_own_diag.begin(), ctx->h_own_diag.end(), out);
  return NOLSM_OK;
}

nolsm_status nolsm_set_schedule_table(nolsm_ctx* ctx, int32_t n_entries, const int32_t* n_pad,
                                      const int32_t* schedule, const double* ms_per_block) {
  if (!ctx) return NOLSM_EINVAL;
  if (n_entries < 0 || (n_entries > 0 && (!n_pad || !schedule))) return fail(ctx, NOLSM_EINVAL, "bad schedule table");
  for (int32_t i = 0; i < n_entries; ++i) {
    if (n_pad[i] <= 0 || (i > 0 && n_pad[i] <= n_pad[i - 1])) return fail(ctx, NOLSM_EINVAL, "table sizes must ascend");
    if (schedule[i] != NOLSM_SCHEDULE_PERSISTENT && schedule[i] != NOLSM_SCHEDULE_PER_PRODUCT &&
        schedule[i] != NOLSM_SCHEDULE_PERSISTENT_INTERLEAVED)
      return fail(ctx, NOLSM_EINVAL, "table schedules must be PERSISTENT, PER_PRODUCT or PERSISTENT_INTERLEAVED");
  }
  if (ms_per_block)
    for (int32_t i = 0; i < 3 * n_entries; ++i)
      if (!(ms_per_block[i] > 0) || !std::isfinite(ms_per_block[i]))
        return fail(ctx, NOLSM_EINVAL, "table times must be positive and finite");
  ctx->sched_pad.assign(n_pad, n_pad + n_entries);
  ctx->sched_kind.assign(schedule, schedule + n_entries);
  if (ms_per_block) ctx->sched_ms.assign(ms_per_block, ms_per_block + 3 * n_entries);
  else ctx->sched_ms.clear();
  return NOLSM_OK;
}

nolsm_status nolsm_last_schedule(const nolsm_ctx* ctx, int32_t* schedule, int32_t* persistent_blocks) {
  if (!ctx || !ctx->have_sign) return NOLSM_ENOTBUILT;
  if (schedule) *schedule = ctx->last_schedule;
  if (persistent_blocks) *persistent_blocks = ctx->n_queue;
  return NOLSM_OK;
}

nolsm_status nolsm_block_info(const nolsm_ctx* ctx, int32_t b, int32_t* n_b, int32_t* n_cols) {
  if (!ctx || !ctx->built || b < 0 || b >= ctx->n_blocks) return NOLSM_EINVAL;
  if (n_b) *n_b = ctx->h_blocks[b].n;
  if (n_cols) *n_cols = ctx->h_blocks[b].c;
  return NOLSM_OK;
}

nolsm_status nolsm_block_index_set(const nolsm_ctx* ctx, int32_t b, int32_t* idx_out) {
  if (!ctx || !ctx->built || b < 0 || b >= ctx->n_blocks || !idx_out) return NOLSM_EINVAL;
  const BlockDesc& bd = ctx->h_blocks[b];
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NOLSM_ECUDA;
  if (cudaMemcpy(idx_out, ctx->d_idx + bd.off_idx, sizeof(int32_t) * bd.n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return NOLSM_ECUDA;
  return NOLSM_OK;
}

nolsm_status nolsm_block_bounds(const nolsm_ctx* ctx, double* lo, double* hi) {
  if (!ctx || !ctx->built) return NOLSM_EINVAL;
  if (lo) std::memcpy(lo, ctx->h_lo.data(), sizeof(double) * ctx->n_blocks);
  if (hi) std::memcpy(hi, ctx->h_hi.data(), sizeof(double) * ctx->n_blocks);
  return NOLSM_OK;
}

nolsm_status nolsm_block_features(nolsm_ctx* ctx, double mu, float* feat) {
  if (!ctx || !ctx->built || !feat || !std::isfinite(mu)) return NOLSM_EINVAL;
  if (launch_features_mu(ctx, mu, feat) != cudaSuccess) return NOLSM_ECUDA;
  ctx->n_launches += 1;
  return NOLSM_OK;
}

nolsm_status nolsm_block_lanczos(nolsm_ctx* ctx, int32_t steps, int32_t op, float* out) {
  if (!ctx || !ctx->built || !out || steps < 1 || steps > 64 || op < 0 || op > 1) return NOLSM_EINVAL;
  if (op == 1 && !ctx->have_sign) return NOLSM_ENOTBUILT;
  if (ctx->sticky != NOLSM_OK) return ctx->sticky;
  return run_lanczos(ctx, ctx->last_mu, op, steps, out);
}

nolsm_status nolsm_keep_bounds(nolsm_ctx* ctx, int32_t steps) {
  if (!ctx || !ctx->built || steps < 1 || steps > 64) return NOLSM_EINVAL;
  if (!ctx->have_sign) return NOLSM_ENOTBUILT;
  if (ctx->sticky != NOLSM_OK) return ctx->sticky;
  // |A0 - mu| (needs the current X) into the first half of d_lz1, A0 into the second half (d_lz,
  // which the Lanczos bounds mode reads, stays as it is)
  CK(dalloc(ctx, &ctx->d_lz1, (size_t)8 * ctx->n_blocks));
  CK(dalloc(ctx, &ctx->d_given, (size_t)3 * ctx->n_blocks));
  float* lz_abs = ctx->d_lz1;
  float* lz_a0 = ctx->d_lz1 + (size_t)4 * ctx->n_blocks;
  nolsm_status st = run_lanczos(ctx, ctx->last_mu, 1, steps, lz_abs);
  if (st != NOLSM_OK) return st;
  st = run_lanczos(ctx, ctx->last_mu, 0, steps, lz_a0);
  if (st != NOLSM_OK) return st;
  CK(launch_given_from_lanczos(ctx, lz_a0, lz_abs, ctx->d_given));
  ctx->n_launches += 1;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->given_blocks = ctx->n_blocks;
  return NOLSM_OK;
}

nolsm_status nolsm_set_block_bounds(nolsm_ctx* ctx, const float* bounds, int32_t memory) {
  if (!ctx || !ctx->built || !bounds || (memory != NOLSM_MEM_HOST && memory != NOLSM_MEM_DEVICE)) return NOLSM_EINVAL;
  if (ctx->sticky != NOLSM_OK) return ctx->sticky;
  CK(dalloc(ctx, &ctx->d_given, (size_t)3 * ctx->n_blocks));
  CK(cudaMemcpyAsync(ctx->d_given, bounds, sizeof(float) * 3 * ctx->n_blocks,
                     memory == NOLSM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->given_blocks = ctx->n_blocks;
  return NOLSM_OK;
}

nolsm_status nolsm_set_predictor(nolsm_ctx* ctx, const nolsm_mlp* mlp) {
  if (!ctx) return NOLSM_EINVAL;
  ctx->predictor = mlp;
  return NOLSM_OK;
}

nolsm_status nolsm_counters(nolsm_ctx* ctx, int64_t* launches, int64_t* gemm_launches, double* gemm_ms,
                            double* gemm_flops, int32_t reset) {
  if (!ctx) return NOLSM_EINVAL;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NOLSM_ECUDA;
  harvest_gemm_events(ctx);
  if (launches) *launches = ctx->n_launches;
  if (gemm_launches) *gemm_launches = ctx->n_gemm;
  if (gemm_ms) *gemm_ms = ctx->gemm_ms;
  if (gemm_flops) *gemm_flops = ctx->gemm_flops;
  if (reset) {
    ctx->n_launches = ctx->n_gemm = 0;
    ctx->gemm_ms = ctx->gemm_flops = 0.0;
  }
  return NOLSM_OK;
}

nolsm_status nolsm_set_wait_budget(nolsm_ctx* ctx, int64_t budget) {
  if (!ctx || budget < 1) return NOLSM_EINVAL;
  ctx->opt.wait_budget = budget;
  return NOLSM_OK;
}

nolsm_status nolsm_phase_times(nolsm_ctx* ctx, double* ms, int32_t n, int32_t reset) {
  if (!ctx || n < 0 || n > NOLSM_NUM_PHASES || (n > 0 && !ms)) return NOLSM_EINVAL;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NOLSM_ECUDA;
  harvest_phases(ctx);
  for (int32_t p = 0; p < n; ++p) ms[p] = ctx->phase_ms[p];
  if (reset)
    for (double& v : ctx->phase_ms) v = 0.0;
  return NOLSM_OK;
}

nolsm_status nolsm_block_state(const nolsm_ctx* ctx, int32_t* iters, double* residual, int32_t* status) {
  if (!ctx || !ctx->built) return NOLSM_EINVAL;
  std::vector<NsState> hs((size_t)ctx->n_blocks);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NOLSM_ECUDA;
  if (cudaMemcpy(hs.data(), ctx->d_state, sizeof(NsState) * ctx->n_blocks, cudaMemcpyDeviceToHost) != cudaSuccess)
    return NOLSM_ECUDA;
  for (int32_t b = 0; b < ctx->n_blocks; ++b) {
    if (iters) iters[b] = hs[b].iters;
    if (residual) residual[b] = hs[b].res;
    if (status) status[b] = hs[b].status;
  }
  return NOLSM_OK;
}

// The double-float modes leave the factor as pairs (h, l) of floats in the 8 bytes of each double.
static bool factor_in_pairs(const nolsm_ctx* ctx) {
  return ctx->opt.chol_precision == NOLSM_CHOL_DF64 || ctx->opt.chol_precision == NOLSM_CHOL_DF64_SIMT;
}
static double pair_value(double raw) {
  float hl[2];
  std::memcpy(hl, &raw, sizeof(hl));
  return (double)hl[0] + (double)hl[1];
}

nolsm_status nolsm_block_factor(const nolsm_ctx* ctx, int32_t b, double* out) {
  if (!ctx || !ctx->built || b < 0 || b >= ctx->n_blocks || !out) return NOLSM_EINVAL;
  const BlockDesc& bd = ctx->h_blocks[b];
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NOLSM_ECUDA;
  if (ctx->opt.chol_precision == NOLSM_CHOL_FP32) {
    std::vector<float> l((size_t)bd.n * bd.n);
    const float* src = reinterpret_cast<const float*>(ctx->d_sb + ctx->sum_sq) + bd.off_mat;
    if (cudaMemcpy2D(l.data(), sizeof(float) * bd.n, src, sizeof(float) * bd.n_pad, sizeof(float) * bd.n, bd.n,
                     cudaMemcpyDeviceToHost) != cudaSuccess)
      return NOLSM_ECUDA;
    for (size_t i = 0; i < l.size(); ++i) out[i] = l[i];
  } else {
    if (cudaMemcpy2D(out, sizeof(double) * bd.n, ctx->d_sb + bd.off_mat, sizeof(double) * bd.n_pad,
                     sizeof(double) * bd.n, bd.n, cudaMemcpyDeviceToHost) != cudaSuccess)
      return NOLSM_ECUDA;
    if (factor_in_pairs(ctx))
      for (size_t i = 0; i < (size_t)bd.n * bd.n; ++i) out[i] = pair_value(out[i]);
  }
  for (int r = 0; r < bd.n; ++r)
    for (int c = r + 1; c < bd.n; ++c) out[(size_t)r * bd.n + c] = 0.0;
  return NOLSM_OK;
}

nolsm_status nolsm_block_matrix(const nolsm_ctx* ctx, int32_t b, int32_t which, float* out) {
  if (!ctx || !ctx->built || b < 0 || b >= ctx->n_blocks || !out || which < 0 || which > 5) return NOLSM_EINVAL;
  const BlockDesc& bd = ctx->h_blocks[b];
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return NOLSM_ECUDA;
  if (which == 5) {
    // the factor: FP32 copy in the scratch half of the S pool for CHOL_FP32, else the FP64 lower triangle
    const size_t nn = (size_t)bd.n * bd.n;
    if (ctx->opt.chol_precision == NOLSM_CHOL_FP32) {
      const float* src = reinterpret_cast<const float*>(ctx->d_sb + ctx->sum_sq) + bd.off_mat;
      if (cudaMemcpy2D(out, sizeof(float) * bd.n, src, sizeof(float) * bd.n_pad, sizeof(float) * bd.n, bd.n,
                       cudaMemcpyDeviceToHost) != cudaSuccess)
        return NOLSM_ECUDA;
    } else {
      std::vector<double> l(nn);
      if (cudaMemcpy2D(l.data(), sizeof(double) * bd.n, ctx->d_sb + bd.off_mat, sizeof(double) * bd.n_pad,
                       sizeof(double) * bd.n, bd.n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return NOLSM_ECUDA;
      for (size_t i = 0; i < nn; ++i) out[i] = (float)(factor_in_pairs(ctx) ? pair_value(l[i]) : l[i]);
    }
    for (int r = 0; r < bd.n; ++r)
      for (int c = r + 1; c < bd.n; ++c) out[(size_t)r * bd.n + c] = 0.f;
    return NOLSM_OK;
  }
  if (which <= 1) {
    const float* src = (which == 0 ? ctx->d_a0 : ctx->d_linv) + bd.off_mat;
    if (cudaMemcpy2D(out, sizeof(float) * bd.n, src, sizeof(float) * bd.n_pad, sizeof(float) * bd.n, bd.n,
                     cudaMemcpyDeviceToHost) != cudaSuccess)
      return NOLSM_ECUDA;
    if (which == 1)   // L^-1 is lower triangular (the mixed paths leave the blocks above unwritten)
      for (int r = 0; r < bd.n; ++r)
        for (int c = r + 1; c < bd.n; ++c) out[(size_t)r * bd.n + c] = 0.f;
    return NOLSM_OK;
  }
  const void* pool = which == 2 ? ctx->d_x[0] : which == 3 ? ctx->d_x[1] : ctx->d_b;
  const int hk = half_kind(ctx);
  const size_t es = hk ? 2 : 4;
  std::vector<uint8_t> raw((size_t)bd.n * bd.n * es);
  if (cudaMemcpy2D(raw.data(), es * bd.n, reinterpret_cast<const uint8_t*>(pool) + es * bd.off_mat, es * bd.n_pad,
                   es * bd.n, bd.n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return NOLSM_ECUDA;
  for (size_t i = 0; i < (size_t)bd.n * bd.n; ++i) {
    if (hk == 0) out[i] = reinterpret_cast<const float*>(raw.data())[i];
    else if (hk == 1) out[i] = __half2float(reinterpret_cast<const __half*>(raw.data())[i]);
    else out[i] = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(raw.data())[i]);
  }
  return NOLSM_OK;
}

}  // extern "C"
