// Internal declarations shared by the translation units of libnolsm.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/nolsm.h"

namespace nolsm {

// Output tile edge of every matrix-product kernel; submatrices are padded to it.
constexpr int kTile = 128;
constexpr int kMaxDim = 4096;           // index-set stride while every block has n_b <= 4096
constexpr int kMaxDimLarge = 16384;     // largest n_b (index-set stride when some block exceeds 4096)
constexpr int kMaxCandidates = 32768;   // own-column rows + extra indices of one block

inline int pad_dim(int n) { return (n + kTile - 1) / kTile * kTile; }

// One submatrix (device-resident table, one entry per block).
struct BlockDesc {
  int32_t n;        // |I_b|
  int32_t n_pad;    // n rounded up to kTile
  int32_t c;        // |C_b|, own columns
  int32_t col0;     // offset of the block's own columns in the blk_cols array
  int32_t bin;      // size bin (blocks of one n_pad are stored contiguously, bin by bin)
  int32_t pos;      // position of the block inside its bin
  int32_t slab_row; // row of the block's first own column in its bin's stack of slabs (c rows of n_pad)
  int32_t row_off;  // sum of n_pad over the blocks laid out before this one (per-row scratch pools)
  int64_t off_idx;  // I_b in idx pool (n int32, ascending); own positions follow in own pool
  int64_t off_own;  // local positions of the own columns (c int32)
  int64_t off_mat;  // n_pad*n_pad element offset in every square pool
  int64_t off_slab; // n_pad*c element offset in every slab pool (column-major, ld = n_pad)
};

// One 128-row tile of the tensor-core TRSM with what its roles need about the block, resolved on
// the host: a role loads one record instead of the dependent chain item -> block descriptor.
struct TrItem {
  int32_t b, m0, n, ld;       // block, first row of the tile, n_b, n_pad
  int32_t row_off, pos, bin, pad;
  int64_t off_mat;
};

// Newton-Schulz state of one block during a sign evaluation.
struct NsState {
  float alpha;      // X_0 = (A0 - mu I) / alpha
  float l;          // lower bound of |eig(X_k)| for the scaled iteration (1 = plain)
  float a;          // scaling of the current step: X+ = a X (3 - a^2 X^2) / 2
  float res;        // ||X_k^2 - I||_F of the last product
  float res_prev;
  int32_t iters;    // completed matrix iterations
  int32_t status;   // kActive / kConverged / kRestart / kFailed
  int32_t cur;      // which X buffer holds the iterate (0/1)
  int32_t grow;     // consecutive residual increases
  int32_t restarts;
};

enum : int32_t { kActive = 0, kConverged = 1, kRestart = 2, kFailed = 3 };

// Scaled Newton-Schulz step coefficient for a lower bound l of |eig(X)| in (0, 1]
// (Chen & Chow 2014): a = sqrt(3 / (1 + l + l^2)) maps [l, 1] onto [l', 1] with the two
// ends equal; l = 1 gives the unscaled iteration of Eq. 6.
__device__ __forceinline__ float cc_scale(float l) { return (l >= 1.f) ? 1.f : sqrtf(3.f / (1.f + l + l * l)); }
__device__ __forceinline__ float cc_next(float l, float a) {
  const float v = 0.5f * a * l * (3.f - a * a * l * l);
  return (v > 1.f - 1e-6f) ? 1.f : v;
}

// A tile of a grouped matrix product: block, first output row, first output column.
struct Tile {
  int32_t block, m0, n0, kend;
};

// Device-side counters and flags of one context.
struct DevFlags {
  int32_t error;        // first device error code (nolsm_status), 0 = none
  int32_t n_tiles;      // tiles in the current list
  int32_t n_active;     // blocks still iterating
  int32_t queue;        // next block to claim (persistent schedule)
  int32_t slab_queue[2];  // next unit to claim by the tensor-core slab kernels (narrow, wide)
  int32_t oversize;     // blocks whose index set exceeded the current stride (the build widens it)
  double sum_n;         // sum of block traces Tr(S D) over own columns
  double sum_e;         // same for Tr(H D)
  double energy;        // band energy reduction
  double mu;            // chemical potential of the current sign evaluation (read by the restart kernels)
  int32_t loop_iter;    // iterations run by the captured per-product loop
  int32_t pad3;
};

}  // namespace nolsm

struct nolsm_ctx {
  nolsm_options opt;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  int pair_clusters = 0;        // resident 2-CTA clusters of the persistent product kernel
  bool pair_interleaved = false;  // the persistent kernel takes two blocks per cluster
  void* d_cg_tmaps = nullptr;   // tensor maps of the congruence kernel (FP32 pools, per bin)
  size_t cg_tmap_cap = 0;
  int64_t cg_maps_gen = -1;     // build whose pools the maps describe, and its T1 pool
  const float* cg_maps_t1 = nullptr;
  // host copies of uploaded tensor maps and per-block tolerances: the sources of their asynchronous
  // uploads stay alive until the next build, so the uploads need no wait on the stream
  std::vector<uint8_t> h_cg_maps, h_oz_maps, h_tc_maps;
  std::vector<float> h_tol;
  bool cong_simt = false;       // congruence on the SIMT FP32 products (tests compare both)
  nolsm_status sticky = NOLSM_OK;
  std::string last_error;

  // build products
  bool built = false;
  bool have_sign = false;
  bool have_density = false;
  int32_t n_blocks = 0;
  int64_t n = 0, nnz = 0;
  std::vector<nolsm::BlockDesc> h_blocks;
  std::vector<int32_t> h_blk_cols;
  std::vector<double> h_lo, h_hi;       // spectral bounds of A0 per block
  std::vector<float> h_own_diag;        // diagonal of A0 at every own column (first point of set_mu)
  float* d_own_diag = nullptr;
  std::vector<int32_t> h_iters;
  int64_t sum_sq = 0, sum_slab = 0, sum_idx = 0, sum_own = 0;
  int32_t idx_stride = nolsm::kMaxDim;  // entries per block in the index-set and per-row pools
  double flops_paper_iter = 0.0, flops_exec_iter = 0.0;

  // device memory owned by the context
  nolsm::BlockDesc* d_blocks = nullptr;
  int32_t* d_idx = nullptr;
  int32_t* d_own = nullptr;
  int32_t* d_blk_cols = nullptr;
  int32_t* d_bptr = nullptr;    // blk_ptr then extra_ptr (device copies)
  int32_t* d_extra = nullptr;   // extra indices (device copy)
  int32_t* d_nb = nullptr;      // |I_b| per block
  float* d_a0 = nullptr;        // A0, fp32, square pool
  float* d_linv = nullptr;      // L^-1, fp32, square pool
  void* d_x[2] = {nullptr, nullptr};   // iterates (fp32 or fp16/bf16), square pools
  void* d_b = nullptr;          // second operand (c1 I - c3 X^2), square pool
  float* d_w = nullptr;         // L^-1[:, C_b], slab pool
  float* d_z = nullptr;         // L^-1 H_b[:, C_b], slab pool
  float* d_lc = nullptr;        // L^-1 S_b[:, C_b] = L[C_b, :]^T, slab pool
  float* d_y = nullptr;         // 1/2 (I - X) W, slab pool
  float* d_tmp = nullptr;       // slab scratch (3 slabs)
  double* d_lo = nullptr;       // spectral bounds per block
  double* d_hi = nullptr;
  double* d_bn = nullptr;       // per-block traces (per slab unit on the tensor-core refinement)
  double* d_be = nullptr;
  bool traces_per_unit = false; // the last evaluation left its traces per slab unit (tensor-core refinement)
  // own-column pieces of the tensor-core refinement: (block, first column, columns), narrow pieces
  // (<= 32 columns) first, then wide ones (<= 192), each group largest block first
  int32_t* d_slab_units = nullptr;
  // blocked double-float Cholesky with tensor-core trailing updates: slicing exponent per row,
  // kOzSlices BF16 slice planes per row of the current panel, work items (block, first column) of
  // every panel's update and where each panel's items start
  int32_t* d_oz_exp = nullptr;
  uint16_t* d_oz_planes = nullptr;
  int32_t* d_oz_items = nullptr;
  uint8_t* d_oz_tmaps = nullptr;
  // M = L11^-1 of the current panel: kOzSlices BF16 slice planes of 64 x 64 per block, each row c on its
  // own scale 2^f_c; per block 68 ints: f_0 .. f_63 and g = the largest row exponent of the panel
  uint16_t* d_oz_m = nullptr;
  int32_t* d_oz_f = nullptr;
  nolsm::TrItem* d_tr_items = nullptr;   // every panel's 128-row TRSM tiles
  std::vector<int32_t> h_oz_items;
  std::vector<int64_t> h_oz_panel;   // item offset of panel p (size panels + 1)
  std::vector<nolsm::TrItem> h_tr_items;
  std::vector<int64_t> h_tr_panel;   // TRSM item offset of panel p (size panels + 1)
  int64_t sum_pad = 0;
  std::vector<int32_t> h_slab_units;
  int32_t n_units_narrow = 0, n_units_wide = 0;
  float* d_resacc = nullptr;    // per-block residual accumulators
  float* d_tol = nullptr;       // per-block stopping tolerance on ||X^2 - I||_F
  nolsm::NsState* d_state = nullptr;
  nolsm::Tile* d_tiles = nullptr;
  int64_t max_tiles = 0;        // full tile count (capacity of d_tiles)
  // the tile lists of the build's tensor-core products (the congruence's two passes, then the tiled
  // inverse's launches) with each tile's first K, kept while the block layout stays the same
  nolsm::Tile* d_bt = nullptr;
  int32_t* d_cg_kbeg = nullptr;
  int64_t bt_cap = 0;                          // capacity of both, in tiles
  std::vector<nolsm::BlockDesc> bt_layout;     // the layout the device lists were made for
  const void* bt_dev = nullptr;                // and the buffers they were written to
  const void* bt_kdev = nullptr;
  std::vector<int64_t> bt_start;               // launch k covers [bt_start[k], bt_start[k + 1])
  int64_t max_tiles_tc = 0;     // upper-triangular tensor-core tiles of all blocks
  nolsm::DevFlags* d_flags = nullptr;
  nolsm::DevFlags* h_flags = nullptr;   // pinned mirror

  // CSR copies / references
  const int64_t* d_row_ptr = nullptr;
  const int32_t* d_col = nullptr;
  const double* d_hval = nullptr;
  const double* d_sval = nullptr;
  void* d_csr_own = nullptr;            // staging when inputs were host-resident
  int64_t* d_transpose = nullptr;       // position of (j,i) for entry (i,j)
  double* d_dval = nullptr;             // assembled D on the pattern

  // chunked solve (nolsm_solve_chunked): the builds of its chunks skip the context's own D and reuse
  // the transpose positions of the first chunk (same CSR); the density of every chunk is scattered
  // into the caller's D, which is cleared once per pass, not per chunk
  bool chunked = false;
  bool transpose_ready = false;         // d_transpose holds the positions of the current CSR
  double* d_dval_target = nullptr;      // when set, the density scatter's destination (not cleared)

  // build scratch kept across builds: FP64 S and its factor (2 sum_sq doubles), T1 (sum_sq floats)
  double* d_sb = nullptr;
  float* d_t1 = nullptr;
  // capacity in bytes of every pool the context owns (pools only grow)
  std::vector<std::pair<void**, size_t>> caps;

  // the per-product iteration captured as one graph (a while node over one iteration), rebuilt after
  // every build and whenever the captured choices change
  cudaGraph_t loop_graph = nullptr;
  cudaGraphExec_t loop_exec = nullptr;
  cudaStream_t cap_stream = nullptr;   // where the graph is captured
  int64_t build_gen = 0;
  int64_t loop_key[6] = {-1, -1, -1, -1, -1, -1};

  // tensor-core operand descriptors (device array of CUtensorMap, opaque bytes)
  void* d_tmaps = nullptr;
  size_t tmap_cap = 0;            // capacity of d_tmaps, in maps
  int n_tmaps = 0;

  // counters (nolsm_counters): every launch through a launcher, and event pairs around the
  // matrix-product launches of the sign iteration
  int64_t n_launches = 0;
  int64_t n_gemm = 0;
  double gemm_ms = 0.0;
  double gemm_flops = 0.0;
  std::vector<cudaEvent_t> gemm_ev;     // pairs, reused
  struct PhaseRec {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<PhaseRec> ph_pending;     // recorded stage intervals not yet read back
  std::vector<cudaEvent_t> ev_free;     // idle events for the stage timers
  int ph_open = -1;
  cudaEvent_t ph_open_ev = nullptr;
  double phase_ms[NOLSM_NUM_PHASES] = {};
  int gemm_ev_used = 0;

  // spectral bounds beyond Gershgorin
  const struct nolsm_mlp* predictor = nullptr;
  float* d_feat = nullptr;      // n_blocks x 32 features
  float* d_pred = nullptr;      // n_blocks x 3 predictions
  float* d_lz = nullptr;        // n_blocks x 4 Lanczos results on A0
  float* d_lz1 = nullptr;       // n_blocks x 4 Lanczos results on |A0 - mu| (kept bounds)
  float* d_given = nullptr;     // n_blocks x 3 bounds kept from an earlier geometry or set by the caller
  int32_t given_blocks = 0;     // blocks d_given describes (0: none)
  float* d_lz_basis = nullptr;  // Lanczos basis scratch
  float* d_rowd = nullptr;      // diag(A0) per row (stride kMaxDim per block)
  float* d_rowr = nullptr;      // Gershgorin radius per row (same layout)
  float* d_feat_static = nullptr;   // mu-independent features (n_blocks x 32)

  // schedule of the mixed-precision products (nolsm_set_schedule_table): per n_pad, the measured best
  // schedule; a sign evaluation whose blocks prefer different schedules runs the persistent kernel on
  // the queue d_queue[0, n_queue) and per-product launches on the remaining blocks
  std::vector<int32_t> sched_pad, sched_kind;
  std::vector<double> sched_ms;         // per entry: ms per block of PERSISTENT, PER_PRODUCT, INTERLEAVED (or empty)
  int32_t* d_queue = nullptr;
  int32_t n_queue = 0;                  // blocks of the persistent launch (n_blocks: all of them)
  int32_t last_schedule = -1;           // schedule the last sign evaluation ran (nolsm_schedule, or -2: split)

  double last_mu = 0.0;
  nolsm_sign_stats last_stats{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace nolsm {

// error helpers (api.cu)
nolsm_status fail(nolsm_ctx* ctx, nolsm_status st, const std::string& msg);
double unit_roundoff(const nolsm_ctx* ctx);   // of the iterate's storage format
// Stage timers (nolsm_phase_times): phase_mark(ctx, p) closes the open stage, if any, and opens p
// (p < 0: close only); events are read back by harvest_phases once the stream has drained.
cudaError_t phase_mark(nolsm_ctx* ctx, int phase);
void harvest_phases(nolsm_ctx* ctx);

// Smallest lower bound l the scaled iteration may assume: one scaled step maps an eigenvalue at 1 to
// about 2.6 l, which must stay clear of the format's rounding of the iterate (about u), so l >= 2 u
// (FP16 2^-10, BF16 2^-7, FP32 2^-23) whatever a bound or a prediction says.
inline float scaled_l_floor(const nolsm_ctx* ctx) { return (float)(2.0 * unit_roundoff(ctx)); }
nolsm_status cuda_fail(nolsm_ctx* ctx, cudaError_t e, const char* what);

// build.cu
cudaError_t launch_gather(nolsm_ctx* ctx, float* hb, double* sb);
cudaError_t launch_cholesky_inverse(nolsm_ctx* ctx, double* sb, int mode);
cudaError_t launch_congruence(nolsm_ctx* ctx, float* t1_scratch);
cudaError_t launch_slabs_impl(nolsm_ctx* ctx, const void* lfac, int fp32, const float* t1);
cudaError_t launch_own_diag(nolsm_ctx* ctx);   // d_own_diag from the per-row diagonal of A0

// sign.cu (SIMT path, control, slab traces)
cudaError_t launch_ns_init(nolsm_ctx* ctx, double mu, int half, int mode, const float* lz, const float* pred,
                           bool fill);
cudaError_t launch_ns_restart(nolsm_ctx* ctx, int half);          // mu from DevFlags::mu
cudaError_t launch_set_loop_mu(nolsm_ctx* ctx, double mu);
cudaError_t launch_loop_cond(nolsm_ctx* ctx, cudaGraphConditionalHandle h);
cudaError_t launch_loop_reset(nolsm_ctx* ctx);
cudaError_t launch_ns_tiles(nolsm_ctx* ctx);
cudaError_t launch_ns_tiles_n(nolsm_ctx* ctx, int tile_n);
cudaError_t launch_ns_check_impl(nolsm_ctx* ctx, const float* tol_b);
cudaError_t launch_ns_check_impl(nolsm_ctx* ctx, const float* tol_b, int detect_divergence);
cudaError_t launch_ns_advance(nolsm_ctx* ctx);
cudaError_t launch_ns_reinit(nolsm_ctx* ctx, double mu, int half);
cudaError_t launch_gemm_f32(nolsm_ctx* ctx, int phase);
cudaError_t launch_slab_traces(nolsm_ctx* ctx, int half);
cudaError_t launch_density(nolsm_ctx* ctx);
cudaError_t launch_band_energy(nolsm_ctx* ctx);

// sign_tc.cu (tcgen05 path)
cudaError_t tc_prepare(nolsm_ctx* ctx);
cudaError_t launch_gemm_tc(nolsm_ctx* ctx, int phase);
cudaError_t launch_ns_pair(nolsm_ctx* ctx, double mu, bool interleaved);
cudaError_t launch_congruence_tc(nolsm_ctx* ctx, float* t1);
cudaError_t launch_slab_tc(nolsm_ctx* ctx);
cudaError_t oz_prepare(nolsm_ctx* ctx);                        // items and tensor maps of the updates
cudaError_t launch_chol_update_tc(nolsm_ctx* ctx, int panel, double* pool);
cudaError_t launch_chol_trsm_tc(nolsm_ctx* ctx, int panel, double* pool, float* l32);
cudaError_t launch_trinv_tc(nolsm_ctx* ctx, const float* l32, float* ypool);   // mixed paths' L^-1
void trinv_diag_launch(nolsm_ctx* ctx, const float* l32, float* ypool, int max_nb);
constexpr int kOzPanel = 64;      // panel width of the blocked double-float Cholesky
int tc_tile_n();
constexpr int kSlabNarrow = 32;   // columns of a narrow refinement piece
constexpr int kSlabWide = 192;    // columns of a wide refinement piece

// learn.cu
cudaError_t launch_bounds_features(nolsm_ctx* ctx, float* feat);   // Gershgorin bounds + static features
cudaError_t launch_features_mu(nolsm_ctx* ctx, double mu, float* feat);
cudaError_t launch_lanczos(nolsm_ctx* ctx, double mu, int op, int k, float* basis, int64_t stride, float* out);
cudaError_t launch_given_from_lanczos(nolsm_ctx* ctx, const float* lz_a0, const float* lz_abs, float* given);
cudaError_t mlp_predict_on(const struct nolsm_mlp* m, cudaStream_t s, const float* x, int n, float* y);

// index.cu
cudaError_t launch_transpose(nolsm_ctx* ctx);
cudaError_t launch_index_sets(nolsm_ctx* ctx, const int32_t* d_blk_ptr, const int32_t* d_extra_ptr,
                              const int32_t* d_extra_idx, int32_t* d_nb, int cap, int max_dim);

// Exact slicing of double-float values for the tensor-core factor (Ozaki, Ogita, Oishi & Rump
// 2012): kOzSlices integer slices of kOzBits bits each, 48 bits in all (the pairs' precision).
constexpr int kOzSlices = 6;
constexpr int kOzBits = 8;
#ifdef __CUDACC__
// The slices of h + l on the scale 2^e (|h + l| <= 2^e), given sc = 2^(8 - e) (oz_scale):
// h + l = 2^(e - 8) sum_s q_s 2^(-8 s) + rest with |q_0| <= 256, |q_s| <= 128 after it and
// |rest| <= 2^(e - 49); every q_s is an integer exact in BF16 (8 significant bits).  A product of two
// slices is exact (at most 2^16), and the sum over a 64-wide panel of the products of one level
// l = s + t <= 5 is at most 64 (l + 3) 2^14 <= 2^23 (level 0: 2^22), an integer exact in FP32.  The
// remainder of each step is carried exactly by a TwoSum with the low word.
__device__ __forceinline__ float oz_scale(int e) { return ldexpf(1.f, kOzBits - e); }
__device__ __forceinline__ void oz_slices(float h, float l, float sc, float (&q)[kOzSlices]) {
  constexpr float radix = (float)(1 << kOzBits);
  float hh = h * sc, ll = l * sc;
#pragma unroll
  for (int s = 0; s < kOzSlices; ++s) {
    q[s] = rintf(hh);
    const float d = hh - q[s];
    const float sum = d + ll;
    const float bb = sum - d;
    const float err = (d - (sum - bb)) + (ll - bb);
    hh = sum * radix;
    ll = err * radix;
  }
}
#endif

// generic SIMT NT product used by the build: C_b = A_b B_b^T on the block table
cudaError_t launch_sgemm_nt(nolsm_ctx* ctx, const float* a, const float* b, float* c, int a_lower, int b_lower,
                            int sym);

}  // namespace nolsm
