// Tensor-core products of the Newton-Schulz sign iteration (Eq. 6) for the mixed-precision
// path: FP16 (or BF16) operands, FP32 accumulation in tensor memory, sm_103a tcgen05.
//
// One persistent kernel per product over a tile list of the blocks still iterating.  Each CTA
// (1 per SM, 192 threads) runs three roles:
//   warp 0      TMA producer: 128x64 A boxes and 128x64 B boxes (128B swizzle) into a 4-stage ring
//   warp 1      MMA issuer (one thread): tcgen05.mma M=128, N=tile_n (<=256), K=16, into one of
//               two TMEM accumulators (256 columns each); allocates and frees tensor memory
//   warps 2..5  epilogue: tcgen05.ld of the accumulator, the iteration's arithmetic, stores
// Phase 1 (T = X X^T, X symmetric) writes B = 1.5 a I - 0.5 a^3 T and adds ||T - I||_F^2 of the
// tile to the block's accumulator; phase 2 writes X+ = X B^T.  All operands are symmetric, so
// row-major storage is the K-major layout of both operands.
//
// Every wait on an mbarrier is bounded: past the budget the kernel records NOLSM_ETIMEOUT,
// tells the other roles to stop, lets its own copies and products land (bounded again),
// frees its tensor memory and returns.
#include "internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>

namespace nolsm {
namespace {

constexpr int TM = 128;           // tile rows (MMA M)
constexpr int TN = 256;           // tile columns (MMA N, last tile of a block may be 128)
constexpr int TK = 64;            // K per stage: one 128-byte swizzle atom of 16-bit elements
constexpr int STAGES = 4;
constexpr int A_BYTES = TM * TK * 2;          // 16 KB
constexpr int B_BYTES = TN * TK * 2;          // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 512;                // two 256-column FP32 accumulators
constexpr int NUM_THREADS = 192;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;

struct TcParams {
  const Tile* tiles;
  const int32_t* n_tiles;
  const BlockDesc* blocks;
  const NsState* st;
  const CUtensorMap* tmaps;     // per bin: [X0, X1, B]
  void* x0;
  void* x1;
  void* bbuf;
  float* resacc;
  DevFlags* flags;
  long long budget;             // polls per wait
  int phase;                    // 1 or 2
  int tile_base;                // first tile of this launch in the list
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true when the phase completed, false after the poll budget or an abort.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long budget, volatile int* abort_flag) {
  for (long long i = 0; i < budget; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tmap, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;      // leading byte offset (not used by swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;               // descriptor version
  d |= (uint64_t)2 << 61;               // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, A/B format (0 = F16, 1 = BF16), both K-major.
__device__ __forceinline__ uint32_t make_idesc(int fmt, int m, int n) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

template <typename T> struct Pack;
template <> struct Pack<__half> {
  static constexpr int fmt = 0;
  __device__ static __half one(float a) { return __float2half_rn(a); }
  __device__ static uint32_t two(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
};
template <> struct Pack<__nv_bfloat16> {
  static constexpr int fmt = 1;
  __device__ static __nv_bfloat16 one(float a) { return __float2bfloat16_rn(a); }
  __device__ static uint32_t two(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
};

__device__ __forceinline__ void set_error(DevFlags* f, int code) { atomicCAS(&f->error, 0, code); }

// Everything a role needs about one tile, resolved once per launch into shared memory (the
// chain tile -> block descriptor -> iteration state is three dependent global loads).
struct TileInfo {
  int64_t out_off;    // element offset of the output matrix in its pool
  int32_t row_a;      // TMA row of the A box (bin-stacked coordinates)
  int32_t row_b;      // TMA row of the first B box
  int32_t m0, n0;     // tile origin inside the block
  int32_t tn, kend;   // tile width (128 or 256), K extent
  int32_t ld;         // n_pad of the block
  int32_t map_a;      // tensor-map index of A
  int32_t map_b;      // tensor-map index of B
  int32_t out_sel;    // 0: x0, 1: x1, 2: bbuf
  int32_t block;
  float c1, c3;       // phase-1 epilogue coefficients
  int32_t pad;
};
constexpr int MAX_LOCAL = 352;                // tiles per CTA per launch
constexpr int INFO_BYTES = MAX_LOCAL * (int)sizeof(TileInfo);
constexpr int SMEM_TOTAL = SMEM_BYTES + INFO_BYTES;

template <typename T>
__global__ void __launch_bounds__(NUM_THREADS, 1) ns_tc_kernel(const __grid_constant__ TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stage_base = smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* full_bar = bars;                       // [STAGES]
  uint64_t* empty_bar = bars + STAGES;             // [STAGES]
  uint64_t* tfull_bar = bars + 2 * STAGES;         // [2]
  uint64_t* tempty_bar = bars + 2 * STAGES + 2;    // [2]
  uint64_t* drain_bar = bars + 2 * STAGES + 4;     // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  TileInfo* info = reinterpret_cast<TileInfo*>(smem + STAGES * STAGE_BYTES + 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Each CTA takes a contiguous run of the tile list: the list holds a block's tiles together, so
  // one SM walks through whole blocks and re-reads each iterate from L2 rather than HBM.
  const int n_tiles = *p.n_tiles;
  const int span = min(max(n_tiles - p.tile_base, 0), MAX_LOCAL * (int)gridDim.x);
  const int first = p.tile_base + (int)(((int64_t)span * blockIdx.x) / gridDim.x);
  const int n_local = p.tile_base + (int)(((int64_t)span * (blockIdx.x + 1)) / gridDim.x) - first;
  for (int i = threadIdx.x; i < n_local; i += NUM_THREADS) {
    const Tile tl = p.tiles[first + i];
    const BlockDesc bd = p.blocks[tl.block];
    const NsState s = p.st[tl.block];
    TileInfo f;
    f.m0 = tl.m0;
    f.n0 = tl.n0;
    f.kend = tl.kend;
    f.ld = bd.n_pad;
    f.tn = min(TN, bd.n_pad - tl.n0);
    f.row_a = bd.pos * bd.n_pad + tl.m0;
    f.row_b = bd.pos * bd.n_pad + tl.n0;
    f.map_a = bd.bin * 3 + s.cur;
    f.map_b = (p.phase == 1) ? f.map_a : bd.bin * 3 + 2;
    f.out_sel = (p.phase == 1) ? 2 : (s.cur ^ 1);
    f.out_off = bd.off_mat;
    f.block = tl.block;
    f.c1 = 1.5f * s.a;
    f.c3 = 0.5f * s.a * s.a * s.a;
    f.pad = 0;
    info[i] = f;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    for (int a = 0; a < 2; ++a) { mbar_init(&tfull_bar[a], 1); mbar_init(&tempty_bar[a], 128); }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const long long budget = p.budget;
  // draining our own copies / products never depends on the caller's budget
  const long long drain_budget = budget > (1LL << 22) ? budget : (1LL << 22);

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      uint32_t armed = 0;                  // bit s: stage s has been armed at least once
      uint32_t arm_parity = 0;             // bit s: phase parity of the last arm of stage s
      bool ok = true;
      for (int i = 0; i < n_local && ok; ++i) {
        const TileInfo& f = info[i];
        const CUtensorMap* ma = p.tmaps + f.map_a;
        const CUtensorMap* mb = p.tmaps + f.map_b;
        const uint32_t bytes = A_BYTES + f.tn * TK * 2;
        for (int k0 = 0; k0 < f.kend; k0 += TK) {
          if (!mbar_wait(&empty_bar[s], ph ^ 1u, budget, abort_flag)) { ok = false; break; }
          mbar_expect_tx(&full_bar[s], bytes);
          uint8_t* a_dst = stage_base + s * STAGE_BYTES;
          uint8_t* b_dst = a_dst + A_BYTES;
          tma_load_2d(a_dst, ma, &full_bar[s], k0, f.row_a);
          for (int h = 0; h < f.tn; h += TM) tma_load_2d(b_dst + h * TK * 2, mb, &full_bar[s], k0, f.row_b + h);
          armed |= 1u << s;
          arm_parity = (arm_parity & ~(1u << s)) | (ph << s);
          if (++s == STAGES) { s = 0; ph ^= 1u; }
        }
      }
      if (!ok) {
        set_error(p.flags, NOLSM_ETIMEOUT);
        *abort_flag = 1;
      }
      // every copy this thread issued must land before the CTA's shared memory is released
      volatile int never = 0;
      for (int st = 0; st < STAGES; ++st)
        if (armed & (1u << st)) mbar_wait(&full_bar[st], (arm_parity >> st) & 1u, drain_budget, &never);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      uint32_t tph[2] = {0u, 0u};
      int acc = 0;
      bool ok = true;
      for (int i = 0; i < n_local && ok; ++i) {
        const TileInfo& f = info[i];
        const uint32_t idesc = make_idesc(Pack<T>::fmt, TM, f.tn);
        if (!mbar_wait(&tempty_bar[acc], tph[acc] ^ 1u, budget, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * TN);
        for (int k0 = 0; k0 < f.kend; k0 += TK) {
          if (!mbar_wait(&full_bar[s], ph, budget, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a_addr = smem_u32(stage_base + s * STAGE_BYTES);
          const uint32_t b_addr = a_addr + A_BYTES;
          const uint64_t adesc = sw128_desc(a_addr);
          const uint64_t bdesc = sw128_desc(b_addr);
#pragma unroll
          for (int kk = 0; kk < TK / 16; ++kk) {
            // advance 16 elements (32 bytes) along K inside the swizzle atom
            umma_f16(d_tmem, adesc + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), idesc, (k0 | kk) != 0);
          }
          umma_commit(&empty_bar[s]);        // stage free once these MMAs have read it
          if (++s == STAGES) { s = 0; ph ^= 1u; }
        }
        if (!ok) break;
        umma_commit(&tfull_bar[acc]);        // accumulator ready for the epilogue
        tph[acc] ^= 1u;
        acc ^= 1;
      }
      if (!ok) {
        set_error(p.flags, NOLSM_ETIMEOUT);
        *abort_flag = 1;
      }
      // let every product issued by this thread land before tensor memory is released
      umma_commit(drain_bar);
      volatile int never = 0;
      mbar_wait(drain_bar, 0, drain_budget, &never);
    }
  } else {
    // ------------------------------------------------------------------ epilogue (warps 2..5)
    const int q = warp & 3;                  // TMEM lane quarter this warp may access
    const int row_in_tile = q * 32 + lane;
    uint32_t tph[2] = {0u, 0u};
    int acc = 0;
    T* const pools[3] = {reinterpret_cast<T*>(p.x0), reinterpret_cast<T*>(p.x1), reinterpret_cast<T*>(p.bbuf)};
    for (int i = 0; i < n_local; ++i) {
      const TileInfo& f = info[i];
      const int ld = f.ld;
      const int tn = f.tn;
      if (!mbar_wait(&tfull_bar[acc], tph[acc], budget, abort_flag)) {
        set_error(p.flags, NOLSM_ETIMEOUT);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      T* out = pools[f.out_sel] + f.out_off;
      const float c1 = f.c1, c3 = f.c3;
      const int r = f.m0 + row_in_tile;
      T* orow = out + (int64_t)r * ld + f.n0;
      float rsq = 0.f;
      // Tiles lie on or above the block diagonal.  Entry (r, c): c > r is stored at (r, c) and at
      // (c, r), the diagonal once, c < r (left part of a diagonal tile) not at all, so every
      // iterate is exactly symmetric -- the products read the transpose of their B operand, and
      // with a non-symmetric iterate the iteration would be X (3 - X X^T) / 2, which doubles
      // antisymmetric rounding errors each step once converged.
      for (int c0 = 0; c0 < tn; c0 += 32) {
        const int cg0 = f.n0 + c0;
        uint32_t v[32];
        tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * TN + c0), v);
        if (cg0 + 31 < r) continue;              // whole chunk left of the diagonal (warp-uniform ld done)
        float fv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          float x = __uint_as_float(v[j]);
          if (p.phase == 1) {
            const int cg = cg0 + j;
            const float d = (cg == r) ? 1.f : 0.f;
            const float e = x - d;
            const float w = (cg > r) ? 2.f : ((cg == r) ? 1.f : 0.f);
            rsq = fmaf(w, e * e, rsq);
            x = c1 * d - c3 * x;
          }
          fv[j] = x;
        }
        if (cg0 >= r) {
          uint32_t packed[16];
#pragma unroll
          for (int j = 0; j < 32; j += 2) packed[j >> 1] = Pack<T>::two(fv[j], fv[j + 1]);
          uint4* dst = reinterpret_cast<uint4*>(orow + c0);
#pragma unroll
          for (int u = 0; u < 4; ++u)
            dst[u] = make_uint4(packed[4 * u], packed[4 * u + 1], packed[4 * u + 2], packed[4 * u + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (cg0 + j >= r) orow[c0 + j] = Pack<T>::one(fv[j]);
        }
        // mirror: column cg of this tile becomes row cg; lanes hold consecutive rows r
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (cg0 + j > r) out[(int64_t)(cg0 + j) * ld + r] = Pack<T>::one(fv[j]);
      }
      tc_fence_before();
      mbar_arrive(&tempty_bar[acc]);
      tph[acc] ^= 1u;
      acc ^= 1;
      if (p.phase == 1) {
        for (int o = 16; o; o >>= 1) rsq += __shfl_xor_sync(0xffffffffu, rsq, o);
        if (lane == 0) atomicAdd(&p.resacc[f.block], rsq);
      }
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

}  // namespace

// Encode one 2-D tensor map per (bin, pool) over the bin's stacked n_pad x n_pad matrices.
cudaError_t tc_prepare(nolsm_ctx* ctx) {
  auto encode = get_encode();
  if (!encode) return cudaErrorNotSupported;
  const bool bf16 = ctx->opt.precision == NOLSM_PREC_MIXED_BF16;
  // bins: consecutive runs of equal n_pad in the layout order (blocks are laid out bin by bin)
  std::vector<CUtensorMap> maps;
  int n_bins = 0;
  for (const auto& b : ctx->h_blocks) n_bins = std::max(n_bins, b.bin + 1);
  std::vector<int64_t> bin_off(n_bins, -1), bin_cnt(n_bins, 0);
  std::vector<int> bin_pad(n_bins, 0);
  for (const auto& b : ctx->h_blocks) {
    if (b.pos == 0) bin_off[b.bin] = b.off_mat;
    bin_cnt[b.bin] += 1;
    bin_pad[b.bin] = b.n_pad;
  }
  maps.resize((size_t)n_bins * 3);
  void* pools[3] = {ctx->d_x[0], ctx->d_x[1], ctx->d_b};
  for (int bi = 0; bi < n_bins; ++bi) {
    for (int pi = 0; pi < 3; ++pi) {
      const uint64_t np = (uint64_t)bin_pad[bi];
      void* base = reinterpret_cast<uint8_t*>(pools[pi]) + bin_off[bi] * 2;
      cuuint64_t gdim[2] = {np, np * (uint64_t)bin_cnt[bi]};
      cuuint64_t gstride[1] = {np * 2};
      cuuint32_t box[2] = {TK, TM};
      cuuint32_t estr[2] = {1, 1};
      CUresult r = encode(&maps[(size_t)bi * 3 + pi], bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                          2, base, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
  }
  if (ctx->d_tmaps) cudaFree(ctx->d_tmaps);
  cudaError_t e = cudaMalloc(&ctx->d_tmaps, maps.size() * sizeof(CUtensorMap));
  if (e != cudaSuccess) return e;
  ctx->n_tmaps = (int)maps.size();
  e = cudaMemcpyAsync(ctx->d_tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return e;
  static bool attr_done = false;
  if (!attr_done) {
    e = cudaFuncSetAttribute(ns_tc_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TOTAL);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ns_tc_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TOTAL);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  return cudaSuccess;
}

cudaError_t launch_ns_tiles_n(nolsm_ctx* ctx, int tile_n);

cudaError_t launch_gemm_tc(nolsm_ctx* ctx, int phase) {
  TcParams p;
  p.tiles = ctx->d_tiles;
  p.n_tiles = &ctx->d_flags->n_tiles;
  p.blocks = ctx->d_blocks;
  p.st = ctx->d_state;
  p.tmaps = reinterpret_cast<const CUtensorMap*>(ctx->d_tmaps);
  p.x0 = ctx->d_x[0];
  p.x1 = ctx->d_x[1];
  p.bbuf = ctx->d_b;
  p.resacc = ctx->d_resacc;
  p.flags = ctx->d_flags;
  p.budget = ctx->opt.wait_budget;
  p.phase = phase;
  const int grid = ctx->num_sms;
  // each CTA resolves at most MAX_LOCAL tiles per launch; cover the largest possible list
  const int64_t per_launch = (int64_t)MAX_LOCAL * grid;
  for (int64_t base = 0; base < std::max<int64_t>(ctx->max_tiles_tc, 1); base += per_launch) {
    p.tile_base = (int)base;
    if (ctx->opt.precision == NOLSM_PREC_MIXED_BF16)
      ns_tc_kernel<__nv_bfloat16><<<grid, NUM_THREADS, SMEM_TOTAL, ctx->stream>>>(p);
    else
      ns_tc_kernel<__half><<<grid, NUM_THREADS, SMEM_TOTAL, ctx->stream>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int tc_tile_n() { return TN; }

}  // namespace nolsm
