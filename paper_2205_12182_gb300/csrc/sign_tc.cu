// Tensor-core products of the Newton-Schulz sign iteration (Eq. 6) for the mixed-precision
// path: FP16 (or BF16) operands, FP32 accumulation in tensor memory, sm_103a tcgen05.
//
// One persistent kernel per product over a tile list of the blocks still iterating.  Each CTA
// (1 per SM) runs three roles:
//   warp 0      TMA producer: 128x64 A boxes and 128x64 B boxes (128B swizzle) into a ring of
//               4 stages (blocks below n_pad 1024) or 3 (larger blocks)
//   warp 1      MMA issuer (one thread): tcgen05.mma M=128, N=tile_n (<=256), K=16, into one of
//               two TMEM accumulators (256 columns each); allocates and frees tensor memory
//   warps 2..   epilogue: tcgen05.ld of the accumulator, the iteration's arithmetic, stores; one
//               warp per TMEM lane quarter (small blocks) or two, each taking half of a tile's
//               columns with double-buffered staging (larger blocks: long tiles back to back)
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
#include <cuda_fp8.h>

#include <cfloat>
#include <cstring>

namespace nolsm {
namespace {

constexpr int TM = 128;           // tile rows (MMA M)
constexpr int TN = 256;           // tile columns (MMA N, last tile of a block may be 128)
constexpr int TK = 64;            // K per stage: one 128-byte swizzle atom of 16-bit elements
constexpr int A_BYTES = TM * TK * 2;          // 16 KB
constexpr int B_BYTES = TN * TK * 2;          // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TMEM_COLS = 512;                // two 256-column FP32 accumulators
constexpr int NUM_THREADS = 192;              // the refinement kernel's roles (producer, issuer, 4 epilogue warps)
// per bin: loads of X0, X1, B (64 x 128 boxes), stores into them (32 x 32 boxes), and loads of the
// refinement's four split slab pools hi0, lo0, hi1, lo1 (64 x 16 boxes)
constexpr int kMapsPerBin = 10;
constexpr int EPI_BUF_BYTES = 4096;           // one staging buffer: a 32 x 32 chunk and its transpose
// shared memory of the product kernels: [stages | epilogue staging, NBUF buffers per epilogue warp |
// barriers | tables], 1024-byte aligned base (TcShape below, and the persistent kernels' PAIR_*)

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
  int interleave;               // 1: tile i of the launch goes to CTA i mod grid; 0: contiguous runs
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

// Tensor store of a 32 x 32 box from shared memory (bulk-group completion).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* tmap, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(tmap)),
               "r"(x), "r"(y), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, "
      "%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, "
      "%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]),
        "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]),
        "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
        "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
        "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
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
  __device__ static float f(__half a) { return __half2float(a); }
  __device__ static uint32_t two(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
};
template <> struct Pack<__nv_bfloat16> {
  static constexpr int fmt = 1;
  __device__ static __nv_bfloat16 one(float a) { return __float2bfloat16_rn(a); }
  __device__ static float f(__nv_bfloat16 a) { return __bfloat162float(a); }
  __device__ static uint32_t two(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
};

__device__ __forceinline__ void set_error(DevFlags* f, int code) { atomicCAS(&f->error, 0, code); }

// Byte offset of element (row, col) of a 32 x 32 16-bit box in the 64-byte-swizzle layout the store
// tensor maps use: the 16-byte unit of a 64-byte row is XORed with bits 1-2 of the row.  Rows written
// by consecutive lanes (and columns of one row) then fall in distinct shared-memory banks.
__device__ __forceinline__ uint32_t sw64(int row, int col) {
  return (uint32_t)(row * 64 + ((((col * 2) >> 4) ^ ((row >> 1) & 3)) << 4) + ((col * 2) & 15));
}

// byte offset of (row, byte column) in a 128-byte-row box with the 128-byte swizzle (16-byte unit XOR row % 8)
__device__ __forceinline__ uint32_t sw128(int row, int colbytes) {
  return (uint32_t)(row * 128 + ((((colbytes >> 4) ^ (row & 7))) << 4) + (colbytes & 15));
}

// Epilogue of one tile (one warp = 32 rows of the 128-row tile, lane = row): the accumulator
// columns in chunks of 32, phase 1's arithmetic (B = c1 I - c3 T and ||T - I||^2 of the stored
// triangle), FP16/BF16 stores.  Tiles lie on or above the block diagonal and the row slices of the
// warps are 32-aligned with the chunks, so a chunk is below the diagonal (skipped), on it, or above
// it.  The stored matrix is exactly symmetric -- the products read the transpose of their B operand,
// and with a non-symmetric iterate the iteration would be X (3 - X X^T) / 2, which doubles
// antisymmetric rounding errors each step once converged:
//   above: the chunk goes to (rows, cols) and its transpose to (cols, rows), both staged in the
//          warp's shared buffer and written by two tensor stores (lane 0, asynchronous);
//   on:    entries c >= r at (r, c) and c > r also at (c, r): the symmetric box is assembled in the
//          staging buffer from the chunk and its transpose and written by one tensor store.
// Returns the lane's ||.||^2 part.  The caller waits for the tensor stores (bulk group) before the
// results are read or the buffer goes away.
// Q8 (the FP8 experiment) rounds every output to an FP8 E4M3 value first.
template <typename T, int NBUF, int LDW, bool Q8 = false>
__device__ __forceinline__ float epi_tile(uint32_t tmem_acc, int q, int lane, T* out, int ld, int m0, int n0, int tn,
                                          int phase, float c1, float c3, const CUtensorMap* smap, int rowbase,
                                          uint8_t* stage, int& buf) {
  const int r0 = m0 + q * 32;
  const int r = r0 + lane;
  float rsq = 0.f;
  // LDW accumulator columns per tensor-memory load (32 or 64; tn is a multiple of 64)
  for (int cl = 0; cl < tn; cl += LDW) {
    uint32_t v[LDW];
    if constexpr (LDW == 64) tmem_ld64(tmem_acc + ((uint32_t)(q * 32) << 16) + (uint32_t)cl, v);
    else tmem_ld32(tmem_acc + ((uint32_t)(q * 32) << 16) + (uint32_t)cl, v);
#pragma unroll
    for (int h = 0; h < LDW / 32; ++h) {
      const int cg0 = n0 + cl + 32 * h;
      if (cg0 < r0) continue;                // whole chunk below the diagonal (warp-uniform)
      const bool diag = cg0 == r0;           // warp-uniform
      float fv[32];
      if (phase == 1 && !diag) {
        // strictly above the diagonal: weight 2, no identity term (the same operations as below
        // with d = 0 and w = 2)
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float x = __uint_as_float(v[32 * h + j]);
          rsq = fmaf(2.f, x * x, rsq);
          fv[j] = 0.f - c3 * x;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          float x = __uint_as_float(v[32 * h + j]);
          if (phase == 1) {
            const int cg = cg0 + j;
            const float d = (cg == r) ? 1.f : 0.f;
            const float e = x - d;
            const float w = (cg > r) ? 2.f : ((cg == r) ? 1.f : 0.f);
            rsq = fmaf(w, e * e, rsq);
            x = c1 * d - c3 * x;
          }
          fv[j] = x;
        }
      }
      if constexpr (Q8) {
#pragma unroll
        for (int j = 0; j < 32; ++j) fv[j] = float(__nv_fp8_e4m3(fv[j]));   // stored in the iterate's format
      }
      // the store that last used this buffer (NBUF chunks ago) has read it
      if (lane == 0) {
        if (NBUF == 1) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        else asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
      }
      __syncwarp();
      uint8_t* D = stage + buf * EPI_BUF_BYTES;   // the chunk, row = lane
      uint8_t* M = D + 2048;                        // its transpose, row = j
#pragma unroll
      for (int u = 0; u < 4; ++u)
        *reinterpret_cast<uint4*>(D + sw64(lane, 8 * u)) =
            make_uint4(Pack<T>::two(fv[8 * u], fv[8 * u + 1]), Pack<T>::two(fv[8 * u + 2], fv[8 * u + 3]),
                       Pack<T>::two(fv[8 * u + 4], fv[8 * u + 5]), Pack<T>::two(fv[8 * u + 6], fv[8 * u + 7]));
      if (diag) {
        // on the diagonal the chunk is its own mirror: once every row is in place, lane c writes its
        // upper-triangle entries (c, j), j > c, over the entries (j, c) below the diagonal, and one
        // store writes the symmetric 32 x 32 box
        __syncwarp();
#pragma unroll
        for (int j = 1; j < 32; ++j)
          if (j > lane) *reinterpret_cast<T*>(D + sw64(j, lane)) = Pack<T>::one(fv[j]);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) *reinterpret_cast<T*>(M + sw64(j, lane)) = Pack<T>::one(fv[j]);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        tma_store_2d(smap, D, cg0, rowbase + r0);
        if (!diag) tma_store_2d(smap, M, r0, rowbase + cg0);
        bulk_commit();
      }
      buf = (NBUF == 1) ? 0 : buf ^ 1;
    }
  }
  return rsq;
}

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
  int32_t map_s;      // tensor-map index of the output stores
};
constexpr int MAX_LOCAL = 200;                // tiles per CTA per launch
constexpr int INFO_BYTES = MAX_LOCAL * (int)sizeof(TileInfo);

// Shapes of the per-product kernel: NST operand stages of 48 KB, EPIW epilogue warps (4: one per
// tensor-memory lane quarter; 8: two per quarter, each taking half of a tile's columns) with NBUF
// staging buffers each.  Shared memory: [stages | epilogue staging | barriers | tile table].
template <int NST, int EPIW, int NBUF>
struct TcShape {
  static constexpr int epi_off = NST * STAGE_BYTES;
  static constexpr int bar_off = epi_off + EPIW * NBUF * EPI_BUF_BYTES;
  static constexpr int tab_off = bar_off + 256;
  static constexpr int smem = 1024 + tab_off + INFO_BYTES;
  static constexpr int threads = 64 + 32 * EPIW;
  static_assert(smem <= 227 * 1024, "shared memory of the per-product kernel");
  static_assert(8 * (2 * NST + 5) + 8 <= 256, "barrier area of the per-product kernel");
  static_assert(EPIW == 4 || EPIW == 8, "one or two epilogue warps per lane quarter");
};
using TcNarrow = TcShape<4, 4, 1>;   // four 48 KB stages in flight, one epilogue warp per quarter
using TcWide = TcShape<3, 8, 2>;     // three stages, two double-buffered epilogue warps per quarter

template <typename T, int NST, int EPIW, int NBUF>
__global__ void __launch_bounds__(TcShape<NST, EPIW, NBUF>::threads, 1)
    ns_tc_kernel(const __grid_constant__ TcParams p) {
  using L = TcShape<NST, EPIW, NBUF>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stage_base = smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::bar_off);
  uint64_t* full_bar = bars;                    // [NST]
  uint64_t* empty_bar = bars + NST;             // [NST]
  uint64_t* tfull_bar = bars + 2 * NST;         // [2]
  uint64_t* tempty_bar = bars + 2 * NST + 2;    // [2]
  uint64_t* drain_bar = bars + 2 * NST + 4;     // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NST + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  TileInfo* info = reinterpret_cast<TileInfo*>(smem + L::tab_off);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // The list holds a block's tiles together.  Small blocks: each CTA takes a contiguous run, so one
  // SM walks through whole blocks and re-reads each iterate from L2 (152 blocks of a few MB in
  // flight).  Large blocks (tens of MB per block): tile i goes to CTA i mod grid, so all SMs work on
  // the same few blocks at a time and share their operand panels in L2.
  const int n_tiles = *p.n_tiles;
  const int span = min(max(n_tiles - p.tile_base, 0), MAX_LOCAL * (int)gridDim.x);
  const int first = p.interleave ? p.tile_base + (int)blockIdx.x
                                 : p.tile_base + (int)(((int64_t)span * blockIdx.x) / gridDim.x);
  const int step = p.interleave ? (int)gridDim.x : 1;
  const int n_local = p.interleave
                          ? (span > (int)blockIdx.x ? (span - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0)
                          : p.tile_base + (int)(((int64_t)span * (blockIdx.x + 1)) / gridDim.x) - first;
  for (int i = threadIdx.x; i < n_local; i += L::threads) {
    const Tile tl = p.tiles[first + i * step];
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
    f.map_a = bd.bin * kMapsPerBin + s.cur;
    f.map_b = (p.phase == 1) ? f.map_a : bd.bin * kMapsPerBin + 2;
    f.out_sel = (p.phase == 1) ? 2 : (s.cur ^ 1);
    f.out_off = bd.off_mat;
    f.block = tl.block;
    f.c1 = 1.5f * s.a;
    f.c3 = 0.5f * s.a * s.a * s.a;
    f.map_s = bd.bin * kMapsPerBin + 3 + f.out_sel;
    info[i] = f;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    for (int a = 0; a < 2; ++a) { mbar_init(&tfull_bar[a], 1); mbar_init(&tempty_bar[a], 32 * EPIW); }
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
          if (++s == NST) { s = 0; ph ^= 1u; }
        }
      }
      if (!ok) {
        set_error(p.flags, NOLSM_ETIMEOUT);
        *abort_flag = 1;
      }
      // every copy this thread issued must land before the CTA's shared memory is released
      volatile int never = 0;
      for (int st = 0; st < NST; ++st)
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
          if (++s == NST) { s = 0; ph ^= 1u; }
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
    uint32_t tph[2] = {0u, 0u};
    int acc = 0;
    int ebuf = 0;
    T* const pools[3] = {reinterpret_cast<T*>(p.x0), reinterpret_cast<T*>(p.x1), reinterpret_cast<T*>(p.bbuf)};
    for (int i = 0; i < n_local; ++i) {
      const TileInfo& f = info[i];
      const int ld = f.ld;
      const int tn = f.tn;
      // the outcome must be the same in all lanes: the tensor-memory loads below are warp-collective
      if (!__all_sync(0xffffffffu, mbar_wait(&tfull_bar[acc], tph[acc], budget, abort_flag))) {
        set_error(p.flags, NOLSM_ETIMEOUT);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      T* out = pools[f.out_sel] + f.out_off;
      // EPIW == 8: warps 2..5 take the left half of the tile's columns, warps 6..9 the right half
      const int hw = EPIW == 8 ? tn / 2 : tn, h0 = EPIW == 8 ? ((warp - 2) / 4) * hw : 0;
      float rsq = epi_tile<T, NBUF, 64>(tmem_base + (uint32_t)(acc * TN + h0), q, lane, out, ld, f.m0, f.n0 + h0, hw,
                                        p.phase, f.c1, f.c3, p.tmaps + f.map_s, f.row_a - f.m0,
                                        smem + L::epi_off + (warp - 2) * NBUF * EPI_BUF_BYTES, ebuf);
      tc_fence_before();
      mbar_arrive(&tempty_bar[acc]);
      tph[acc] ^= 1u;
      acc ^= 1;
      if (p.phase == 1) {
        for (int o = 16; o; o >>= 1) rsq += __shfl_xor_sync(0xffffffffu, rsq, o);
        if (lane == 0) atomicAdd(&p.resacc[f.block], rsq);
      }
    }
    if (lane == 0) bulk_wait0();             // tensor stores complete before the kernel ends
    __syncwarp();
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


// ---------------------------------------------------------------------------------------------
// Persistent schedule: one launch per sign evaluation.  The grid is made of 2-CTA clusters; a
// cluster takes one block at a time off a queue and runs that block's whole iteration -- X_0 from
// A0, then T = X X^T and X+ = X B^T until the block converges -- with the tiles of every product
// split between its two CTAs (same roles, ring buffers and epilogue as ns_tc_kernel).  A block's
// three n_pad^2 buffers stay in L2 for its whole iteration (76 blocks in flight x 1.5 MB at n_pad
// 512), so the products read L2 instead of streaming HBM, and no launch or host round trip sits
// between products.  The two CTAs pass through the same sequence of cluster barriers: the claimed
// block, the residual partials of the first product and any abort are published in shared memory
// and read by both after a barrier, so both take the same decisions (the rules of the check,
// advance and restart kernels of the per-product schedule).
constexpr int PAIR_MAX_TILES = 160;           // tiles of one product per CTA (n_pad 4096: 136)

struct PairParams {
  const BlockDesc* blocks;
  NsState* st;
  const CUtensorMap* tmaps;     // per bin: [X0, X1, B]
  const float* a0;
  const double* lo;
  const double* hi;
  const float* tol;
  void* x0;
  void* x1;
  void* bbuf;
  DevFlags* flags;
  long long budget;
  double mu;
  float margin;
  float l0;
  int scaled;
  int max_iter;
  int detect_divergence;
  int n_blocks;
  int fp8_iters;                // experiment: iterations whose outputs are rounded to FP8 E4M3 values
  const int32_t* queue_map;     // blocks this launch takes, in queue order (NULL: every block, 0..n_blocks)
  int n_queue;                  // entries of the queue
};

// The q-th block of a persistent launch's queue, or n_blocks once the queue is exhausted.
__device__ __forceinline__ int queue_block(const PairParams& p, int q) {
  if (q >= p.n_queue) return p.n_blocks;
  return p.queue_map ? p.queue_map[q] : q;
}

struct PairTile {
  int16_t m0, n0, tn, pad;
};

struct PairCtl {
  int block;                    // claimed block (rank 0 writes it into both CTAs)
  int n_local;                  // tiles of each product held by this CTA
  float rsq[2];                 // this CTA's ||T - I||_F^2 partial, by round parity
  int abort_pub[2];             // this CTA's abort flag as published for the round, by parity
  PairTile tiles[PAIR_MAX_TILES];
};
constexpr int PAIR_THREADS = 320;             // producer, MMA issuer, 8 epilogue warps (2 per TMEM lane quarter)
constexpr int PAIR_EPI_WARPS = 8;
constexpr int PAIR_NBUF = 2;                  // staging buffers per epilogue warp (a chunk's store overlaps the next)
constexpr int PAIR_STAGES = 3;                // operand stages (48 KB each)
constexpr int PAIR_EPI_OFF = PAIR_STAGES * STAGE_BYTES;
constexpr int PAIR_BAR_OFF = PAIR_EPI_OFF + PAIR_EPI_WARPS * PAIR_NBUF * EPI_BUF_BYTES;
constexpr int PAIR_TAB_OFF = PAIR_BAR_OFF + 256;
constexpr int PAIR_SMEM = 1024 + PAIR_TAB_OFF + (int)sizeof(PairCtl);
static_assert(PAIR_SMEM <= 227 * 1024, "shared memory of the persistent kernel");
static_assert(2 * PAIR_STAGES + 7 <= 32, "barrier area of the persistent kernel");

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// generic address of the same shared-memory object in CTA `rank` of the cluster
template <typename P>
__device__ __forceinline__ P* cluster_peer(P* local, uint32_t rank) {
  uint64_t out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(reinterpret_cast<uint64_t>(local)), "r"(rank));
  return reinterpret_cast<P*>(out);
}

// X_0 = (A0 - mu I) / alpha on the n x n part, identity on the padding; CTA `rank` writes rows
// [rank n_pad / 2, (rank + 1) n_pad / 2).  Several 16-byte loads per thread are in flight at a time
// (A0 comes from HBM: its latency, not its bandwidth, bounds a dependent load-convert-store loop),
// read as streaming data so they do not evict the resident iterates from L2.  The stores are made
// visible to the tensor-copy proxy.
template <typename T, int THREADS>
__device__ __forceinline__ void pair_fill(const BlockDesc& bd, const float* __restrict__ a0, float alpha, double mu,
                                          T* __restrict__ x, uint32_t rank) {
  constexpr int U = THREADS >= 256 ? 4 : 8;
  const int n = bd.n, ld = bd.n_pad, half = ld / 2, q4 = ld / 4;
  const int total = half * q4;
  const float inv = 1.f / alpha, muf = (float)mu;
  const float* A = a0 + bd.off_mat + (int64_t)rank * half * ld;
  T* X = x + bd.off_mat + (int64_t)rank * half * ld;
  for (int e0 = threadIdx.x; e0 < total; e0 += THREADS * U) {
    float4 a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * THREADS;
      if (e < total) a[u] = __ldcs(reinterpret_cast<const float4*>(A) + e);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * THREADS;
      if (e >= total) break;
      const int r = (int)rank * half + e / q4, c = (e % q4) * 4;
      const float av[4] = {a[u].x, a[u].y, a[u].z, a[u].w};
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cc = c + j;
        v[j] = (r < n && cc < n) ? (av[j] - (r == cc ? muf : 0.f)) * inv : (r == cc ? 1.f : 0.f);
      }
      reinterpret_cast<uint2*>(X)[e] = make_uint2(Pack<T>::two(v[0], v[1]), Pack<T>::two(v[2], v[3]));
    }
  }
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Upper-triangular 128 x (<= 256) tiles of an n_pad x n_pad product, dealt to the two CTAs so that
// their column counts stay balanced (both CTAs compute the same assignment).  Each CTA runs its
// narrow (128-column) tiles last: the epilogue of the last tile is the tail of the product.
__device__ inline int pair_tiles(int ld, uint32_t rank, PairTile* out) {
  int load[2] = {0, 0}, k = 0;
  for (int pass = 0; pass < 2; ++pass) {
    load[0] = load[1] = 0;
    for (int m0 = 0; m0 < ld; m0 += TM)
      for (int n0 = m0; n0 < ld; n0 += TN) {
        const int tn = min(TN, ld - n0);
        const int owner = load[1] < load[0] ? 1 : 0;
        load[owner] += tn;
        if (owner == (int)rank && (tn == TN) == (pass == 0)) {
          if (k >= PAIR_MAX_TILES) return -1;
          out[k++] = PairTile{(int16_t)m0, (int16_t)n0, (int16_t)tn, 0};
        }
      }
  }
  return k;
}

// Q8: the FP8 experiment's instantiation (outputs of the first p.fp8_iters iterations rounded to
// FP8 E4M3 values); the default instantiation carries none of it.
template <typename T, bool Q8>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PAIR_THREADS, 1) ns_pair_kernel(const __grid_constant__ PairParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stage_base = smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + PAIR_BAR_OFF);
  uint64_t* full_bar = bars;                       // [PAIR_STAGES]
  uint64_t* empty_bar = bars + PAIR_STAGES;             // [PAIR_STAGES]
  uint64_t* tfull_bar = bars + 2 * PAIR_STAGES;         // [2]
  uint64_t* tempty_bar = bars + 2 * PAIR_STAGES + 2;    // [2]
  uint64_t* drain_bar = bars + 2 * PAIR_STAGES + 4;     // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * PAIR_STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  PairCtl* ctl = reinterpret_cast<PairCtl*>(smem + PAIR_TAB_OFF);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  PairCtl* ctl0 = cluster_peer(ctl, 0u);
  PairCtl* ctl1 = cluster_peer(ctl, 1u);
  if (threadIdx.x == 0) {
    for (int s = 0; s < PAIR_STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    for (int a = 0; a < 2; ++a) { mbar_init(&tfull_bar[a], 1); mbar_init(&tempty_bar[a], 32 * PAIR_EPI_WARPS); }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    ctl->rsq[0] = ctl->rsq[1] = 0.f;
    ctl->abort_pub[0] = ctl->abort_pub[1] = 0;
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
  cluster_sync_all();   // both CTAs initialised before either touches the other's shared memory
  const uint32_t tmem_base = *tmem_slot;
  const long long budget = p.budget;
  const long long drain_budget = budget > (1LL << 22) ? budget : (1LL << 22);
  const int q = warp & 3;

  // ring state of each role, carried across products and blocks
  int ps = 0;
  uint32_t pph = 0, armed = 0, arm_parity = 0;
  int ms = 0;
  uint32_t mph = 0, mtph[2] = {0u, 0u};
  int macc = 0;
  uint32_t etph[2] = {0u, 0u};
  int eacc = 0;
  int ebuf = 0;
  int round = 0;

  // one product of the current block: phase 1 T = X X^T -> B, phase 2 X+ = X B^T
  auto product = [&](const BlockDesc& bd, const NsState& s, int phase, int par) {
    const int ld = bd.n_pad;
    const int n_local = ctl->n_local;
    if (warp == 0) {
      if (lane == 0) {
        const CUtensorMap* ma = p.tmaps + bd.bin * kMapsPerBin + s.cur;
        const CUtensorMap* mb = (phase == 1) ? ma : p.tmaps + bd.bin * kMapsPerBin + 2;
        const int rowbase = bd.pos * ld;
        bool ok = true;
        for (int i = 0; i < n_local && ok; ++i) {
          const PairTile t = ctl->tiles[i];
          const uint32_t bytes = A_BYTES + t.tn * TK * 2;
          for (int k0 = 0; k0 < ld; k0 += TK) {
            if (!mbar_wait(&empty_bar[ps], pph ^ 1u, budget, abort_flag)) { ok = false; break; }
            mbar_expect_tx(&full_bar[ps], bytes);
            uint8_t* a_dst = stage_base + ps * STAGE_BYTES;
            uint8_t* b_dst = a_dst + A_BYTES;
            tma_load_2d(a_dst, ma, &full_bar[ps], k0, rowbase + t.m0);
            for (int h = 0; h < t.tn; h += TM) tma_load_2d(b_dst + h * TK * 2, mb, &full_bar[ps], k0, rowbase + t.n0 + h);
            armed |= 1u << ps;
            arm_parity = (arm_parity & ~(1u << ps)) | (pph << ps);
            if (++ps == PAIR_STAGES) { ps = 0; pph ^= 1u; }
          }
        }
        if (!ok) {
          set_error(p.flags, NOLSM_ETIMEOUT);
          *abort_flag = 1;
        }
      }
    } else if (warp == 1) {
      if (lane == 0) {
        bool ok = true;
        for (int i = 0; i < n_local && ok; ++i) {
          const PairTile t = ctl->tiles[i];
          const uint32_t idesc = make_idesc(Pack<T>::fmt, TM, t.tn);
          if (!mbar_wait(&tempty_bar[macc], mtph[macc] ^ 1u, budget, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(macc * TN);
          for (int k0 = 0; k0 < ld; k0 += TK) {
            if (!mbar_wait(&full_bar[ms], mph, budget, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t a_addr = smem_u32(stage_base + ms * STAGE_BYTES);
            const uint64_t adesc = sw128_desc(a_addr);
            const uint64_t bdesc = sw128_desc(a_addr + A_BYTES);
#pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk)
              umma_f16(d_tmem, adesc + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), idesc, (k0 | kk) != 0);
            umma_commit(&empty_bar[ms]);
            if (++ms == PAIR_STAGES) { ms = 0; mph ^= 1u; }
          }
          if (!ok) break;
          umma_commit(&tfull_bar[macc]);
          mtph[macc] ^= 1u;
          macc ^= 1;
        }
        if (!ok) {
          set_error(p.flags, NOLSM_ETIMEOUT);
          *abort_flag = 1;
        }
      }
    } else {
      T* out = reinterpret_cast<T*>(phase == 1 ? p.bbuf : (s.cur ? p.x0 : p.x1)) + bd.off_mat;
      const CUtensorMap* smap = p.tmaps + bd.bin * kMapsPerBin + 3 + (phase == 1 ? 2 : (s.cur ^ 1));
      const float c1 = 1.5f * s.a, c3 = 0.5f * s.a * s.a * s.a;
      float rsq = 0.f;
      for (int i = 0; i < n_local; ++i) {
        const PairTile t = ctl->tiles[i];
        // the outcome must be the same in all lanes: the tensor-memory loads below are warp-collective
        if (!__all_sync(0xffffffffu, mbar_wait(&tfull_bar[eacc], etph[eacc], budget, abort_flag))) {
          set_error(p.flags, NOLSM_ETIMEOUT);
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        // warps 2..5 take the left half of the tile's columns, warps 6..9 the right half
        const int hw = t.tn / 2, h0 = ((warp - 2) / 4) * hw;
        if constexpr (Q8) {
          uint8_t* stg = smem + PAIR_EPI_OFF + (warp - 2) * PAIR_NBUF * EPI_BUF_BYTES;
          if (s.iters < p.fp8_iters)   // the FP8 experiment (block-uniform)
            rsq += epi_tile<T, PAIR_NBUF, 32, true>(tmem_base + (uint32_t)(eacc * TN + h0), q, lane, out, ld, t.m0,
                                                    t.n0 + h0, hw, phase, c1, c3, smap, bd.pos * ld, stg, ebuf);
          else
            rsq += epi_tile<T, PAIR_NBUF, 64>(tmem_base + (uint32_t)(eacc * TN + h0), q, lane, out, ld, t.m0,
                                              t.n0 + h0, hw, phase, c1, c3, smap, bd.pos * ld, stg, ebuf);
        } else {
          rsq += epi_tile<T, PAIR_NBUF, 64>(tmem_base + (uint32_t)(eacc * TN + h0), q, lane, out, ld, t.m0, t.n0 + h0, hw,
                                        phase, c1, c3, smap, bd.pos * ld,
                                        smem + PAIR_EPI_OFF + (warp - 2) * PAIR_NBUF * EPI_BUF_BYTES, ebuf);
        }
        tc_fence_before();
        mbar_arrive(&tempty_bar[eacc]);
        etph[eacc] ^= 1u;
        eacc ^= 1;
      }
      if (phase == 1) {
        for (int o = 16; o; o >>= 1) rsq += __shfl_xor_sync(0xffffffffu, rsq, o);
        if (lane == 0) atomicAdd(&ctl->rsq[par], rsq);
      }
      if (lane == 0) bulk_wait0();           // this product's tensor stores are complete
      __syncwarp();
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
  };

  for (;;) {
    if (rank == 0 && threadIdx.x == 0) {
      const int b = queue_block(p, atomicAdd(&p.flags->queue, 1));
      ctl0->block = b;
      ctl1->block = b;
    }
    cluster_sync_all();
    const int b = ctl->block;
    if (b >= p.n_blocks) break;
    const BlockDesc bd = p.blocks[b];
    NsState s = p.st[b];
    if (threadIdx.x == 0) {
      const int k = pair_tiles(bd.n_pad, rank, ctl->tiles);
      ctl->n_local = k < 0 ? 0 : k;
      if (k < 0) {
        set_error(p.flags, NOLSM_EINVAL);
        *abort_flag = 1;
      }
    }
    pair_fill<T, PAIR_THREADS>(bd, p.a0, s.alpha, p.mu, reinterpret_cast<T*>(p.x0), rank);
    __syncthreads();
    cluster_sync_all();
    bool stop = false;
    for (;;) {
      const int par = round & 1;
      product(bd, s, 1, par);
      if (threadIdx.x == 0) ctl->abort_pub[par] = *abort_flag;
      cluster_sync_all();
      const float rsq = ctl0->rsq[par] + ctl1->rsq[par];
      const int aborted = ctl0->abort_pub[par] | ctl1->abort_pub[par];
      if (threadIdx.x == 0) ctl->rsq[par ^ 1] = 0.f;   // next round's slot (last read one round ago)
      round += 1;
      if (aborted) { stop = true; break; }
      const float res = sqrtf(rsq);
      if (p.detect_divergence && s.iters >= 1 && s.restarts == 0 &&
          (!isfinite(res) || res > 1.5f * sqrtf((float)bd.n_pad))) {
        // the scale was too small: restart from the Gershgorin scale (once per block)
        s.restarts += 1;
        s.alpha = (float)(fmax(fabs(p.hi[b] - p.mu), fabs(p.mu - p.lo[b])) * (1.0 + p.margin));
        s.l = p.scaled ? fminf(p.l0, 1.f) : 1.f;   // p.l0 carries the format's floor
        s.a = cc_scale(s.l);
        s.res = FLT_MAX;
        s.res_prev = FLT_MAX;
        s.cur = 0;
        s.grow = 0;
        s.status = kActive;
        pair_fill<T, PAIR_THREADS>(bd, p.a0, s.alpha, p.mu, reinterpret_cast<T*>(p.x0), rank);
        cluster_sync_all();
        continue;
      }
      if (!isfinite(res)) {
        s.status = kFailed;
        s.res = res;
        if (rank == 0 && threadIdx.x == 0) set_error(p.flags, NOLSM_ENONFINITE);
        break;
      }
      s.res_prev = s.res;
      s.res = res;
      const bool plain = s.l >= 1.f;
      if (res <= p.tol[b]) { s.status = kConverged; break; }
      if (plain && s.iters >= 2 && res < 0.25f && res > 0.5f * s.res_prev) { s.status = kConverged; break; }
      if (s.iters >= p.max_iter) {
        s.status = kFailed;
        if (rank == 0 && threadIdx.x == 0) set_error(p.flags, NOLSM_ENOCONV);
        break;
      }
      product(bd, s, 2, par);
      cluster_sync_all();
      s.cur ^= 1;
      s.iters += 1;
      s.l = cc_next(s.l, s.a);
      s.a = cc_scale(s.l);
    }
    if (rank == 0 && threadIdx.x == 0) p.st[b] = s;
    if (stop) break;
  }

  // teardown: every copy and product issued here lands before shared and tensor memory go away
  if (warp == 0 && lane == 0) {
    volatile int never = 0;
    for (int st = 0; st < PAIR_STAGES; ++st)
      if (armed & (1u << st)) mbar_wait(&full_bar[st], (arm_parity >> st) & 1u, drain_budget, &never);
  } else if (warp == 1 && lane == 0) {
    umma_commit(drain_bar);
    volatile int never = 0;
    mbar_wait(drain_bar, 0, drain_budget, &never);
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
  cluster_sync_all();
}

// The persistent schedule with two blocks per cluster (NOLSM_SCHEDULE_PERSISTENT_INTERLEAVED).
// ns_pair_kernel passes a cluster barrier after every product of its one block: the tail of the
// product (last epilogue, completion of its tensor stores, the skew between the two CTAs) and the
// ramp of the next one leave the tensor pipe idle.  Here a cluster holds two blocks (slots) and
// runs, per round, the phase-1 products of both, one barrier, the checks of both, the phase-2
// products of both and one barrier, so each barrier covers two products and the second product's
// loads and MMAs overlap the first one's tail.  Blocks are independent, so the arithmetic of every
// block is that of ns_pair_kernel.  A slot whose block converges, fails or finds the queue empty is
// refilled at the end of the round (its claim published before the round's second barrier); the
// restart of a diverged block refills its X_0 before that barrier.  Every branch around a cluster
// barrier depends only on values both CTAs read after a barrier, so both pass the same sequence.
struct Pair2Ctl {
  int block[2];                 // claimed block per slot (rank 0 writes it into both CTAs)
  int n_local[2];               // tiles of each product held by this CTA, per slot
  float rsq[2][2];              // ||T - I||_F^2 partial per slot and round parity
  int abort_pub[2];             // this CTA's abort flag as published for the round, by parity
  PairTile tiles[2][PAIR_MAX_TILES];
};
constexpr int PAIR2_SMEM = 1024 + PAIR_TAB_OFF + (int)sizeof(Pair2Ctl);
static_assert(PAIR2_SMEM <= 227 * 1024, "shared memory of the interleaved persistent kernel");

template <typename T>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PAIR_THREADS, 1) ns_pair2_kernel(const __grid_constant__ PairParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stage_base = smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + PAIR_BAR_OFF);
  uint64_t* full_bar = bars;                             // [PAIR_STAGES]
  uint64_t* empty_bar = bars + PAIR_STAGES;              // [PAIR_STAGES]
  uint64_t* tfull_bar = bars + 2 * PAIR_STAGES;          // [2]
  uint64_t* tempty_bar = bars + 2 * PAIR_STAGES + 2;     // [2]
  uint64_t* drain_bar = bars + 2 * PAIR_STAGES + 4;      // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * PAIR_STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  Pair2Ctl* ctl = reinterpret_cast<Pair2Ctl*>(smem + PAIR_TAB_OFF);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  Pair2Ctl* ctl0 = cluster_peer(ctl, 0u);
  Pair2Ctl* ctl1 = cluster_peer(ctl, 1u);
  if (threadIdx.x == 0) {
    for (int s = 0; s < PAIR_STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    for (int a = 0; a < 2; ++a) { mbar_init(&tfull_bar[a], 1); mbar_init(&tempty_bar[a], 32 * PAIR_EPI_WARPS); }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    for (int k = 0; k < 2; ++k) ctl->rsq[k][0] = ctl->rsq[k][1] = 0.f;
    ctl->abort_pub[0] = ctl->abort_pub[1] = 0;
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
  cluster_sync_all();   // both CTAs initialised before either touches the other's shared memory
  const uint32_t tmem_base = *tmem_slot;
  const long long budget = p.budget;
  const long long drain_budget = budget > (1LL << 22) ? budget : (1LL << 22);
  const int q = warp & 3;

  // ring state of each role, carried across products, slots and blocks
  int ps = 0;
  uint32_t pph = 0, armed = 0, arm_parity = 0;
  int ms = 0;
  uint32_t mph = 0, mtph[2] = {0u, 0u};
  int macc = 0;
  uint32_t etph[2] = {0u, 0u};
  int eacc = 0;
  int ebuf = 0;
  int round = 0;

  // one product of slot k: phase 1 T = X X^T -> B, phase 2 X+ = X B^T (as in ns_pair_kernel)
  auto product = [&](int k, const BlockDesc& bd, const NsState& s, int phase, int par) {
    const int ld = bd.n_pad;
    const int n_local = ctl->n_local[k];
    const PairTile* tiles = ctl->tiles[k];
    if (warp == 0) {
      if (lane == 0) {
        const CUtensorMap* ma = p.tmaps + bd.bin * kMapsPerBin + s.cur;
        const CUtensorMap* mb = (phase == 1) ? ma : p.tmaps + bd.bin * kMapsPerBin + 2;
        const int rowbase = bd.pos * ld;
        bool ok = true;
        for (int i = 0; i < n_local && ok; ++i) {
          const PairTile t = tiles[i];
          const uint32_t bytes = A_BYTES + t.tn * TK * 2;
          for (int k0 = 0; k0 < ld; k0 += TK) {
            if (!mbar_wait(&empty_bar[ps], pph ^ 1u, budget, abort_flag)) { ok = false; break; }
            mbar_expect_tx(&full_bar[ps], bytes);
            uint8_t* a_dst = stage_base + ps * STAGE_BYTES;
            uint8_t* b_dst = a_dst + A_BYTES;
            tma_load_2d(a_dst, ma, &full_bar[ps], k0, rowbase + t.m0);
            for (int h = 0; h < t.tn; h += TM) tma_load_2d(b_dst + h * TK * 2, mb, &full_bar[ps], k0, rowbase + t.n0 + h);
            armed |= 1u << ps;
            arm_parity = (arm_parity & ~(1u << ps)) | (pph << ps);
            if (++ps == PAIR_STAGES) { ps = 0; pph ^= 1u; }
          }
        }
        if (!ok) {
          set_error(p.flags, NOLSM_ETIMEOUT);
          *abort_flag = 1;
        }
      }
    } else if (warp == 1) {
      if (lane == 0) {
        bool ok = true;
        for (int i = 0; i < n_local && ok; ++i) {
          const PairTile t = tiles[i];
          const uint32_t idesc = make_idesc(Pack<T>::fmt, TM, t.tn);
          if (!mbar_wait(&tempty_bar[macc], mtph[macc] ^ 1u, budget, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(macc * TN);
          for (int k0 = 0; k0 < ld; k0 += TK) {
            if (!mbar_wait(&full_bar[ms], mph, budget, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t a_addr = smem_u32(stage_base + ms * STAGE_BYTES);
            const uint64_t adesc = sw128_desc(a_addr);
            const uint64_t bdesc = sw128_desc(a_addr + A_BYTES);
#pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk)
              umma_f16(d_tmem, adesc + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), idesc, (k0 | kk) != 0);
            umma_commit(&empty_bar[ms]);
            if (++ms == PAIR_STAGES) { ms = 0; mph ^= 1u; }
          }
          if (!ok) break;
          umma_commit(&tfull_bar[macc]);
          mtph[macc] ^= 1u;
          macc ^= 1;
        }
        if (!ok) {
          set_error(p.flags, NOLSM_ETIMEOUT);
          *abort_flag = 1;
        }
      }
    } else {
      T* out = reinterpret_cast<T*>(phase == 1 ? p.bbuf : (s.cur ? p.x0 : p.x1)) + bd.off_mat;
      const CUtensorMap* smap = p.tmaps + bd.bin * kMapsPerBin + 3 + (phase == 1 ? 2 : (s.cur ^ 1));
      const float c1 = 1.5f * s.a, c3 = 0.5f * s.a * s.a * s.a;
      float rsq = 0.f;
      for (int i = 0; i < n_local; ++i) {
        const PairTile t = tiles[i];
        // the outcome must be the same in all lanes: the tensor-memory loads below are warp-collective
        if (!__all_sync(0xffffffffu, mbar_wait(&tfull_bar[eacc], etph[eacc], budget, abort_flag))) {
          set_error(p.flags, NOLSM_ETIMEOUT);
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        // warps 2..5 take the left half of the tile's columns, warps 6..9 the right half
        const int hw = t.tn / 2, h0 = ((warp - 2) / 4) * hw;
        rsq += epi_tile<T, PAIR_NBUF, 32>(tmem_base + (uint32_t)(eacc * TN + h0), q, lane, out, ld, t.m0, t.n0 + h0, hw,
                                      phase, c1, c3, smap, bd.pos * ld,
                                      smem + PAIR_EPI_OFF + (warp - 2) * PAIR_NBUF * EPI_BUF_BYTES, ebuf);
        tc_fence_before();
        mbar_arrive(&tempty_bar[eacc]);
        etph[eacc] ^= 1u;
        eacc ^= 1;
      }
      if (phase == 1) {
        for (int o = 16; o; o >>= 1) rsq += __shfl_xor_sync(0xffffffffu, rsq, o);
        if (lane == 0) atomicAdd(&ctl->rsq[k][par], rsq);
      }
      if (lane == 0) bulk_wait0();           // this product's tensor stores are complete
      __syncwarp();
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
  };

  int b[2] = {0, 0};
  bool live[2] = {false, false};
  BlockDesc bd[2];
  NsState s[2];
  // rank 0 claims the next block for slot k and writes it into both CTAs (read after a barrier)
  auto claim = [&](int k) {
    if (rank == 0 && threadIdx.x == 0) {
      const int nb = queue_block(p, atomicAdd(&p.flags->queue, 1));
      ctl0->block[k] = nb;
      ctl1->block[k] = nb;
    }
  };
  // after a barrier that published ctl->block[k]: the slot's block, tile table and X_0 (all threads)
  auto start = [&](int k) {
    b[k] = ctl->block[k];
    live[k] = b[k] < p.n_blocks;
    if (!live[k]) return;
    bd[k] = p.blocks[b[k]];
    s[k] = p.st[b[k]];
    if (threadIdx.x == 0) {
      const int m = pair_tiles(bd[k].n_pad, rank, ctl->tiles[k]);
      ctl->n_local[k] = m < 0 ? 0 : m;
      if (m < 0) {
        set_error(p.flags, NOLSM_EINVAL);
        *abort_flag = 1;
      }
    }
    pair_fill<T, PAIR_THREADS>(bd[k], p.a0, s[k].alpha, p.mu, reinterpret_cast<T*>(p.x0), rank);
  };

  claim(0);
  claim(1);
  cluster_sync_all();
  start(0);
  start(1);
  __syncthreads();
  cluster_sync_all();
  while (live[0] || live[1]) {
    const int par = round & 1;
    for (int k = 0; k < 2; ++k)
      if (live[k]) product(k, bd[k], s[k], 1, par);
    if (threadIdx.x == 0) ctl->abort_pub[par] = *abort_flag;
    cluster_sync_all();
    const int aborted = ctl0->abort_pub[par] | ctl1->abort_pub[par];
    float rsum[2];
    for (int k = 0; k < 2; ++k) rsum[k] = ctl0->rsq[k][par] + ctl1->rsq[k][par];
    if (threadIdx.x == 0) ctl->rsq[0][par ^ 1] = ctl->rsq[1][par ^ 1] = 0.f;   // last read one round ago
    round += 1;
    if (aborted) {
      for (int k = 0; k < 2; ++k)
        if (live[k] && rank == 0 && threadIdx.x == 0) p.st[b[k]] = s[k];
      break;
    }
    bool go[2] = {false, false}, done[2] = {false, false};
    for (int k = 0; k < 2; ++k) {
      if (!live[k]) continue;
      NsState& sk = s[k];
      const BlockDesc& bk = bd[k];
      const float res = sqrtf(rsum[k]);
      if (p.detect_divergence && sk.iters >= 1 && sk.restarts == 0 &&
          (!isfinite(res) || res > 1.5f * sqrtf((float)bk.n_pad))) {
        // the scale was too small: restart from the Gershgorin scale (once per block); X_0 is
        // refilled now and read after the round's second barrier
        sk.restarts += 1;
        sk.alpha = (float)(fmax(fabs(p.hi[b[k]] - p.mu), fabs(p.mu - p.lo[b[k]])) * (1.0 + p.margin));
        sk.l = p.scaled ? fminf(p.l0, 1.f) : 1.f;   // p.l0 carries the format's floor
        sk.a = cc_scale(sk.l);
        sk.res = FLT_MAX;
        sk.res_prev = FLT_MAX;
        sk.cur = 0;
        sk.grow = 0;
        sk.status = kActive;
        pair_fill<T, PAIR_THREADS>(bk, p.a0, sk.alpha, p.mu, reinterpret_cast<T*>(p.x0), rank);
        continue;
      }
      if (!isfinite(res)) {
        sk.status = kFailed;
        sk.res = res;
        if (rank == 0 && threadIdx.x == 0) set_error(p.flags, NOLSM_ENONFINITE);
        done[k] = true;
        continue;
      }
      sk.res_prev = sk.res;
      sk.res = res;
      const bool plain = sk.l >= 1.f;
      if (res <= p.tol[b[k]]) { sk.status = kConverged; done[k] = true; continue; }
      if (plain && sk.iters >= 2 && res < 0.25f && res > 0.5f * sk.res_prev) {
        sk.status = kConverged;
        done[k] = true;
        continue;
      }
      if (sk.iters >= p.max_iter) {
        sk.status = kFailed;
        if (rank == 0 && threadIdx.x == 0) set_error(p.flags, NOLSM_ENOCONV);
        done[k] = true;
        continue;
      }
      go[k] = true;
    }
    for (int k = 0; k < 2; ++k)
      if (done[k]) {
        if (rank == 0 && threadIdx.x == 0) p.st[b[k]] = s[k];
        claim(k);
      }
    for (int k = 0; k < 2; ++k)
      if (go[k]) product(k, bd[k], s[k], 2, par);
    __syncthreads();      // restart refills complete in this CTA before the barrier publishes them
    cluster_sync_all();
    for (int k = 0; k < 2; ++k)
      if (go[k]) {
        s[k].cur ^= 1;
        s[k].iters += 1;
        s[k].l = cc_next(s[k].l, s[k].a);
        s[k].a = cc_scale(s[k].l);
      }
    if (done[0] || done[1]) {
      for (int k = 0; k < 2; ++k)
        if (done[k]) start(k);
      __syncthreads();
      cluster_sync_all();
    }
  }

  // teardown: every copy and product issued here lands before shared and tensor memory go away
  if (warp == 0 && lane == 0) {
    volatile int never = 0;
    for (int st = 0; st < PAIR_STAGES; ++st)
      if (armed & (1u << st)) mbar_wait(&full_bar[st], (arm_parity >> st) & 1u, drain_budget, &never);
  } else if (warp == 1 && lane == 0) {
    umma_commit(drain_bar);
    volatile int never = 0;
    mbar_wait(drain_bar, 0, drain_budget, &never);
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
  cluster_sync_all();
}

// ---------------------------------------------------------------------------------------------
// The refinement steps on the own-column slab and the block traces (Eq. 4, Eq. 8) on the tensor
// cores.  With V_0 = W = L^-1[:, C_b] and X the final iterate in its FP16/BF16 storage, one step of
// Eq. 6 applied to the slab is f(X) V = 1.5 X V - 0.5 X (X (X V)); refine_iters >= 2 evaluates the
// two-step map as G = 1.5 F1 - 0.5 F3 with F1 = f(X) W, F2 = f(X) F1, F3 = f(X) F2 (nine products),
// refine_iters = 1 takes G = f(X) W (three), 0 takes G = X W (one).  Then Y = (W - G) / 2 and the
// block's traces N_b = <L[C_b, :]^T, Y>, E_b = <L^-1 T_b(H0)[:, C_b], Y> in FP64.
// A product P = X V runs as 128-row tiles of M = 128, N = the piece's column count rounded up to 16,
// K = 16 MMAs: X is the A operand exactly as stored, the FP32 slab V is the B operand split into
// hi = V rounded to the iterate's format and lo = (V - hi) rounded again, and every k-step
// accumulates X hi + X lo in FP32 tensor memory.  In FP16 the pair resolves V to 2^-22 of its size or
// 2^-24 absolute (the subnormal spacing), below FP32 rounding for the O(1) entries of these slabs;
// in BF16 to 2^-16 of its size.  Columns of a B box past the piece (the next piece's rows, or zero
// fill past the pool) only reach accumulator columns that are never read.
// One persistent CTA per SM takes pieces (block, up to NMAX own columns) off a queue and runs the
// whole chain of its piece; the products are sequential (each needs every row of the previous one)
// and separated by a CTA barrier after the epilogue's stores.  Roles (192 threads): warp 0 TMA
// producer (a 128 x 64 box of X and N/16 16 x 64 boxes each of hi and lo per stage), warp 1 MMA
// issuer, warps 2..5 epilogue (lane = row: TMEM -> registers, the step's arithmetic, coalesced
// column stores of the FP32 values and of the split of the next operand; the split pools alternate
// between two pairs).  Waits are bounded as in ns_tc_kernel.
struct SlabParams {
  const int32_t* units;         // (block, first own column, columns, 0) per piece
  int n_units;
  int32_t* queue;
  const BlockDesc* blocks;
  const NsState* st;
  const CUtensorMap* tmaps;
  const float* w;
  const float* z;
  const float* lc;
  float* y;
  float* s1;                    // P1 = X V of the current step (FP32 slab pool)
  float* f1;                    // F1 = f(X) W (FP32 slab pool)
  void* hl[4];                  // split pools hi0, lo0, hi1, lo1 (the iterate's format)
  double* bn;                   // traces per piece
  double* be;
  DevFlags* flags;
  long long budget;
  int refine;
};

template <int NMAX, int NST>
struct SlabLayout {
  static constexpr int B_BYTES = NMAX * TK * 2;          // one of hi / lo
  static constexpr int STAGE = A_BYTES + 2 * B_BYTES;
  static constexpr int BAR_OFF = NST * STAGE;
  static constexpr int SMEM = 1024 + BAR_OFF + 512;
  static_assert(NMAX % 16 == 0 && NMAX <= 256, "MMA N");
  static_assert(B_BYTES % 1024 == 0, "swizzle atoms of the B boxes");
  static_assert((2 * NST + 15) * 8 <= 512, "barrier area");
  static_assert(SMEM <= 227 * 1024, "shared memory of the slab kernel");
};

template <typename T, int NMAX, int NST>
__global__ void __launch_bounds__(NUM_THREADS, 1) slab_tc_kernel(const __grid_constant__ SlabParams p) {
  using L = SlabLayout<NMAX, NST>;
  // tensor memory: two accumulator sets of N <= NMAX columns (narrow pieces take 64 columns, so that
  // two CTAs share an SM)
  constexpr int ACC = NMAX <= 32 ? 32 : TN;
  constexpr uint32_t ALLOC = NMAX <= 32 ? 64u : (uint32_t)TMEM_COLS;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stage_base = smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::BAR_OFF);
  uint64_t* full_bar = bars;                       // [NST]
  uint64_t* empty_bar = bars + NST;                // [NST]
  uint64_t* tfull_bar = bars + 2 * NST;            // [2]
  uint64_t* tempty_bar = bars + 2 * NST + 2;       // [2]
  uint64_t* drain_bar = bars + 2 * NST + 4;        // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NST + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* s_unit = reinterpret_cast<int*>(bars + 2 * NST + 6);
  double* red = reinterpret_cast<double*>(bars + 2 * NST + 7);   // [4 warps][2]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    for (int a = 0; a < 2; ++a) { mbar_init(&tfull_bar[a], 1); mbar_init(&tempty_bar[a], 128); }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ALLOC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const long long budget = p.budget;
  const long long drain_budget = budget > (1LL << 22) ? budget : (1LL << 22);
  const int q = warp & 3;

  int ps = 0;
  uint32_t pph = 0, armed = 0, arm_parity = 0;
  int ms = 0;
  uint32_t mph = 0, mtph[2] = {0u, 0u};
  int macc = 0;
  uint32_t etph[2] = {0u, 0u};
  int eacc = 0;

  for (;;) {
    if (threadIdx.x == 0) *s_unit = atomicAdd(p.queue, 1);
    __syncthreads();
    const int u = *s_unit;
    if (u >= p.n_units || *abort_flag) break;
    const int b = p.units[4 * u], c0 = p.units[4 * u + 1], cw = p.units[4 * u + 2];
    const BlockDesc bd = p.blocks[b];
    const int cur = p.st[b].cur;
    const int ld = bd.n_pad, N = (cw + 15) & ~15;
    const int64_t so = bd.off_slab + (int64_t)c0 * ld;   // the piece's first column in the slab pools
    const int nf = p.refine >= 2 ? 3 : p.refine;         // steps of Eq. 6 (0: the single product G = X W)
    const int nprod = nf == 0 ? 1 : 3 * nf;
    {
      // V_0 = W, split into the first pool pair
      const int64_t len = (int64_t)cw * ld;
      for (int64_t e = threadIdx.x; e < len; e += NUM_THREADS) {
        const float v = p.w[so + e];
        const T hi = Pack<T>::one(v);
        reinterpret_cast<T*>(p.hl[0])[so + e] = hi;
        reinterpret_cast<T*>(p.hl[1])[so + e] = Pack<T>::one(v - Pack<T>::f(hi));
      }
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    __syncthreads();
    double sn = 0.0, se = 0.0;
    for (int pi = 0; pi < nprod && !*abort_flag; ++pi) {
      const int src = pi & 1;                              // pool pair read by this product
      if (warp == 0) {
        if (lane == 0) {
          const CUtensorMap* ma = p.tmaps + bd.bin * kMapsPerBin + cur;
          const CUtensorMap* mh = p.tmaps + bd.bin * kMapsPerBin + 6 + 2 * src;
          const CUtensorMap* ml = mh + 1;
          const uint32_t bytes = (uint32_t)A_BYTES + 4u * (uint32_t)N * TK;
          const int ra = bd.pos * ld, rb = bd.slab_row + c0;
          bool ok = true;
          for (int m0 = 0; m0 < ld && ok; m0 += TM)
            for (int k0 = 0; k0 < ld; k0 += TK) {
              if (!mbar_wait(&empty_bar[ps], pph ^ 1u, budget, abort_flag)) { ok = false; break; }
              mbar_expect_tx(&full_bar[ps], bytes);
              uint8_t* a_dst = stage_base + ps * L::STAGE;
              uint8_t* h_dst = a_dst + A_BYTES;
              uint8_t* l_dst = h_dst + L::B_BYTES;
              tma_load_2d(a_dst, ma, &full_bar[ps], k0, ra + m0);
              for (int h = 0; h < N; h += 16) {
                tma_load_2d(h_dst + h * TK * 2, mh, &full_bar[ps], k0, rb + h);
                tma_load_2d(l_dst + h * TK * 2, ml, &full_bar[ps], k0, rb + h);
              }
              armed |= 1u << ps;
              arm_parity = (arm_parity & ~(1u << ps)) | (pph << ps);
              if (++ps == NST) { ps = 0; pph ^= 1u; }
            }
          if (!ok) {
            set_error(p.flags, NOLSM_ETIMEOUT);
            *abort_flag = 1;
          }
        }
      } else if (warp == 1) {
        if (lane == 0) {
          const uint32_t idesc = make_idesc(Pack<T>::fmt, TM, N);
          bool ok = true;
          for (int m0 = 0; m0 < ld && ok; m0 += TM) {
            if (!mbar_wait(&tempty_bar[macc], mtph[macc] ^ 1u, budget, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t d_tmem = tmem_base + (uint32_t)(macc * ACC);
            for (int k0 = 0; k0 < ld; k0 += TK) {
              if (!mbar_wait(&full_bar[ms], mph, budget, abort_flag)) { ok = false; break; }
              tc_fence_after();
              const uint32_t a_addr = smem_u32(stage_base + ms * L::STAGE);
              const uint64_t adesc = sw128_desc(a_addr);
              const uint64_t hdesc = sw128_desc(a_addr + A_BYTES);
              const uint64_t ldesc = sw128_desc(a_addr + A_BYTES + L::B_BYTES);
#pragma unroll
              for (int kk = 0; kk < TK / 16; ++kk) {
                umma_f16(d_tmem, adesc + (uint64_t)(kk * 2), hdesc + (uint64_t)(kk * 2), idesc, (k0 | kk) != 0);
                umma_f16(d_tmem, adesc + (uint64_t)(kk * 2), ldesc + (uint64_t)(kk * 2), idesc, 1);
              }
              umma_commit(&empty_bar[ms]);
              if (++ms == NST) { ms = 0; mph ^= 1u; }
            }
            if (!ok) break;
            umma_commit(&tfull_bar[macc]);
            mtph[macc] ^= 1u;
            macc ^= 1;
          }
          if (!ok) {
            set_error(p.flags, NOLSM_ETIMEOUT);
            *abort_flag = 1;
          }
        }
      } else {
        const int t = pi % 3, f = pi / 3;
        T* dh = reinterpret_cast<T*>(src ? p.hl[0] : p.hl[2]);   // the pool pair the next product reads
        T* dl = reinterpret_cast<T*>(src ? p.hl[1] : p.hl[3]);
        for (int m0 = 0; m0 < ld; m0 += TM) {
          // the outcome must be the same in all lanes: the tensor-memory loads below are warp-collective
          if (!__all_sync(0xffffffffu, mbar_wait(&tfull_bar[eacc], etph[eacc], budget, abort_flag))) {
            set_error(p.flags, NOLSM_ETIMEOUT);
            *abort_flag = 1;
            break;
          }
          tc_fence_after();
          const int m = m0 + q * 32 + lane;
          const uint32_t tb = tmem_base + (uint32_t)(eacc * ACC) + ((uint32_t)(q * 32) << 16);
          for (int j0 = 0; j0 < N; j0 += 16) {
            uint32_t v[16];
            tmem_ld16(tb + (uint32_t)j0, v);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
              const int j = j0 + jj;
              if (j >= cw) break;
              const int64_t o = so + (int64_t)j * ld + m;
              const float x = __uint_as_float(v[jj]);
              float nv = 0.f, g = 0.f;
              bool split = false, last = false;
              if (nf == 0) {
                g = x;
                last = true;
              } else if (t == 0) {
                p.s1[o] = x;
                nv = x;
                split = true;
              } else if (t == 1) {
                nv = x;
                split = true;
              } else {
                const float fv = 1.5f * p.s1[o] - 0.5f * x;
                if (f == 0 && nf > 1) p.f1[o] = fv;
                if (f < nf - 1) {
                  nv = fv;
                  split = true;
                } else {
                  g = nf > 1 ? 1.5f * p.f1[o] - 0.5f * fv : fv;
                  last = true;
                }
              }
              if (split) {
                const T hi = Pack<T>::one(nv);
                dh[o] = hi;
                dl[o] = Pack<T>::one(nv - Pack<T>::f(hi));
              }
              if (last) {
                const float yv = 0.5f * (p.w[o] - g);
                p.y[o] = yv;
                sn += (double)p.lc[o] * (double)yv;
                se += (double)p.z[o] * (double)yv;
              }
            }
          }
          tc_fence_before();
          mbar_arrive(&tempty_bar[eacc]);
          etph[eacc] ^= 1u;
          eacc ^= 1;
        }
        asm volatile("fence.proxy.async.global;" ::: "memory");   // the next product's operand loads
      }
      __syncthreads();
    }
    if (warp >= 2) {
      for (int o = 16; o; o >>= 1) {
        sn += __shfl_xor_sync(0xffffffffu, sn, o);
        se += __shfl_xor_sync(0xffffffffu, se, o);
      }
      if (lane == 0) {
        red[2 * (warp - 2)] = sn;
        red[2 * (warp - 2) + 1] = se;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      p.bn[u] = (red[0] + red[2]) + (red[4] + red[6]);
      p.be[u] = (red[1] + red[3]) + (red[5] + red[7]);
    }
  }

  // teardown: every copy and product issued here lands before shared and tensor memory go away
  if (warp == 0 && lane == 0) {
    volatile int never = 0;
    for (int s = 0; s < NST; ++s)
      if (armed & (1u << s)) mbar_wait(&full_bar[s], (arm_parity >> s) & 1u, drain_budget, &never);
  } else if (warp == 1 && lane == 0) {
    umma_commit(drain_bar);
    volatile int never = 0;
    mbar_wait(drain_bar, 0, drain_budget, &never);
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(ALLOC) : "memory");
  }
}

// ---------------------------------------------------------------------------------------------
// Trailing update of the blocked double-float Cholesky on the tensor cores.  After panel p (columns
// [c0, c0 + 64)) is factored, every trailing entry C[r, c] (c0 + 64 <= c <= r) loses
// sum_{k in panel} L[r, k] L[c, k].  Each L entry is split into six 8-bit integers on its row's
// scale (oz_slices; Ozaki, Ogita, Oishi & Rump 2012), so
//   L[r, k] L[c, k] = 2^(e_r + e_c - 16) sum_{s, t} q_s(r, k) q_t(c, k) 2^(-8 (s + t))
// and the pairs with s + t = l <= 5 are summed over k by BF16 MMAs into the FP32 tensor-memory
// accumulator of level l: every product is an integer of at most 2^16 and a level's sum stays at
// or below 2^23, so the accumulators are exact.  Pairs with s + t > 5 lie below 2^-47 of the scale
// per term and are dropped (the double-float arithmetic keeps 2^-48).  The epilogue adds the levels
// in double-float from the smallest up, scales by the power of two and subtracts from C (pairs in
// place).
// Work item = (block, 32 columns n0): the six 32 x 64 B planes of rows n0.. stay in shared memory
// (double-buffered across items) while the 128-row A tiles of rows >= n0 - 127 stream through a
// six-stage ring, one plane per stage.  Plane s of A meets the B planes t = 0 .. 5 - s in one MMA of
// N = 32 (6 - s) (the B planes are stacked, so its output columns are the accumulators of levels
// s .. 5): 6 x 4 K-steps = 24 MMAs (M = 128, K = 16, 21 slice pairs) per tile into 6 x 32
// accumulator columns, two
// accumulator sets.  The tile's 128 x 32 pairs of C
// (32 KB) come into shared memory by two tensor copies issued with the tile's planes (two C buffers,
// so the next tile's C is in flight while the epilogue works) and go back by one tensor store per
// epilogue warp (its 32 rows x 16 columns); the pool is read and written as whole boxes instead of
// per-lane rows that the epilogue would wait on.  Items go round-robin to the CTAs (neighbouring
// columns of one block run side by side and share its A planes in L2).  Roles (320
// threads): warp 0 TMA producer, warp 1 MMA issuer, warps 2..9 epilogue (two per TMEM lane quarter,
// 16 columns each).  Waits are bounded as in ns_tc_kernel.
// A 128-row box that starts 64 rows before the end of the block reaches into the next block of the
// bin's stack: its loads are harmless and unused, and no store is issued for a 32-row group that
// starts at or past n (so nothing outside the block's own rows is written).
constexpr int OZ_NSL = kOzSlices;
constexpr int OZ_TN = 32;
constexpr int OZ_NST = 6;
constexpr int OZ_A_BYTES = TM * kOzPanel * 2;                  // one plane of a 128-row tile
constexpr int OZ_PLANE_B = OZ_TN * kOzPanel * 2;               // one plane of 32 rows
constexpr int OZ_B_BYTES = OZ_NSL * OZ_PLANE_B;                // 24 KB
constexpr int OZ_B_OFF = OZ_NST * OZ_A_BYTES;
constexpr int OZ_CBOX_BYTES = TM * 16 * 8;                     // 128 rows x 16 pairs (128-byte rows)
constexpr int OZ_C_BYTES = 2 * OZ_CBOX_BYTES;                  // the tile's 128 x 32 pairs of C
constexpr int OZ_C_OFF = OZ_B_OFF + 2 * OZ_B_BYTES;
constexpr int OZ_BAR_OFF = OZ_C_OFF + 2 * OZ_C_BYTES;
constexpr int OZ_SMEM = 1024 + OZ_BAR_OFF + 256;
constexpr int OZ_THREADS = 320;
constexpr int OZ_ACC = 256;                                     // column offset of the second set
static_assert(OZ_NSL * OZ_TN <= OZ_ACC, "accumulator set");
static_assert(OZ_SMEM <= 227 * 1024, "shared memory of the update kernel");
static_assert(kOzPanel == TK, "one 128-byte swizzle row per plane row");

struct OzParams {
  const int32_t* items;         // (block, n0) pairs of this panel
  int n_items;
  const BlockDesc* blocks;
  const CUtensorMap* maps;      // [0]: 64 x 128 boxes, [1]: 64 x 32 boxes over the slice planes;
                                // per bin [2 + 2 bin]: 16 x 128 loads, [3 + 2 bin]: 16 x 32 stores of C
  double* pool;
  const int32_t* scale_exp;
  int t0;                       // first trailing row / column
  DevFlags* flags;
  long long budget;
};

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// first 128-row tile of column chunk n0 that reaches the diagonal
__device__ __forceinline__ int oz_first_m(int t0, int n0) {
  const int d = n0 - t0 - (TM - 1);
  return t0 + (d > 0 ? (d + TM - 1) / TM : 0) * TM;
}

__global__ void __launch_bounds__(OZ_THREADS, 1) chol_update_kernel(const __grid_constant__ OzParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OZ_BAR_OFF);
  uint64_t* full_bar = bars;                        // [OZ_NST]
  uint64_t* empty_bar = bars + OZ_NST;              // [OZ_NST]
  uint64_t* bfull_bar = bars + 2 * OZ_NST;          // [2]
  uint64_t* bempty_bar = bars + 2 * OZ_NST + 2;     // [2]
  uint64_t* tfull_bar = bars + 2 * OZ_NST + 4;      // [2]
  uint64_t* tempty_bar = bars + 2 * OZ_NST + 6;     // [2]
  uint64_t* cfull_bar = bars + 2 * OZ_NST + 8;      // [2] the tile's C landed
  uint64_t* cempty_bar = bars + 2 * OZ_NST + 10;    // [2] every epilogue warp's store has read its C
  uint64_t* drain_bar = bars + 2 * OZ_NST + 12;     // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * OZ_NST + 13);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_NST; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&bfull_bar[a], 1);
      mbar_init(&bempty_bar[a], 1);
      mbar_init(&tfull_bar[a], 1);
      mbar_init(&tempty_bar[a], 256);
      mbar_init(&cfull_bar[a], 1);
      mbar_init(&cempty_bar[a], 8);
    }
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
  const long long drain_budget = budget > (1LL << 22) ? budget : (1LL << 22);
  const int t0 = p.t0;

  if (warp == 0) {
    if (lane == 0) {
      int ps = 0, bb = 0, cb = 0;
      uint32_t pph = 0, bph[2] = {0u, 0u}, cph[2] = {0u, 0u};
      uint32_t armed = 0, arm_parity = 0, barmed = 0, barm_parity = 0, carmed = 0, carm_parity = 0;
      bool ok = true;
      for (int it = blockIdx.x; it < p.n_items && ok; it += gridDim.x) {
        const int b = p.items[2 * it], n0 = p.items[2 * it + 1];
        const BlockDesc bd = p.blocks[b];
        const int np = bd.n_pad, rbase = OZ_NSL * bd.row_off;
        const CUtensorMap* cmap = p.maps + 2 + 2 * bd.bin;
        const int crow = bd.pos * np;
        if (!mbar_wait(&bempty_bar[bb], bph[bb] ^ 1u, budget, abort_flag)) { ok = false; break; }
        mbar_expect_tx(&bfull_bar[bb], OZ_B_BYTES);
        uint8_t* bdst = smem + OZ_B_OFF + bb * OZ_B_BYTES;
        for (int t = 0; t < OZ_NSL; ++t) tma_load_2d(bdst + t * OZ_PLANE_B, p.maps + 1, &bfull_bar[bb], 0, rbase + t * np + n0);
        barmed |= 1u << bb;
        barm_parity = (barm_parity & ~(1u << bb)) | (bph[bb] << bb);
        bph[bb] ^= 1u;
        bb ^= 1;
        for (int m0 = oz_first_m(t0, n0); m0 < bd.n && ok; m0 += TM) {
          // the tile's C: two 128 x 16 boxes of pairs
          if (!mbar_wait(&cempty_bar[cb], cph[cb] ^ 1u, budget, abort_flag)) { ok = false; break; }
          mbar_expect_tx(&cfull_bar[cb], OZ_C_BYTES);
          uint8_t* cdst = smem + OZ_C_OFF + cb * OZ_C_BYTES;
          tma_load_2d(cdst, cmap, &cfull_bar[cb], n0, crow + m0);
          tma_load_2d(cdst + OZ_CBOX_BYTES, cmap, &cfull_bar[cb], n0 + 16, crow + m0);
          carmed |= 1u << cb;
          carm_parity = (carm_parity & ~(1u << cb)) | (cph[cb] << cb);
          cph[cb] ^= 1u;
          cb ^= 1;
          for (int s = 0; s < OZ_NSL; ++s) {
            if (!mbar_wait(&empty_bar[ps], pph ^ 1u, budget, abort_flag)) { ok = false; break; }
            mbar_expect_tx(&full_bar[ps], OZ_A_BYTES);
            tma_load_2d(smem + ps * OZ_A_BYTES, p.maps, &full_bar[ps], 0, rbase + s * np + m0);
            armed |= 1u << ps;
            arm_parity = (arm_parity & ~(1u << ps)) | (pph << ps);
            if (++ps == OZ_NST) { ps = 0; pph ^= 1u; }
          }
        }
      }
      if (!ok) {
        set_error(p.flags, NOLSM_ETIMEOUT);
        *abort_flag = 1;
      }
      // every copy issued here lands before the CTA's shared memory goes away
      volatile int never = 0;
      for (int s = 0; s < OZ_NST; ++s)
        if (armed & (1u << s)) mbar_wait(&full_bar[s], (arm_parity >> s) & 1u, drain_budget, &never);
      for (int a = 0; a < 2; ++a) {
        if (barmed & (1u << a)) mbar_wait(&bfull_bar[a], (barm_parity >> a) & 1u, drain_budget, &never);
        if (carmed & (1u << a)) mbar_wait(&cfull_bar[a], (carm_parity >> a) & 1u, drain_budget, &never);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int ms = 0, bb = 0, acc = 0;
      uint32_t mph = 0, bph[2] = {0u, 0u}, tph[2] = {0u, 0u};
      bool ok = true;
      for (int it = blockIdx.x; it < p.n_items && ok; it += gridDim.x) {
        const int b = p.items[2 * it], n0 = p.items[2 * it + 1];
        const int nb = p.blocks[b].n;
        if (!mbar_wait(&bfull_bar[bb], bph[bb], budget, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t b_addr = smem_u32(smem + OZ_B_OFF + bb * OZ_B_BYTES);
        for (int m0 = oz_first_m(t0, n0); m0 < nb && ok; m0 += TM) {
          if (!mbar_wait(&tempty_bar[acc], tph[acc] ^ 1u, budget, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d0 = tmem_base + (uint32_t)(acc * OZ_ACC);
          for (int s = 0; s < OZ_NSL; ++s) {
            if (!mbar_wait(&full_bar[ms], mph, budget, abort_flag)) { ok = false; break; }
            tc_fence_after();
            // A plane s against B planes t = 0 .. 5 - s in one MMA: the planes lie back to back (32 rows
            // each), so output column 32 t + j lands in the accumulator of level s + t, column j
            const uint64_t adesc = sw128_desc(smem_u32(smem + ms * OZ_A_BYTES));
            const uint64_t bdesc = sw128_desc(b_addr);
            const uint32_t idesc = make_idesc(1, TM, OZ_TN * (OZ_NSL - s));   // BF16 operands
            const uint32_t d = d0 + (uint32_t)(s * OZ_TN);
#pragma unroll
            for (int kk = 0; kk < kOzPanel / 16; ++kk)
              umma_f16(d, adesc + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), idesc, (s | kk) != 0);
            umma_commit(&empty_bar[ms]);
            if (++ms == OZ_NST) { ms = 0; mph ^= 1u; }
          }
          if (!ok) break;
          umma_commit(&tfull_bar[acc]);
          tph[acc] ^= 1u;
          acc ^= 1;
        }
        if (!ok) break;
        umma_commit(&bempty_bar[bb]);   // the item's planes are free once its products are done
        bph[bb] ^= 1u;
        bb ^= 1;
      }
      if (!ok) {
        set_error(p.flags, NOLSM_ETIMEOUT);
        *abort_flag = 1;
      }
      umma_commit(drain_bar);
      volatile int never = 0;
      mbar_wait(drain_bar, 0, drain_budget, &never);
    }
  } else {
    const int q = warp & 3, half = (warp - 2) >> 2;
    int acc = 0, cb = 0, pend = -1;
    uint32_t tph[2] = {0u, 0u}, cph[2] = {0u, 0u};
    for (int it = blockIdx.x; it < p.n_items; it += gridDim.x) {
      const int b = p.items[2 * it], n0 = p.items[2 * it + 1];
      const BlockDesc bd = p.blocks[b];
      const int np = bd.n_pad, n = bd.n;
      const CUtensorMap* smap = p.maps + 3 + 2 * bd.bin;
      const int32_t* ex = p.scale_exp + bd.row_off;
      bool stop = false;
      for (int m0 = oz_first_m(t0, n0); m0 < n; m0 += TM) {
        // the previous tile's store has read its C buffer: hand the buffer back to the producer
        if (pend >= 0) {
          if (lane == 0) {
            bulk_wait_read0();
            mbar_arrive(&cempty_bar[pend]);
          }
          pend = -1;
        }
        const bool got = mbar_wait(&cfull_bar[cb], cph[cb], budget, abort_flag) &&
                         mbar_wait(&tfull_bar[acc], tph[acc], budget, abort_flag);
        if (!__all_sync(0xffffffffu, got)) {
          set_error(p.flags, NOLSM_ETIMEOUT);
          *abort_flag = 1;
          stop = true;
          break;
        }
        tc_fence_after();
        const int rw0 = m0 + q * 32;              // first row of this warp
        const int r = rw0 + lane;
        const int er = r < n ? ex[r] : 0;
        // e_c of this warp's 16 columns (lane l < 16 holds column n0 + 16 half + l; handed out by shuffles)
        const int cl = n0 + half * 16 + (lane & 15);
        const int ecl = cl < n ? ex[cl] : 0;
        uint8_t* cbox = smem + OZ_C_OFF + cb * OZ_C_BYTES + half * OZ_CBOX_BYTES;   // 128 rows x 16 pairs
        const int crow = q * 32 + lane;           // this lane's row in the box
        // both 8-column chunks' levels are loaded before one wait (a chunk above every row of this
        // warp is skipped; warp-uniform)
        uint32_t vv[2][OZ_NSL][8];
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          if (n0 + half * 16 + ch * 8 > rw0 + 31) continue;
          const uint32_t tb = tmem_base + (uint32_t)(acc * OZ_ACC + half * 16 + ch * 8) + ((uint32_t)(q * 32) << 16);
#pragma unroll
          for (int l = 0; l < OZ_NSL; ++l) tmem_ld8(tb + (uint32_t)(l * OZ_TN), vv[ch][l]);
        }
        tmem_wait_ld();
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          const int c0 = n0 + half * 16 + ch * 8;
          if (c0 > rw0 + 31) continue;            // chunk above every row of this warp (uniform)
          const uint32_t (&v)[OZ_NSL][8] = vv[ch];
          int ec[8];                              // every lane takes part in the shuffles
#pragma unroll
          for (int j = 0; j < 8; ++j) ec[j] = __shfl_sync(0xffffffffu, ecl, ch * 8 + j);
          if (r >= n || c0 > r) continue;
          // the lane's 8 pairs: 64 bytes = four 16-byte units of its 128-byte row (128-byte swizzle)
          float4 cv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) cv[u] = *reinterpret_cast<const float4*>(cbox + sw128(crow, ch * 64 + 16 * u));
          float* cf = reinterpret_cast<float*>(cv);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int c = c0 + j;
            if (c > r) break;
            // sum_l v_l 2^(-8 l) in double-float, smallest level first (every term is exact)
            float h = __uint_as_float(v[OZ_NSL - 1][j]) * 0x1p-40f, lo = 0.f;
#pragma unroll
            for (int l = OZ_NSL - 2; l >= 0; --l) {
              const float x = __uint_as_float(v[l][j]) * __int_as_float((127 - kOzBits * l) << 23);
              const float s = h + x;
              const float bb2 = s - h;
              lo += (h - (s - bb2)) + (x - bb2);
              h = s;
            }
            const float sc = __int_as_float((127 + er + ec[j] - 2 * kOzBits) << 23);
            h *= sc;
            lo *= sc;
            // C - (h + lo), renormalised
            const float ch0 = cf[2 * j], cl0 = cf[2 * j + 1];
            const float s = ch0 - h;
            const float bb2 = s - ch0;
            const float err = (ch0 - (s - bb2)) - (h + bb2);
            const float t = err + cl0 - lo;
            const float sh = s + t;                  // TwoSum(s, t)
            const float bb3 = sh - s;
            cf[2 * j] = sh;
            cf[2 * j + 1] = (s - (sh - bb3)) + (t - bb3);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) *reinterpret_cast<float4*>(cbox + sw128(crow, ch * 64 + 16 * u)) = cv[u];
        }
        tc_fence_before();
        mbar_arrive(&tempty_bar[acc]);
        tph[acc] ^= 1u;
        acc ^= 1;
        // this warp's 32 rows x 16 columns back to the pool, when it changed any of them: rows from
        // n on are left alone (a group that starts before n ends before n_pad)
        fence_async_smem();
        __syncwarp();
        if (lane == 0 && rw0 < n && n0 + half * 16 <= rw0 + 31) {
          tma_store_2d(smap, cbox + q * 32 * 128, n0 + half * 16, bd.pos * np + rw0);
          bulk_commit();
        }
        pend = cb;
        cph[cb] ^= 1u;
        cb ^= 1;
      }
      if (stop) break;
    }
    if (lane == 0) bulk_wait0();                  // every store of this warp has landed
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

// ---------------------------------------------------------------------------------------------
// TRSM of the blocked double-float Cholesky on the tensor cores: after the diagonal block of panel
// [c0, c0 + 64) is factored, the rows below it become L21 = A21 L11^-T, i.e.
//   L21[r, c] = sum_{k in panel} A21[r, k] Minv[c, k],   Minv = L11^-1 (lower triangular),
// with the same exact slicing as the trailing update (Ozaki, Ogita, Oishi & Rump 2012).  A21[r, k]
// is split on the scale 2^(e_r + g), g = max_k e_k over the panel's rows: by Cauchy-Schwarz on the
// rows of the factor |A21[r, k]| <= sqrt(S_rr S_kk) <= 2^(e_r + g).  Row c of Minv is split on its own
// scale 2^f_c (chol_diag64_kernel).  So
//   L21[r, c] = 2^(e_r + g + f_c - 16) sum_l 2^(-8 l) sum_{s + t = l} sum_k q_s(r, k) p_t(c, k),
// every level sum exact in FP32 (at most 2^23, see oz_slices), the pairs with s + t > 5 (below
// 2^-47 of the scale per term) dropped.  The epilogue adds the levels in double-float, writes
// L21 as pairs over A21 and its slices on the row scale e_r into the planes the trailing update reads.
// Work item = (block, 128 rows m0 of the rows below the diagonal block): the CTA keeps the block's
// Minv planes (both 32-column halves, 48 KB) while its items follow each other (contiguous runs of
// the item list per CTA), the item's 128 x 64 A21 pairs arrive as four 128 x 16 tensor copies through
// a three-box staging ring, converter warps slice them into six A planes in shared memory, and the
// MMA issuer runs, per half and per A plane s, one MMA against the stacked
// B planes t = 0 .. 5 - s (N = 32 (6 - s)), so the 6 levels x 32 columns of a half land in one of
// the two accumulator sets.  Roles (448 threads): warp 0 TMA producer (Minv planes), warp 1 MMA
// issuer, warps 2..5 converter, warps 6..13 epilogue (one per TMEM lane quarter and half).  Waits
// are bounded as in ns_tc_kernel.  Rows from n on are neither read nor written.
constexpr int TR_THREADS = 448;
constexpr int TR_A_OFF = 0;                                    // 6 A planes of 128 x 64 BF16
constexpr int TR_B_OFF = OZ_NSL * OZ_A_BYTES;                  // 2 halves x 6 planes of 32 x 64 BF16
constexpr int TR_NSS = 3;                                      // staging ring of A21 boxes (128 x 16 pairs)
constexpr int TR_S_OFF = TR_B_OFF + 2 * OZ_B_BYTES;
constexpr int TR_BAR_OFF = TR_S_OFF + TR_NSS * OZ_CBOX_BYTES;
constexpr int TR_SMEM = 1024 + TR_BAR_OFF + 256;
static_assert(TR_SMEM <= 227 * 1024, "shared memory of the TRSM kernel");

struct TrParams {
  const TrItem* items;          // this panel's tiles, grouped by block
  int n_items;
  const CUtensorMap* mmap;      // 64 x 32 boxes over the Minv planes (6 x 64 rows per block)
  const CUtensorMap* cmaps;     // per bin [2 bin]: 16 x 128 boxes over the pool of pairs
  double* pool;                 // factor in double-float pairs (8 bytes an entry)
  const int32_t* scale_exp;     // e_r per row (row_off indexing)
  const int32_t* mf;            // per block: f_0 .. f_63, g
  __nv_bfloat16* planes;        // slices of L21 for the trailing update
  float* l32;                   // the factor's FP32 rounding fl(h + l) (same layout as the pool)
  int c0;
  DevFlags* flags;
  long long budget;
};

__global__ void __launch_bounds__(TR_THREADS, 1) chol_trsm_tc_kernel(const __grid_constant__ TrParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + TR_BAR_OFF);
  uint64_t* bfull_bar = bars;          // Minv planes landed
  uint64_t* bempty_bar = bars + 1;     // the MMAs on the previous block's planes are done
  uint64_t* afull_bar = bars + 2;      // the converter wrote the item's A planes
  uint64_t* aempty_bar = bars + 3;     // the MMAs on the A planes are done
  uint64_t* tfull_bar = bars + 4;      // both accumulator sets hold the item's levels
  uint64_t* tempty_bar = bars + 5;     // the epilogue has read them
  uint64_t* drain_bar = bars + 6;
  uint64_t* sfull_bar = bars + 7;      // [TR_NSS] an A21 box landed in the staging ring
  uint64_t* sempty_bar = bars + 7 + TR_NSS;   // [TR_NSS] the converter has read it
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 7 + 2 * TR_NSS);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // contiguous run of the item list (consecutive items of one block reuse its Minv planes)
  const int first = (int)(((int64_t)p.n_items * blockIdx.x) / gridDim.x);
  const int last = (int)(((int64_t)p.n_items * (blockIdx.x + 1)) / gridDim.x);
  if (threadIdx.x == 0) {
    mbar_init(bfull_bar, 1);
    mbar_init(bempty_bar, 1);
    mbar_init(afull_bar, 128);
    mbar_init(aempty_bar, 1);
    mbar_init(tfull_bar, 1);
    mbar_init(tempty_bar, 256);
    mbar_init(drain_bar, 1);
    for (int i = 0; i < TR_NSS; ++i) {
      mbar_init(&sfull_bar[i], 1);
      mbar_init(&sempty_bar[i], 128);
    }
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
  const long long drain_budget = budget > (1LL << 22) ? budget : (1LL << 22);
  const int c0 = p.c0;

  if (warp == 0) {
    // ------------------------------------------------------------ producer: Minv planes per block,
    // the item's A21 pairs as four 128 x 16 boxes through the staging ring
    if (lane == 0) {
      int cur = -1, ps = 0;
      uint32_t bph = 0, pph = 0;
      bool armed = false, ok = true;
      uint32_t arm_parity = 0, sarmed = 0, sarm_parity = 0;
      for (int it = first; it < last && ok; ++it) {
        const TrItem ti = p.items[it];
        const int b = ti.b;
        if (b != cur) {
          cur = b;
          if (!mbar_wait(bempty_bar, bph ^ 1u, budget, abort_flag)) { ok = false; break; }
          mbar_expect_tx(bfull_bar, 2 * OZ_B_BYTES);
          for (int h = 0; h < 2; ++h)
            for (int t = 0; t < OZ_NSL; ++t)
              tma_load_2d(smem + TR_B_OFF + h * OZ_B_BYTES + t * OZ_PLANE_B, p.mmap, bfull_bar, 0,
                          (b * OZ_NSL + t) * 64 + 32 * h);
          armed = true;
          arm_parity = bph;
          bph ^= 1u;
        }
        const CUtensorMap* cmap = p.cmaps + 2 * ti.bin;
        for (int box = 0; box < 4; ++box) {
          if (!mbar_wait(&sempty_bar[ps], pph ^ 1u, budget, abort_flag)) { ok = false; break; }
          mbar_expect_tx(&sfull_bar[ps], OZ_CBOX_BYTES);
          tma_load_2d(smem + TR_S_OFF + ps * OZ_CBOX_BYTES, cmap, &sfull_bar[ps], c0 + 16 * box, ti.pos * ti.ld + ti.m0);
          sarmed |= 1u << ps;
          sarm_parity = (sarm_parity & ~(1u << ps)) | (pph << ps);
          if (++ps == TR_NSS) { ps = 0; pph ^= 1u; }
        }
      }
      if (!ok) {
        set_error(p.flags, NOLSM_ETIMEOUT);
        *abort_flag = 1;
      }
      volatile int never = 0;
      if (armed) mbar_wait(bfull_bar, arm_parity, drain_budget, &never);
      for (int i = 0; i < TR_NSS; ++i)
        if (sarmed & (1u << i)) mbar_wait(&sfull_bar[i], (sarm_parity >> i) & 1u, drain_budget, &never);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int cur = -1;
      uint32_t bph = 0, aph = 0, tph = 0;
      bool ok = true;
      for (int it = first; it < last && ok; ++it) {
        const int b = p.items[it].b;
        if (b != cur) {
          if (cur >= 0) umma_commit(bempty_bar);   // the previous block's planes are free once its MMAs are done
          cur = b;
          if (!mbar_wait(bfull_bar, bph, budget, abort_flag)) { ok = false; break; }
          bph ^= 1u;
        }
        if (!mbar_wait(afull_bar, aph, budget, abort_flag) || !mbar_wait(tempty_bar, tph ^ 1u, budget, abort_flag)) {
          ok = false;
          break;
        }
        aph ^= 1u;
        tc_fence_after();
        for (int h = 0; h < 2; ++h) {
          const uint64_t bdesc = sw128_desc(smem_u32(smem + TR_B_OFF + h * OZ_B_BYTES));
          for (int s = 0; s < OZ_NSL; ++s) {
            const uint64_t adesc = sw128_desc(smem_u32(smem + TR_A_OFF + s * OZ_A_BYTES));
            const uint32_t idesc = make_idesc(1, TM, OZ_TN * (OZ_NSL - s));
            const uint32_t d = tmem_base + (uint32_t)(h * OZ_ACC + s * OZ_TN);
#pragma unroll
            for (int kk = 0; kk < kOzPanel / 16; ++kk)
              umma_f16(d, adesc + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), idesc, (s | kk) != 0);
          }
        }
        umma_commit(aempty_bar);
        umma_commit(tfull_bar);
        tph ^= 1u;
      }
      if (!ok) {
        set_error(p.flags, NOLSM_ETIMEOUT);
        *abort_flag = 1;
      }
      umma_commit(drain_bar);
      volatile int never = 0;
      mbar_wait(drain_bar, 0, drain_budget, &never);
    }
  } else if (warp < 6) {
    // ------------------------------------------------------------ converter: A21 pairs -> 6 A planes
    // (thread = row of the tile; per staged box its 16 pairs, two 16-byte units of every plane)
    const int ct = threadIdx.x - 64;   // 0..127
    uint32_t aph = 0, sph = 0;
    int ss = 0;
    bool ok = true;
    // the next item's record is loaded one item ahead (no dependent load waits at the item's start)
    TrItem nx = first < last ? p.items[first] : TrItem{};
    for (int it = first; it < last && ok; ++it) {
      const TrItem ti = nx;
      if (it + 1 < last) nx = p.items[it + 1];
      const int r = ti.m0 + ct;
      const bool live = r < ti.n;
      const float esc = oz_scale(live ? p.scale_exp[ti.row_off + r] + p.mf[(int64_t)ti.b * 68 + 64] : 0);
      if (!mbar_wait(aempty_bar, aph ^ 1u, budget, abort_flag)) { ok = false; break; }
      aph ^= 1u;
      for (int box = 0; box < 4; ++box) {
        if (!mbar_wait(&sfull_bar[ss], sph, budget, abort_flag)) { ok = false; break; }
        const uint8_t* st = smem + TR_S_OFF + ss * OZ_CBOX_BYTES;
        float f[32];
#pragma unroll
        for (int w = 0; w < 8; ++w) {
          const float4 x = live ? *reinterpret_cast<const float4*>(st + sw128(ct, 16 * w)) : make_float4(0.f, 0.f, 0.f, 0.f);
          f[4 * w] = x.x;
          f[4 * w + 1] = x.y;
          f[4 * w + 2] = x.z;
          f[4 * w + 3] = x.w;
        }
        // the next tensor copy into this slot (async proxy) must not overtake these generic reads
        fence_async_smem();
        mbar_arrive(&sempty_bar[ss]);
        if (++ss == TR_NSS) { ss = 0; sph ^= 1u; }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          uint32_t pk[OZ_NSL][4];
#pragma unroll
          for (int x = 0; x < 8; x += 2) {
            float q0[OZ_NSL], q1[OZ_NSL];
            oz_slices(f[16 * u + 2 * x], f[16 * u + 2 * x + 1], esc, q0);
            oz_slices(f[16 * u + 2 * x + 2], f[16 * u + 2 * x + 3], esc, q1);
#pragma unroll
            for (int sl = 0; sl < OZ_NSL; ++sl) pk[sl][x >> 1] = Pack<__nv_bfloat16>::two(q0[sl], q1[sl]);
          }
#pragma unroll
          for (int sl = 0; sl < OZ_NSL; ++sl)
            *reinterpret_cast<uint4*>(smem + TR_A_OFF + sl * OZ_A_BYTES + sw128(ct, 16 * (2 * box + u))) =
                make_uint4(pk[sl][0], pk[sl][1], pk[sl][2], pk[sl][3]);
        }
      }
      if (!ok) break;
      fence_async_smem();
      mbar_arrive(afull_bar);
    }
    if (!ok) {
      set_error(p.flags, NOLSM_ETIMEOUT);
      *abort_flag = 1;
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3, h = (warp - 6) >> 2;   // a warp reads the TMEM lanes of quarter warp % 4
    uint32_t tph = 0;
    // the next item's record is loaded one item ahead; the exponents it points to are loaded before
    // the wait for the accumulators, so that neither load chain stalls the epilogue
    TrItem nx = first < last ? p.items[first] : TrItem{};
    for (int it = first; it < last; ++it) {
      const TrItem ti = nx;
      if (it + 1 < last) nx = p.items[it + 1];
      const int n = ti.n, ld = ti.ld;
      const int r = ti.m0 + q * 32 + lane;
      const int32_t* F = p.mf + (int64_t)ti.b * 68;
      const int er = r < n ? p.scale_exp[ti.row_off + r] : 0;
      const int g = F[64];
      const int fl = F[32 * h + lane];            // f_c of this half's column lane, shared by shuffles
      if (!__all_sync(0xffffffffu, mbar_wait(tfull_bar, tph, budget, abort_flag))) {
        set_error(p.flags, NOLSM_ETIMEOUT);
        *abort_flag = 1;
        break;
      }
      tph ^= 1u;
      tc_fence_after();
      const int eg = er + g - 2 * kOzBits;
      const float rsc = oz_scale(er);
      float2* Lrow = reinterpret_cast<float2*>(p.pool + ti.off_mat) + (int64_t)r * ld + c0;
      float* L32row = p.l32 + ti.off_mat + (int64_t)r * ld + c0;
      __nv_bfloat16* P = p.planes + ((int64_t)OZ_NSL * ti.row_off + r) * 64;
      for (int j = 0; j < 4; ++j) {
        const int cb = 32 * h + 8 * j;            // first of this chunk's 8 columns of the panel
        uint32_t v[OZ_NSL][8];
        const uint32_t tb = tmem_base + (uint32_t)(h * OZ_ACC + 8 * j) + ((uint32_t)(q * 32) << 16);
#pragma unroll
        for (int l = 0; l < OZ_NSL; ++l) tmem_ld8(tb + (uint32_t)(l * OZ_TN), v[l]);
        tmem_wait_ld();
        int fc[8];                                // every lane takes part in the shuffles
#pragma unroll
        for (int x = 0; x < 8; ++x) fc[x] = __shfl_sync(0xffffffffu, fl, 8 * j + x);
        if (r >= n) continue;
        float out[16];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          // sum_l v_l 2^(-8 l) in double-float, smallest level first (every term is exact)
          float hi = __uint_as_float(v[OZ_NSL - 1][x]) * 0x1p-40f, lo = 0.f;
#pragma unroll
          for (int l = OZ_NSL - 2; l >= 0; --l) {
            const float y = __uint_as_float(v[l][x]) * __int_as_float((127 - kOzBits * l) << 23);
            const float s = hi + y;
            const float bb = s - hi;
            lo += (hi - (s - bb)) + (y - bb);
            hi = s;
          }
          const float sc = __int_as_float((127 + eg + fc[x]) << 23);
          hi *= sc;
          lo *= sc;
          const float s = hi + lo;                // renormalised pair
          const float bb = s - hi;
          out[2 * x] = s;
          out[2 * x + 1] = (hi - (s - bb)) + (lo - bb);
        }
#pragma unroll
        for (int w = 0; w < 4; ++w)
          reinterpret_cast<float4*>(Lrow + cb)[w] = make_float4(out[4 * w], out[4 * w + 1], out[4 * w + 2], out[4 * w + 3]);
#pragma unroll
        for (int w = 0; w < 2; ++w)
          reinterpret_cast<float4*>(L32row + cb)[w] =
              make_float4(out[8 * w] + out[8 * w + 1], out[8 * w + 2] + out[8 * w + 3], out[8 * w + 4] + out[8 * w + 5],
                          out[8 * w + 6] + out[8 * w + 7]);
        // slices of the row on its own scale for the trailing update: plane s, row r, columns cb ..
        uint32_t pk[OZ_NSL][4];
#pragma unroll
        for (int x = 0; x < 8; x += 2) {
          float q0[OZ_NSL], q1[OZ_NSL];
          oz_slices(out[2 * x], out[2 * x + 1], rsc, q0);
          oz_slices(out[2 * x + 2], out[2 * x + 3], rsc, q1);
#pragma unroll
          for (int sl = 0; sl < OZ_NSL; ++sl) pk[sl][x >> 1] = Pack<__nv_bfloat16>::two(q0[sl], q1[sl]);
        }
#pragma unroll
        for (int sl = 0; sl < OZ_NSL; ++sl)
          *reinterpret_cast<uint4*>(P + (int64_t)sl * ld * 64 + cb) = make_uint4(pk[sl][0], pk[sl][1], pk[sl][2], pk[sl][3]);
      }
      tc_fence_before();
      mbar_arrive(tempty_bar);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

// ---------------------------------------------------------------------------------------------
// The congruence A0 = L^-1 T_b(H0) L^-T on the tensor cores, FP32-accurate by three TF32 passes.
// A product C = A B^T (both operands row-major, K contiguous) over a tile list of 128 x 128 tiles.
// Each FP32 operand x is split in shared memory into hi = x rounded to TF32 (exact in TF32) and
// lo = x - hi (exact in FP32, read as TF32), and every k-step accumulates lo_A hi_B + hi_A lo_B +
// hi_A hi_B in FP32 tensor memory.  lo keeps 11 bits and lo_A lo_B is dropped, so a product term
// carries about 2^-21 relative error, ten times FP32's: A0 lands within ~3e-6 of the FP32 result,
// far below the FP16 rounding of X_0 that the mixed paths apply next (the FP32 path keeps the SIMT
// products).
// Roles (320 threads): warp 0 TMA producer (raw 128 x 32 FP32 boxes, 128-byte swizzle), warp 1 MMA
// issuer (kind::tf32, M = N = 128, K = 8), warps 2..5 split each stage in place (hi over the raw box,
// lo beside it), warps 6..9 epilogue (TMEM -> registers -> staged 32 x 32 FP32 chunks -> tensor
// stores; with sym, tiles on or above the diagonal only, each chunk stored twice so that the output
// is exactly symmetric).  Waits are bounded as in ns_tc_kernel.
constexpr int CG_TN = 128;
constexpr int CG_TK = 32;                                   // FP32 elements per 128-byte row
constexpr int CG_STAGES = 3;
constexpr int CG_BOX_BYTES = 128 * CG_TK * 4;               // 16 KB
constexpr int CG_STAGE_BYTES = 4 * CG_BOX_BYTES;            // A hi, B hi, A lo, B lo
constexpr int CG_EPI_OFF = CG_STAGES * CG_STAGE_BYTES;
constexpr int CG_EPI_WARP_BYTES = 8192;                     // a 32 x 32 FP32 chunk and its transpose
constexpr int CG_BAR_OFF = CG_EPI_OFF + 4 * CG_EPI_WARP_BYTES;
constexpr int CG_SMEM = 1024 + CG_BAR_OFF + 256;
constexpr int CG_THREADS = 320;
constexpr int CG_TMEM_COLS = 256;                           // two 128-column accumulators
static_assert(CG_SMEM <= 227 * 1024, "shared memory of the congruence kernel");

constexpr int CG_POOLS = 5;  // 0 L^-1, 1 A0 pool, 2 T1 (Y = X^T during the inverse), 3 L (FP32), 4 R^T scratch
struct CgParams {
  const Tile* tiles;
  const int32_t* kbeg;        // first K of each tile (NULL: 0)
  int n_tiles;
  const BlockDesc* blocks;
  const CUtensorMap* tmaps;   // per bin: loads of the CG_POOLS pools, then stores into them
  int map_a, map_b, map_c;    // pools of A, B and the output
  int map_t;                  // pool that also receives the transposed output (-1: none)
  int neg;                    // store -C
  int sym;
  int interleave;             // 1: tile i to CTA i mod grid (large blocks); 0: contiguous runs
  float* out_pool;
  DevFlags* flags;
  long long budget;
};

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}


__global__ void __launch_bounds__(CG_THREADS, 1) cong_tc_kernel(const __grid_constant__ CgParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + CG_BAR_OFF);
  uint64_t* full_bar = bars;                       // [CG_STAGES] TMA landed
  uint64_t* conv_bar = bars + CG_STAGES;           // [STAGES] split done
  uint64_t* empty_bar = bars + 2 * CG_STAGES;      // [STAGES] MMA done with the stage
  uint64_t* tfull_bar = bars + 3 * CG_STAGES;      // [2]
  uint64_t* tempty_bar = bars + 3 * CG_STAGES + 2; // [2]
  uint64_t* drain_bar = bars + 3 * CG_STAGES + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * CG_STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // contiguous runs of the tile list per CTA for small blocks (each SM walks whole blocks); tiles
  // dealt round-robin for large ones, so that all SMs share a few blocks' operands in L2
  const int span = p.n_tiles;
  const int first = p.interleave ? (int)blockIdx.x : (int)(((int64_t)span * blockIdx.x) / gridDim.x);
  const int step = p.interleave ? (int)gridDim.x : 1;
  const int n_local = p.interleave ? (span > (int)blockIdx.x ? (span - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0)
                                   : (int)(((int64_t)span * (blockIdx.x + 1)) / gridDim.x) - first;
  if (threadIdx.x == 0) {
    for (int s = 0; s < CG_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&conv_bar[s], 128);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) { mbar_init(&tfull_bar[a], 1); mbar_init(&tempty_bar[a], 128); }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(CG_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const long long budget = p.budget;
  const long long drain_budget = budget > (1LL << 22) ? budget : (1LL << 22);
  uint32_t armed = 0, arm_parity = 0;

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int i = 0; i < n_local && ok; ++i) {
        const Tile tl = p.tiles[first + i * step];
        const BlockDesc bd = p.blocks[tl.block];
        const CUtensorMap* ma = p.tmaps + bd.bin * 2 * CG_POOLS + p.map_a;
        const CUtensorMap* mb = p.tmaps + bd.bin * 2 * CG_POOLS + p.map_b;
        const int rowbase = bd.pos * bd.n_pad;
        const int kb = p.kbeg ? p.kbeg[first + i * step] : 0;
        for (int k0 = kb; k0 < tl.kend; k0 += CG_TK) {
          if (!mbar_wait(&empty_bar[s], ph ^ 1u, budget, abort_flag)) { ok = false; break; }
          mbar_expect_tx(&full_bar[s], 2 * CG_BOX_BYTES);
          uint8_t* st = smem + s * CG_STAGE_BYTES;
          tma_load_2d(st, ma, &full_bar[s], k0, rowbase + tl.m0);
          tma_load_2d(st + CG_BOX_BYTES, mb, &full_bar[s], k0, rowbase + tl.n0);
          armed |= 1u << s;
          arm_parity = (arm_parity & ~(1u << s)) | (ph << s);
          if (++s == CG_STAGES) { s = 0; ph ^= 1u; }
        }
      }
      if (!ok) {
        set_error(p.flags, NOLSM_ETIMEOUT);
        *abort_flag = 1;
      }
      volatile int never = 0;
      for (int st = 0; st < CG_STAGES; ++st)
        if (armed & (1u << st)) mbar_wait(&full_bar[st], (arm_parity >> st) & 1u, drain_budget, &never);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0, tph[2] = {0u, 0u};
      int acc = 0;
      bool ok = true;
      // kind::tf32: FP32 accumulator (bit 4), A and B TF32 (format 2), both K-major, N >> 3, M >> 4
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(CG_TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
      for (int i = 0; i < n_local && ok; ++i) {
        const Tile tl = p.tiles[first + i * step];
        if (!mbar_wait(&tempty_bar[acc], tph[acc] ^ 1u, budget, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * CG_TN);
        const int kb = p.kbeg ? p.kbeg[first + i * step] : 0;
        for (int k0 = kb; k0 < tl.kend; k0 += CG_TK) {
          if (!mbar_wait(&conv_bar[s], ph, budget, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t base = smem_u32(smem + s * CG_STAGE_BYTES);
          const uint64_t ah = sw128_desc(base), bh = sw128_desc(base + CG_BOX_BYTES);
          const uint64_t al = sw128_desc(base + 2 * CG_BOX_BYTES), bl = sw128_desc(base + 3 * CG_BOX_BYTES);
#pragma unroll
          for (int kk = 0; kk < CG_TK / 8; ++kk) {
            const uint64_t o = (uint64_t)(kk * 2);   // 8 FP32 = 32 bytes along K inside the swizzle atom
            umma_tf32(d_tmem, al + o, bh + o, idesc, (k0 != kb || kk != 0) ? 1u : 0u);
            umma_tf32(d_tmem, ah + o, bl + o, idesc, 1u);
            umma_tf32(d_tmem, ah + o, bh + o, idesc, 1u);
          }
          umma_commit(&empty_bar[s]);
          if (++s == CG_STAGES) { s = 0; ph ^= 1u; }
        }
        if (!ok) break;
        umma_commit(&tfull_bar[acc]);
        tph[acc] ^= 1u;
        acc ^= 1;
      }
      if (!ok) {
        set_error(p.flags, NOLSM_ETIMEOUT);
        *abort_flag = 1;
      }
      umma_commit(drain_bar);
      volatile int never = 0;
      mbar_wait(drain_bar, 0, drain_budget, &never);
    }
  } else if (warp < 6) {
    // ------------------------------------------------------------------ split: hi in place, lo beside it
    const int ct = threadIdx.x - 64;            // 0..127
    int s = 0;
    uint32_t ph = 0;
    for (int i = 0; i < n_local; ++i) {
      const Tile tl = p.tiles[first + i * step];
      const int kb = p.kbeg ? p.kbeg[first + i * step] : 0;
      bool ok = true;
      for (int k0 = kb; k0 < tl.kend; k0 += CG_TK) {
        if (!mbar_wait(&full_bar[s], ph, budget, abort_flag)) { ok = false; break; }
        uint8_t* st = smem + s * CG_STAGE_BYTES;
        // 2 boxes x 16 KB = 2048 float4; 16 per thread (position-wise, so the swizzle is irrelevant)
#pragma unroll 4
        for (int j = 0; j < 16; ++j) {
          const int e = ct + 128 * j;           // float4 index over A hi (0..1023) then B hi (1024..2047)
          float4* hp = reinterpret_cast<float4*>(st) + e;
          float4* lp = reinterpret_cast<float4*>(st + 2 * CG_BOX_BYTES) + e;
          const float4 x = *hp;
          // hi: x rounded to the nearest TF32 (add half of the dropped range, clear it), exact in TF32
          float4 h, l;
          h.x = __uint_as_float((__float_as_uint(x.x) + 0x1000u) & 0xFFFFE000u); l.x = x.x - h.x;
          h.y = __uint_as_float((__float_as_uint(x.y) + 0x1000u) & 0xFFFFE000u); l.y = x.y - h.y;
          h.z = __uint_as_float((__float_as_uint(x.z) + 0x1000u) & 0xFFFFE000u); l.z = x.z - h.z;
          h.w = __uint_as_float((__float_as_uint(x.w) + 0x1000u) & 0xFFFFE000u); l.w = x.w - h.w;
          *hp = h;
          *lp = l;
        }
        fence_async_smem();
        mbar_arrive(&conv_bar[s]);
        if (++s == CG_STAGES) { s = 0; ph ^= 1u; }
      }
      if (!ok) {
        set_error(p.flags, NOLSM_ETIMEOUT);
        *abort_flag = 1;
        break;
      }
    }
  } else {
    // ------------------------------------------------------------------ epilogue (warps 6..9)
    const int q = warp & 3;
    uint8_t* stage = smem + CG_EPI_OFF + (warp - 6) * CG_EPI_WARP_BYTES;
    uint32_t tph[2] = {0u, 0u};
    int acc = 0;
    for (int i = 0; i < n_local; ++i) {
      const Tile tl = p.tiles[first + i * step];
      const BlockDesc bd = p.blocks[tl.block];
      if (!__all_sync(0xffffffffu, mbar_wait(&tfull_bar[acc], tph[acc], budget, abort_flag))) {
        set_error(p.flags, NOLSM_ETIMEOUT);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const int ld = bd.n_pad, rowbase = bd.pos * ld;
      const CUtensorMap* smap = p.tmaps + bd.bin * 2 * CG_POOLS + CG_POOLS + p.map_c;
      const bool mir = p.sym || p.map_t >= 0;   // the transposed chunk is stored too
      const CUtensorMap* tmap = p.sym ? smap : p.tmaps + bd.bin * 2 * CG_POOLS + CG_POOLS + (p.map_t < 0 ? 0 : p.map_t);
      const uint32_t sgn = p.neg ? 0x80000000u : 0u;
      float* out = p.out_pool + bd.off_mat;
      const int r0 = tl.m0 + q * 32, r = r0 + lane;
      for (int c0 = 0; c0 < CG_TN; c0 += 32) {
        const int cg0 = tl.n0 + c0;
        uint32_t v[32];
        tmem_ld32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * CG_TN + c0), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] ^= sgn;
        if (p.sym && cg0 < r0) continue;        // below the diagonal: the mirror of another chunk
        if (p.sym && cg0 == r0) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float x = __uint_as_float(v[j]);
            if (cg0 + j >= r) out[(int64_t)r * ld + cg0 + j] = x;
            if (cg0 + j > r) out[(int64_t)(cg0 + j) * ld + r] = x;
          }
          continue;
        }
        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        __syncwarp();
        uint8_t* D = stage;
        uint8_t* M = stage + 4096;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          *reinterpret_cast<uint4*>(D + sw128(lane, 16 * u)) = make_uint4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
        if (mir) {
#pragma unroll
          for (int j = 0; j < 32; ++j) *reinterpret_cast<uint32_t*>(M + sw128(j, 4 * lane)) = v[j];
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          tma_store_2d(smap, D, cg0, rowbase + r0);
          if (mir) tma_store_2d(tmap, M, r0, rowbase + cg0);
          bulk_commit();
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty_bar[acc]);
      tph[acc] ^= 1u;
      acc ^= 1;
    }
    if (lane == 0) bulk_wait0();
    __syncwarp();
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(CG_TMEM_COLS) : "memory");
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
  std::vector<int64_t> bin_off(n_bins, -1), bin_cnt(n_bins, 0), bin_slab(n_bins, 0), bin_rows(n_bins, 0);
  std::vector<int> bin_pad(n_bins, 0);
  for (const auto& b : ctx->h_blocks) {
    if (b.pos == 0) {
      bin_off[b.bin] = b.off_mat;
      bin_slab[b.bin] = b.off_slab;
    }
    bin_cnt[b.bin] += 1;
    bin_rows[b.bin] += b.c;
    bin_pad[b.bin] = b.n_pad;
  }
  maps.resize((size_t)n_bins * kMapsPerBin);
  void* pools[3] = {ctx->d_x[0], ctx->d_x[1], ctx->d_b};
  const CUtensorMapDataType dt = bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  for (int bi = 0; bi < n_bins; ++bi) {
    for (int pi = 0; pi < 3; ++pi) {
      const uint64_t np = (uint64_t)bin_pad[bi];
      void* base = reinterpret_cast<uint8_t*>(pools[pi]) + bin_off[bi] * 2;
      cuuint64_t gdim[2] = {np, np * (uint64_t)bin_cnt[bi]};
      cuuint64_t gstride[1] = {np * 2};
      cuuint32_t estr[2] = {1, 1};
      // operand loads: 64 x 128 boxes, 128-byte swizzle (the MMA's K-major layout)
      cuuint32_t box[2] = {TK, TM};
      CUresult r = encode(&maps[(size_t)bi * kMapsPerBin + pi], dt, 2, base, gdim, gstride, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
      // epilogue stores: 32 x 32 boxes, 64-byte swizzle (the staging layout of epi_tile)
      cuuint32_t sbox[2] = {32, 32};
      r = encode(&maps[(size_t)bi * kMapsPerBin + 3 + pi], dt, 2, base, gdim, gstride, sbox, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    // the refinement's split slab pools (in the slab scratch after two FP32 slabs): each bin's slabs
    // are a stack of c-row, n_pad-column matrices; 64 x 16 boxes, 128-byte swizzle
    for (int pi = 0; pi < 4; ++pi) {
      const uint64_t np = (uint64_t)bin_pad[bi];
      void* base = reinterpret_cast<uint8_t*>(ctx->d_tmp + 2 * ctx->sum_slab) + 2 * (pi * ctx->sum_slab + bin_slab[bi]);
      cuuint64_t gdim[2] = {np, (uint64_t)std::max<int64_t>(bin_rows[bi], 1)};
      cuuint64_t gstride[1] = {np * 2};
      cuuint32_t estr[2] = {1, 1};
      cuuint32_t box[2] = {TK, 16};
      CUresult r = encode(&maps[(size_t)bi * kMapsPerBin + 6 + pi], dt, 2, base, gdim, gstride, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
  }
  // the device copy keeps its allocation across builds (it only grows), and the upload's source lives
  // in the context until the next build, so a build neither frees nor waits here
  cudaError_t e = cudaSuccess;
  if (ctx->tmap_cap < maps.size()) {
    if (ctx->d_tmaps) cudaFree(ctx->d_tmaps);
    ctx->d_tmaps = nullptr;
    ctx->tmap_cap = 0;
    e = cudaMalloc(&ctx->d_tmaps, maps.size() * sizeof(CUtensorMap));
    if (e != cudaSuccess) return e;
    ctx->tmap_cap = maps.size();
  }
  ctx->n_tmaps = (int)maps.size();
  ctx->h_tc_maps.assign(reinterpret_cast<const uint8_t*>(maps.data()),
                        reinterpret_cast<const uint8_t*>(maps.data() + maps.size()));
  e = cudaMemcpyAsync(ctx->d_tmaps, ctx->h_tc_maps.data(), ctx->h_tc_maps.size(), cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return e;
  static bool attr_done = false;
  if (!attr_done) {
    e = cudaFuncSetAttribute(ns_tc_kernel<__half, 4, 4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcNarrow::smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ns_tc_kernel<__nv_bfloat16, 4, 4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TcNarrow::smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ns_tc_kernel<__half, 3, 8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcWide::smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ns_tc_kernel<__nv_bfloat16, 3, 8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TcWide::smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ns_pair_kernel<__half, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, PAIR_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ns_pair_kernel<__nv_bfloat16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             PAIR_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ns_pair_kernel<__half, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, PAIR_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ns_pair_kernel<__nv_bfloat16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             PAIR_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ns_pair2_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, PAIR2_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ns_pair2_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, PAIR2_SMEM);
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
  int max_pad = 0;
  for (const auto& bd : ctx->h_blocks) max_pad = std::max(max_pad, bd.n_pad);
  p.interleave = max_pad >= 1024;
  const int grid = ctx->num_sms;
  // each CTA resolves at most MAX_LOCAL tiles per launch; cover the largest possible list
  const int64_t per_launch = (int64_t)MAX_LOCAL * grid;
  for (int64_t base = 0; base < std::max<int64_t>(ctx->max_tiles_tc, 1); base += per_launch) {
    p.tile_base = (int)base;
    // large blocks (long K loops, 128 x 256 tiles back to back): the shape with two double-buffered
    // epilogue warps per lane quarter keeps the epilogue of a tile within the next tile's products
    const bool bf = ctx->opt.precision == NOLSM_PREC_MIXED_BF16;
    if (p.interleave) {
      if (bf) ns_tc_kernel<__nv_bfloat16, 3, 8, 2><<<grid, TcWide::threads, TcWide::smem, ctx->stream>>>(p);
      else ns_tc_kernel<__half, 3, 8, 2><<<grid, TcWide::threads, TcWide::smem, ctx->stream>>>(p);
    } else {
      if (bf) ns_tc_kernel<__nv_bfloat16, 4, 4, 1><<<grid, TcNarrow::threads, TcNarrow::smem, ctx->stream>>>(p);
      else ns_tc_kernel<__half, 4, 4, 1><<<grid, TcNarrow::threads, TcNarrow::smem, ctx->stream>>>(p);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Tensor maps of the 3 x TF32 product kernel, per bin over the FP32 pools L^-1, A0, T1, L (the
// factor's FP32 rounding) and the R^T scratch (loads: 128 x 32 boxes, stores: 32 x 32 boxes).  L and
// the scratch lie in the second half of the build's FP64 scratch (sb + sum_sq).
cudaError_t cg_maps(nolsm_ctx* ctx, float* t1) {
  if (ctx->cg_maps_gen == ctx->build_gen && ctx->cg_maps_t1 == t1) return cudaSuccess;   // encoded for this build
  auto encode = get_encode();
  if (!encode) return cudaErrorNotSupported;
  int n_bins = 0;
  for (const auto& b : ctx->h_blocks) n_bins = std::max(n_bins, b.bin + 1);
  std::vector<int64_t> bin_off(n_bins, -1), bin_cnt(n_bins, 0);
  std::vector<int> bin_pad(n_bins, 0);
  for (const auto& b : ctx->h_blocks) {
    if (b.pos == 0) bin_off[b.bin] = b.off_mat;
    bin_cnt[b.bin] += 1;
    bin_pad[b.bin] = b.n_pad;
  }
  std::vector<CUtensorMap> maps((size_t)n_bins * 2 * CG_POOLS);
  float* l32 = reinterpret_cast<float*>(ctx->d_sb + ctx->sum_sq);
  float* pools[CG_POOLS] = {ctx->d_linv, ctx->d_a0, t1, l32, l32 + ctx->sum_sq};
  for (int bi = 0; bi < n_bins; ++bi)
    for (int pi = 0; pi < CG_POOLS; ++pi) {
      const uint64_t np = (uint64_t)bin_pad[bi];
      void* base = pools[pi] + bin_off[bi];
      cuuint64_t gdim[2] = {np, np * (uint64_t)bin_cnt[bi]};
      cuuint64_t gstride[1] = {np * 4};
      cuuint32_t estr[2] = {1, 1};
      cuuint32_t box[2] = {CG_TK, TM};
      CUresult r = encode(&maps[(size_t)bi * 2 * CG_POOLS + pi], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, gdim, gstride,
                          box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
      cuuint32_t sbox[2] = {32, 32};
      r = encode(&maps[(size_t)bi * 2 * CG_POOLS + CG_POOLS + pi], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, gdim,
                 gstride, sbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                 CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
  if (ctx->cg_tmap_cap < maps.size()) {
    if (ctx->d_cg_tmaps) cudaFree(ctx->d_cg_tmaps);
    ctx->d_cg_tmaps = nullptr;
    cudaError_t e = cudaMalloc(&ctx->d_cg_tmaps, maps.size() * sizeof(CUtensorMap));
    if (e != cudaSuccess) return e;
    ctx->cg_tmap_cap = maps.size();
  }
  // one encode per build (both callers pass the build's T1 pool); the upload's source lives in the
  // context until the next build
  ctx->h_cg_maps.assign(reinterpret_cast<const uint8_t*>(maps.data()),
                        reinterpret_cast<const uint8_t*>(maps.data() + maps.size()));
  cudaError_t e = cudaMemcpyAsync(ctx->d_cg_tmaps, ctx->h_cg_maps.data(), ctx->h_cg_maps.size(),
                                  cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return e;
  static bool attr_done = false;
  if (!attr_done) {
    e = cudaFuncSetAttribute(cong_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, CG_SMEM);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  ctx->cg_maps_gen = ctx->build_gen;
  ctx->cg_maps_t1 = t1;
  return cudaSuccess;
}

CgParams cg_params(nolsm_ctx* ctx, const Tile* tiles, const int32_t* kbeg, int n_tiles, int a, int b, int c, int t,
                   int neg, int sym, float* out) {
  int max_pad = 0;
  for (const auto& bd : ctx->h_blocks) max_pad = std::max(max_pad, bd.n_pad);
  CgParams p;
  p.tiles = tiles;
  p.kbeg = kbeg;
  p.n_tiles = n_tiles;
  p.blocks = ctx->d_blocks;
  p.tmaps = reinterpret_cast<const CUtensorMap*>(ctx->d_cg_tmaps);
  p.map_a = a;
  p.map_b = b;
  p.map_c = c;
  p.map_t = t;
  p.neg = neg;
  p.sym = sym;
  p.interleave = max_pad >= 1024;
  p.out_pool = out;
  p.flags = ctx->d_flags;
  p.budget = ctx->opt.wait_budget;
  return p;
}

// The tile lists of the build's tensor-core products in one device list, made and uploaded only when
// the block layout differs from the one they were made for (a rebuild of the same system neither
// uploads nor waits on the stream):
//   launch 0: congruence pass 0, T1 = L^-1 T_b(H0): all tiles; L^-1 is lower triangular, so a tile's
//             K stops at m0 + 128;
//   launch 1: congruence pass 1, A0 = T1 L^-T: tiles on or above the diagonal, K stops at n0 + 128;
//   launches 2, 3, ...: the tiled inverse, two per block row i >= 1 (launch_trinv_tc).
static cudaError_t build_tile_lists(nolsm_ctx* ctx) {
  const size_t nbk = ctx->h_blocks.size();
  if (ctx->bt_dev == ctx->d_bt && ctx->bt_kdev == ctx->d_cg_kbeg && ctx->d_bt && ctx->bt_layout.size() == nbk &&
      std::memcmp(ctx->bt_layout.data(), ctx->h_blocks.data(), nbk * sizeof(BlockDesc)) == 0)
    return cudaSuccess;
  std::vector<Tile> tl;
  std::vector<int32_t> kb;
  std::vector<int64_t> start;
  for (int pass = 0; pass < 2; ++pass) {
    start.push_back((int64_t)tl.size());
    for (int32_t i = 0; i < ctx->n_blocks; ++i) {
      const BlockDesc& bd = ctx->h_blocks[i];
      for (int m0 = 0; m0 < bd.n_pad; m0 += TM)
        for (int n0 = pass ? m0 : 0; n0 < bd.n_pad; n0 += CG_TN) {
          tl.push_back(Tile{i, m0, n0, std::min(bd.n_pad, (pass ? n0 : m0) + TM)});
          kb.push_back(0);
        }
    }
  }
  int max_nb = 0;
  for (const auto& bd : ctx->h_blocks) max_nb = std::max(max_nb, bd.n_pad / TM);
  for (int i = 1; i < max_nb; ++i)
    for (int prod = 0; prod < 2; ++prod) {
      start.push_back((int64_t)tl.size());
      for (int32_t b = 0; b < ctx->n_blocks; ++b) {
        if (ctx->h_blocks[b].n_pad / TM <= i) continue;
        for (int c = 0; c < i; ++c) {
          if (prod == 0) {
            tl.push_back(Tile{b, TM * c, TM * i, TM * i});   // R^T tile (c, i), K over [128 c, 128 i)
            kb.push_back(TM * c);
          } else {
            tl.push_back(Tile{b, TM * i, TM * c, TM * (i + 1)});   // X tile (i, c), K over the block row i
            kb.push_back(TM * i);
          }
        }
      }
    }
  start.push_back((int64_t)tl.size());
  if ((int64_t)tl.size() > ctx->bt_cap) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemcpyAsync(ctx->d_bt, tl.data(), tl.size() * sizeof(Tile), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->d_cg_kbeg, kb.data(), kb.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);   // host temporaries
  if (e != cudaSuccess) return e;
  ctx->bt_start.swap(start);
  ctx->bt_layout = ctx->h_blocks;
  ctx->bt_dev = ctx->d_bt;
  ctx->bt_kdev = ctx->d_cg_kbeg;
  return cudaSuccess;
}

// The congruence on the tensor cores over launches 0 and 1 of the build's tile lists; the second
// pass mirrors its output.
cudaError_t launch_congruence_tc(nolsm_ctx* ctx, float* t1) {
  cudaError_t e = cg_maps(ctx, t1);
  if (e == cudaSuccess) e = build_tile_lists(ctx);
  if (e != cudaSuccess) return e;
  for (int pass = 0; pass < 2; ++pass) {
    const int n = (int)(ctx->bt_start[pass + 1] - ctx->bt_start[pass]);
    const Tile* t = ctx->d_bt + ctx->bt_start[pass];
    // pass 0: T1 (pool 2) = L^-1 (pool 0) x T_b(H0) (A0 pool, 1); pass 1: A0 pool = T1 x L^-1, mirrored
    const CgParams p = pass ? cg_params(ctx, t, nullptr, n, 2, 0, 1, -1, 0, 1, ctx->d_a0)
                            : cg_params(ctx, t, nullptr, n, 0, 1, 2, -1, 0, 0, t1);
    cong_tc_kernel<<<ctx->num_sms, CG_THREADS, CG_SMEM, ctx->stream>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// L^-1 of every block (mixed paths) by 128-row block rows, X = L^-1 and its transpose Y = X^T:
//   X_ii = L_ii^-1 (trinv_diag_launch: the 128 x 128 diagonal blocks, which also writes Y_ii and
//   zeroes the strict upper blocks), then for i = 1, 2, ...:
//   R_ic^T = sum_{k=c}^{i-1} Y_ck L_ik^T   and   X_ic = -X_ii R_ic  (Y_ci = X_ic^T stored beside it)
// for every c < i, as 3 x TF32 tensor-core products over launches 2, 3, ... of the build's tile lists
// (two launches per block row: the second needs the first's R^T, the next row needs this row's X and
// Y).  Y lives in the T1 pool (T1 is formed after the inverse), R^T in the scratch after the FP32
// factor.
cudaError_t launch_trinv_tc(nolsm_ctx* ctx, const float* l32, float* ypool) {
  int max_nb = 0;
  for (const auto& bd : ctx->h_blocks) max_nb = std::max(max_nb, bd.n_pad / TM);
  trinv_diag_launch(ctx, l32, ypool, max_nb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || max_nb < 2) return e;
  if ((e = cg_maps(ctx, ypool)) != cudaSuccess) return e;
  if ((e = build_tile_lists(ctx)) != cudaSuccess) return e;
  float* rt = const_cast<float*>(l32) + ctx->sum_sq;
  for (size_t k = 2; k + 1 < ctx->bt_start.size(); ++k) {
    const int n = (int)(ctx->bt_start[k + 1] - ctx->bt_start[k]);
    if (n == 0) continue;
    const Tile* t = ctx->d_bt + ctx->bt_start[k];
    const int32_t* kp = ctx->d_cg_kbeg + ctx->bt_start[k];
    // pools: 0 X = L^-1, 2 Y, 3 L, 4 R^T
    const CgParams p = (k % 2 == 0) ? cg_params(ctx, t, kp, n, 2, 3, 4, -1, 0, 0, rt)
                                    : cg_params(ctx, t, kp, n, 0, 4, 0, 2, 1, 0, ctx->d_linv);
    cong_tc_kernel<<<ctx->num_sms, CG_THREADS, CG_SMEM, ctx->stream>>>(p);
    ctx->n_launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int tc_tile_n() { return TN; }

// Work items (block, 32-column chunk) of every panel's trailing update, two tensor maps over the
// slice planes (OZ_NSL n_pad rows of 64 BF16 per block, blocks in layout order) and two per bin over the
// double-float pool the factor is computed in (ctx->d_sb).
cudaError_t oz_prepare(nolsm_ctx* ctx) {
  auto encode = get_encode();
  if (!encode || !ctx->d_oz_planes) return cudaErrorNotSupported;
  int max_pad = 0;
  for (const auto& bd : ctx->h_blocks) max_pad = std::max(max_pad, bd.n_pad);
  const int panels = (max_pad + kOzPanel - 1) / kOzPanel;
  ctx->h_oz_items.clear();
  ctx->h_oz_panel.assign((size_t)panels + 1, 0);
  for (int pnl = 0; pnl < panels; ++pnl) {
    ctx->h_oz_panel[pnl] = (int64_t)ctx->h_oz_items.size() / 2;
    const int t0 = (pnl + 1) * kOzPanel;
    for (int32_t b = 0; b < ctx->n_blocks; ++b) {
      const BlockDesc& bd = ctx->h_blocks[b];
      if (t0 >= bd.n) continue;
      for (int n0 = t0; n0 < bd.n; n0 += OZ_TN) ctx->h_oz_items.insert(ctx->h_oz_items.end(), {b, n0});
    }
  }
  ctx->h_oz_panel[panels] = (int64_t)ctx->h_oz_items.size() / 2;
  // TRSM items of every panel: (block, 128-row tile) of the rows below its diagonal block
  ctx->h_tr_items.clear();
  ctx->h_tr_panel.assign((size_t)panels + 1, 0);
  for (int pnl = 0; pnl < panels; ++pnl) {
    ctx->h_tr_panel[pnl] = (int64_t)ctx->h_tr_items.size();
    const int t0 = (pnl + 1) * kOzPanel;
    for (int32_t b = 0; b < ctx->n_blocks; ++b) {
      const BlockDesc& bd = ctx->h_blocks[b];
      for (int m0 = t0; m0 < bd.n; m0 += TM)
        ctx->h_tr_items.push_back(TrItem{b, m0, bd.n, bd.n_pad, bd.row_off, bd.pos, bd.bin, 0, bd.off_mat});
    }
  }
  ctx->h_tr_panel[panels] = (int64_t)ctx->h_tr_items.size();
  if (!ctx->h_tr_items.empty()) {
    cudaError_t e = cudaMemcpyAsync(ctx->d_tr_items, ctx->h_tr_items.data(), sizeof(TrItem) * ctx->h_tr_items.size(),
                                    cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return e;
  }
  if (!ctx->h_oz_items.empty()) {
    cudaError_t e = cudaMemcpyAsync(ctx->d_oz_items, ctx->h_oz_items.data(), sizeof(int32_t) * ctx->h_oz_items.size(),
                                    cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return e;
  }
  int n_bins = 0;
  for (const auto& b : ctx->h_blocks) n_bins = std::max(n_bins, b.bin + 1);
  std::vector<CUtensorMap> maps((size_t)(3 + 2 * n_bins));
  const uint64_t rows = (uint64_t)OZ_NSL * (uint64_t)std::max<int64_t>(ctx->sum_pad, 1);
  cuuint64_t gdim[2] = {(cuuint64_t)kOzPanel, rows};
  cuuint64_t gstride[1] = {(cuuint64_t)kOzPanel * 2};
  cuuint32_t estr[2] = {1, 1};
  cuuint32_t box_a[2] = {(cuuint32_t)kOzPanel, (cuuint32_t)TM};
  cuuint32_t box_b[2] = {(cuuint32_t)kOzPanel, (cuuint32_t)OZ_TN};
  CUresult r = encode(&maps[0], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ctx->d_oz_planes, gdim, gstride, box_a, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r == CUDA_SUCCESS)
    r = encode(&maps[1], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ctx->d_oz_planes, gdim, gstride, box_b, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  // per bin, over the pool of double-float pairs (8 bytes an entry, the bin's blocks stacked as
  // n_pad-row matrices): 16 x 128 loads and 16 x 32 stores of the updated tiles, 128-byte swizzle
  std::vector<int64_t> bin_off(n_bins, 0), bin_cnt(n_bins, 0);
  std::vector<int> bin_pad(n_bins, 0);
  for (const auto& b : ctx->h_blocks) {
    if (b.pos == 0) bin_off[b.bin] = b.off_mat;
    bin_cnt[b.bin] += 1;
    bin_pad[b.bin] = b.n_pad;
  }
  for (int bi = 0; bi < n_bins && r == CUDA_SUCCESS; ++bi) {
    const uint64_t np = (uint64_t)bin_pad[bi];
    cuuint64_t cdim[2] = {np, np * (uint64_t)std::max<int64_t>(bin_cnt[bi], 1)};
    cuuint64_t cstride[1] = {np * 8};
    cuuint32_t cbox_l[2] = {16, (cuuint32_t)TM};
    cuuint32_t cbox_s[2] = {16, 32};
    void* base = ctx->d_sb + bin_off[bi];
    r = encode(&maps[2 + 2 * bi], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, base, cdim, cstride, cbox_l, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS)
      r = encode(&maps[3 + 2 * bi], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, base, cdim, cstride, cbox_s, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  // the TRSM's Minv planes: 6 x 64 rows of 64 BF16 per block, 64 x 32 boxes
  {
    cuuint64_t mdim[2] = {(cuuint64_t)kOzPanel, (cuuint64_t)OZ_NSL * 64 * (cuuint64_t)std::max(ctx->n_blocks, 1)};
    cuuint64_t mstride[1] = {(cuuint64_t)kOzPanel * 2};
    r = encode(&maps[2 + 2 * n_bins], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ctx->d_oz_m, mdim, mstride, box_b, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  ctx->h_oz_maps.assign(reinterpret_cast<const uint8_t*>(maps.data()),
                        reinterpret_cast<const uint8_t*>(maps.data() + maps.size()));
  cudaError_t e = cudaMemcpyAsync(ctx->d_oz_tmaps, ctx->h_oz_maps.data(), ctx->h_oz_maps.size(),
                                  cudaMemcpyHostToDevice, ctx->stream);   // source kept in the context
  if (e != cudaSuccess) return e;
  static bool attr_done = false;
  if (!attr_done) {
    e = cudaFuncSetAttribute(chol_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(chol_trsm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TR_SMEM);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  return cudaSuccess;
}

cudaError_t launch_chol_trsm_tc(nolsm_ctx* ctx, int panel, double* pool, float* l32) {
  if (panel + 1 >= (int)ctx->h_tr_panel.size()) return cudaSuccess;
  const int64_t first = ctx->h_tr_panel[panel], count = ctx->h_tr_panel[panel + 1] - first;
  if (count <= 0) return cudaSuccess;
  int n_bins = 0;
  for (const auto& b : ctx->h_blocks) n_bins = std::max(n_bins, b.bin + 1);
  TrParams p;
  p.items = ctx->d_tr_items + first;
  p.n_items = (int)count;
  p.mmap = reinterpret_cast<const CUtensorMap*>(ctx->d_oz_tmaps) + 2 + 2 * n_bins;
  p.cmaps = reinterpret_cast<const CUtensorMap*>(ctx->d_oz_tmaps) + 2;
  p.pool = pool;
  p.scale_exp = ctx->d_oz_exp;
  p.mf = ctx->d_oz_f;
  p.planes = reinterpret_cast<__nv_bfloat16*>(ctx->d_oz_planes);
  p.l32 = l32;
  p.c0 = panel * kOzPanel;
  p.flags = ctx->d_flags;
  p.budget = ctx->opt.wait_budget;
  const int grid = (int)std::min<int64_t>(ctx->num_sms, count);
  chol_trsm_tc_kernel<<<grid, TR_THREADS, TR_SMEM, ctx->stream>>>(p);
  ctx->n_launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_chol_update_tc(nolsm_ctx* ctx, int panel, double* pool) {
  if (panel + 1 >= (int)ctx->h_oz_panel.size()) return cudaSuccess;
  const int64_t first = ctx->h_oz_panel[panel], count = ctx->h_oz_panel[panel + 1] - first;
  if (count <= 0) return cudaSuccess;
  OzParams p;
  p.items = ctx->d_oz_items + 2 * first;
  p.n_items = (int)count;
  p.blocks = ctx->d_blocks;
  p.maps = reinterpret_cast<const CUtensorMap*>(ctx->d_oz_tmaps);
  p.pool = pool;
  p.scale_exp = ctx->d_oz_exp;
  p.t0 = (panel + 1) * kOzPanel;
  p.flags = ctx->d_flags;
  p.budget = ctx->opt.wait_budget;
  const int grid = (int)std::min<int64_t>(ctx->num_sms, count);
  chol_update_kernel<<<grid, OZ_THREADS, OZ_SMEM, ctx->stream>>>(p);
  ctx->n_launches += 1;
  return cudaGetLastError();
}

// The refinement on the tensor cores: narrow pieces (<= 32 columns, four 24 KB stages, 64 tensor-memory
// columns, two CTAs per SM so that one piece's chain of dependent products hides the other's), then wide
// ones (<= 192 columns, three 64 KB stages), one persistent CTA per SM each.  Slab scratch: P1 and
// F1 (FP32), then the four split pools hi0, lo0, hi1, lo1 in the iterate's format.
cudaError_t launch_slab_tc(nolsm_ctx* ctx) {
  const bool bf16 = ctx->opt.precision == NOLSM_PREC_MIXED_BF16;
  using LN = SlabLayout<kSlabNarrow, 4>;
  using LW = SlabLayout<kSlabWide, 3>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(slab_tc_kernel<__half, kSlabNarrow, 4>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, LN::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(slab_tc_kernel<__nv_bfloat16, kSlabNarrow, 4>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, LN::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(slab_tc_kernel<__half, kSlabWide, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               LW::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(slab_tc_kernel<__nv_bfloat16, kSlabWide, 3>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, LW::SMEM);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  if (!ctx->d_tmaps || !ctx->d_tmp || !ctx->d_slab_units) return cudaErrorInvalidValue;
  SlabParams p;
  p.blocks = ctx->d_blocks;
  p.st = ctx->d_state;
  p.tmaps = reinterpret_cast<const CUtensorMap*>(ctx->d_tmaps);
  p.w = ctx->d_w;
  p.z = ctx->d_z;
  p.lc = ctx->d_lc;
  p.y = ctx->d_y;
  p.s1 = ctx->d_tmp;
  p.f1 = ctx->d_tmp + ctx->sum_slab;
  uint16_t* pools = reinterpret_cast<uint16_t*>(ctx->d_tmp + 2 * ctx->sum_slab);
  for (int i = 0; i < 4; ++i) p.hl[i] = pools + (int64_t)i * ctx->sum_slab;
  p.flags = ctx->d_flags;
  p.budget = ctx->opt.wait_budget;
  p.refine = ctx->opt.refine_iters;
  cudaError_t e = cudaMemsetAsync(&ctx->d_flags->slab_queue[0], 0, 2 * sizeof(int32_t), ctx->stream);
  if (e != cudaSuccess) return e;
  if (ctx->n_units_narrow > 0) {
    p.units = ctx->d_slab_units;
    p.n_units = ctx->n_units_narrow;
    p.queue = &ctx->d_flags->slab_queue[0];
    p.bn = ctx->d_bn;
    p.be = ctx->d_be;
    const int grid = std::min(2 * ctx->num_sms, ctx->n_units_narrow);   // two CTAs per SM
    if (bf16) slab_tc_kernel<__nv_bfloat16, kSlabNarrow, 4><<<grid, NUM_THREADS, LN::SMEM, ctx->stream>>>(p);
    else slab_tc_kernel<__half, kSlabNarrow, 4><<<grid, NUM_THREADS, LN::SMEM, ctx->stream>>>(p);
    ctx->n_launches += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (ctx->n_units_wide > 0) {
    p.units = ctx->d_slab_units + 4 * ctx->n_units_narrow;
    p.n_units = ctx->n_units_wide;
    p.queue = &ctx->d_flags->slab_queue[1];
    p.bn = ctx->d_bn + ctx->n_units_narrow;
    p.be = ctx->d_be + ctx->n_units_narrow;
    const int grid = std::min(ctx->num_sms, ctx->n_units_wide);
    if (bf16) slab_tc_kernel<__nv_bfloat16, kSlabWide, 3><<<grid, NUM_THREADS, LW::SMEM, ctx->stream>>>(p);
    else slab_tc_kernel<__half, kSlabWide, 3><<<grid, NUM_THREADS, LW::SMEM, ctx->stream>>>(p);
    ctx->n_launches += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The persistent schedule: one launch for the whole iteration of every block (see ns_pair_kernel;
// interleaved: two blocks per cluster, see ns_pair2_kernel).
cudaError_t launch_ns_pair(nolsm_ctx* ctx, double mu, bool interleaved) {
  PairParams p;
  p.blocks = ctx->d_blocks;
  p.st = ctx->d_state;
  p.tmaps = reinterpret_cast<const CUtensorMap*>(ctx->d_tmaps);
  p.a0 = ctx->d_a0;
  p.lo = ctx->d_lo;
  p.hi = ctx->d_hi;
  p.tol = ctx->d_tol;
  p.x0 = ctx->d_x[0];
  p.x1 = ctx->d_x[1];
  p.bbuf = ctx->d_b;
  p.flags = ctx->d_flags;
  p.budget = ctx->opt.wait_budget;
  p.mu = mu;
  p.margin = (float)ctx->opt.alpha_margin;
  p.l0 = std::max((float)ctx->opt.lower_bound, scaled_l_floor(ctx));
  p.scaled = ctx->opt.scaled;
  p.max_iter = ctx->opt.max_iter;
  p.detect_divergence = ctx->opt.bounds != NOLSM_BOUNDS_GERSHGORIN;
  p.n_blocks = ctx->n_blocks;
  p.fp8_iters = ctx->opt.fp8_iters;
  p.queue_map = ctx->n_queue < ctx->n_blocks ? ctx->d_queue : nullptr;
  p.n_queue = ctx->n_queue;
  const bool bf16 = ctx->opt.precision == NOLSM_PREC_MIXED_BF16;
  if (ctx->pair_clusters <= 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * 256, 1, 1);
    cfg.blockDim = dim3(PAIR_THREADS, 1, 1);
    cfg.dynamicSmemBytes = PAIR_SMEM;
    cfg.stream = ctx->stream;
    int n = 0;
    cudaError_t e = bf16 ? cudaOccupancyMaxActiveClusters(&n, ns_pair_kernel<__nv_bfloat16, false>, &cfg)
                         : cudaOccupancyMaxActiveClusters(&n, ns_pair_kernel<__half, false>, &cfg);
    if (e != cudaSuccess) return e;
    ctx->pair_clusters = n > 0 ? n : ctx->num_sms / 2;
  }
  if (interleaved) {
    // two slots per cluster: enough clusters for every block to start in the first round
    const int clusters = std::max(1, std::min(ctx->pair_clusters, (ctx->n_queue + 1) / 2));
    if (bf16)
      ns_pair2_kernel<__nv_bfloat16><<<2 * clusters, PAIR_THREADS, PAIR2_SMEM, ctx->stream>>>(p);
    else
      ns_pair2_kernel<__half><<<2 * clusters, PAIR_THREADS, PAIR2_SMEM, ctx->stream>>>(p);
    return cudaGetLastError();
  }
  const int clusters = std::max(1, std::min(ctx->pair_clusters, ctx->n_queue));
  const bool q8 = p.fp8_iters > 0;
  if (bf16 && q8)
    ns_pair_kernel<__nv_bfloat16, true><<<2 * clusters, PAIR_THREADS, PAIR_SMEM, ctx->stream>>>(p);
  else if (bf16)
    ns_pair_kernel<__nv_bfloat16, false><<<2 * clusters, PAIR_THREADS, PAIR_SMEM, ctx->stream>>>(p);
  else if (q8)
    ns_pair_kernel<__half, true><<<2 * clusters, PAIR_THREADS, PAIR_SMEM, ctx->stream>>>(p);
  else
    ns_pair_kernel<__half, false><<<2 * clusters, PAIR_THREADS, PAIR_SMEM, ctx->stream>>>(p);
  return cudaGetLastError();
}

}  // namespace nolsm
