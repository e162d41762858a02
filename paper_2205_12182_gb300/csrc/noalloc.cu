// Band energy without any allocation: the partial sums live in a fixed file-scope device array.
//
// nolsm_band_energy needs a context, and a context allocates device memory.  Some callers cannot
// allocate at the point where they want the energy: code running between the steps of a
// molecular-dynamics integrator with a pre-sized memory budget, runtimes that own every device
// allocation through their own pool, or a hot loop where an allocation would synchronise the
// device.  For them this entry point computes the same reduction from caller-provided device
// arrays, writing its intermediate sums into `g_partials` below, which every GPU that loads the
// library holds (128 KB) until the process exits.
#include "internal.h"

namespace {

constexpr int kChunk = 1 << 14;                 // stored entries per partial sum (one CTA each)
constexpr int kMaxPartials = 1 << 14;           // capacity of the scratch array (128 KB)
constexpr int64_t kMaxEntries = (int64_t)kChunk * kMaxPartials;   // 268,435,456

// Scratch shared by every call on this device: the partial sums of the latest call.
static __device__ __align__(256) double g_partials[kMaxPartials];

// One CTA per chunk of kChunk entries: partial[chunk] = sum D_e H_e over the chunk (FP64).
__global__ void __launch_bounds__(256) energy_partials_kernel(int64_t nnz, const double* __restrict__ d,
                                                              const double* __restrict__ h,
                                                              double* __restrict__ partials) {
  __shared__ double red[8];
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  const int64_t end = min(base + (int64_t)kChunk, nnz);
  double s = 0.0;
  for (int64_t i = base + threadIdx.x; i < end; i += blockDim.x) s += d[i] * h[i];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    partials[blockIdx.x] = t;      // every used slot is overwritten: nothing has to start at zero
  }
}

// Single CTA: e_out = spin_factor * sum of the n partials, in a fixed order.
__global__ void __launch_bounds__(256) energy_total_kernel(int n, const double* __restrict__ partials,
                                                           double spin_factor, double* __restrict__ e_out) {
  __shared__ double red[8];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    *e_out = spin_factor * t;
  }
}

// Device address of g_partials in the current device's context.  In host code the symbol is only
// a host-side stand-in, so kernels must be given the address cudaGetSymbolAddress returns with the
// device current.  The lookup is repeated on every call (it allocates nothing once the module is
// loaded): an address kept from an earlier call could belong to a context that was reset since,
// or to another context of the same device.
cudaError_t scratch_for_current_device(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" nolsm_status nolsm_band_energy_noalloc(int64_t nnz, const double* d_val, const double* h_val,
                                                  double spin_factor, double* e_out, void* cuda_stream) {
  if (nnz <= 0 || !d_val || !h_val || !e_out || !(spin_factor > 0)) return NOLSM_EINVAL;
  if (nnz > kMaxEntries) return NOLSM_EINVAL;   // more partial sums than the fixed scratch holds
  double* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return NOLSM_ECUDA;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int n_part = (int)((nnz + kChunk - 1) / kChunk);
  // A launch error is read (and cleared) with cudaGetLastError, which would also return an error
  // left pending by earlier work of the caller.  Such an error is cleared here, before the first
  // launch, so that the status below reports this call's own launches only.
  (void)cudaGetLastError();
  energy_partials_kernel<<<n_part, 256, 0, stream>>>(nnz, d_val, h_val, scratch);
  if (cudaGetLastError() != cudaSuccess) return NOLSM_ECUDA;
  energy_total_kernel<<<1, 256, 0, stream>>>(n_part, scratch, spin_factor, e_out);
  return cudaGetLastError() == cudaSuccess ? NOLSM_OK : NOLSM_ECUDA;
}
