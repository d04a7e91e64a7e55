// lbpf_field_sums_noalloc: the FP64 conservation sums of lbpf_diagnostics,
// computed from caller-owned device fields without allocating anything.
//
// Some callers cannot allocate device memory at the point where they need
// these sums: code running inside a memory pool or allocator callback, a
// host that has handed every byte of the GPU to its own arena, or a real-time
// loop where an allocation would stall.  This entry point keeps its only
// scratch, the per-block partial sums of the two-pass reduction, in a
// file-scope device array of fixed size that every GPU loading the library
// holds until the process exits.
#include <cuda.h>

#include <cstdint>
#include <cstdio>

#include "../../include/lbpf.h"
#include "lbpf_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 64;  // nodes per thread at the largest grid
constexpr int kSlots = 3;   // sum(U + phi_prev), sum(rho), sum((1 + clamp(phi))/2)

// Scratch: one row of partial sums per block.
static __device__ __align__(256) double g_partials[LBPF_NOALLOC_MAX_BLOCKS * kSlots];

template <typename V>
__global__ void __launch_bounds__(kThreads)
    sums_partial_kernel(const V* phi, const V* phi_prev, const V* U, const V* rho, int64_t n,
                        double* partials) {
  double acc[kSlots] = {0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    const double p = double(phi[i]);
    const double ph = p < -1.0 ? -1.0 : (p > 1.0 ? 1.0 : p);
    acc[0] += double(U[i]) + double(phi_prev[i]);
    acc[1] += rho ? double(rho[i]) : 1.0;
    acc[2] += 0.5 * (1.0 + ph);
  }
  __shared__ double sh[kSlots][kThreads];
  for (int k = 0; k < kSlots; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < kSlots; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < kSlots) partials[blockIdx.x * kSlots + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kThreads)
    sums_final_kernel(const double* partials, int nblocks, double* out) {
  __shared__ double sh[kSlots][kThreads];
  double acc[kSlots] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += kThreads)
    for (int k = 0; k < kSlots; ++k) acc[k] += partials[b * kSlots + k];
  for (int k = 0; k < kSlots; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < kSlots; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < kSlots) out[threadIdx.x] = sh[threadIdx.x][0];
}

// Device address of g_partials per device, looked up with that device
// current (in host code the symbol is only a host-side stand-in).  The address
// belongs to the device's current context: after a cudaDeviceReset the
// primary context and the module are created anew, so the cache is keyed by
// the context's unique ID as well and looked up again when that changes.
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// unique ID of the current context (0 if the driver cannot say)
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(p);
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
      get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

double* scratch_for_current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  // 0 when no context is current yet (the lookup below creates it) or the
  // driver cannot name it: then the address is looked up again
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess) return nullptr;
    g_scratch_ptr[dev] = static_cast<double*>(p);
    g_scratch_ctx[dev] = current_context_id();
  }
  return g_scratch_ptr[dev];
}

}  // namespace

namespace lbk {

int field_sums_blocks(int64_t n) {
  int64_t blocks = (n + (int64_t)kThreads * kItems - 1) / ((int64_t)kThreads * kItems);
  if (blocks < 1) blocks = 1;
  if (blocks > LBPF_NOALLOC_MAX_BLOCKS) blocks = LBPF_NOALLOC_MAX_BLOCKS;
  return int(blocks);
}

cudaError_t launch_field_sums(const void* phi, const void* phi_prev, const void* U,
                              const void* rho, int64_t n, int fp64, double* partials,
                              int blocks, double* out, cudaStream_t s) {
  // every block writes its own row of partials, so they need no clearing
  if (fp64)
    sums_partial_kernel<double><<<blocks, kThreads, 0, s>>>(
        static_cast<const double*>(phi), static_cast<const double*>(phi_prev),
        static_cast<const double*>(U), static_cast<const double*>(rho), n, partials);
  else
    sums_partial_kernel<float><<<blocks, kThreads, 0, s>>>(
        static_cast<const float*>(phi), static_cast<const float*>(phi_prev),
        static_cast<const float*>(U), static_cast<const float*>(rho), n, partials);
  sums_final_kernel<<<1, kThreads, 0, s>>>(partials, blocks, out);
  return cudaGetLastError();
}

}  // namespace lbk

extern "C" lbpf_status lbpf_field_sums_noalloc(const void* phi, const void* phi_prev, const void* U,
                                       const void* rho, int64_t n, int fp64, double* out,
                                       void* stream) {
  if (!phi || !phi_prev || !U || !out || n < 0) return LBPF_EINVAL;
  if (n > (int64_t)LBPF_NOALLOC_MAX_NODES) {
    fprintf(stderr,
            "lbpf_field_sums_noalloc: n = %lld exceeds the maximum of %lld nodes "
            "(fixed scratch of %d blocks)\n",
            (long long)n, (long long)LBPF_NOALLOC_MAX_NODES, LBPF_NOALLOC_MAX_BLOCKS);
    return LBPF_EINVAL;
  }
  double* scratch = scratch_for_current_device();
  if (!scratch) return LBPF_ECUDA;
  return lbk::launch_field_sums(phi, phi_prev, U, rho, n, fp64, scratch,
                                lbk::field_sums_blocks(n), out,
                                static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? LBPF_OK
             : LBPF_ECUDA;
}
