// Crystal-shape measurement on the device (Sec. 3.1.2 and Sec. 3.2): the
// support values of the phi = 0 contour along the facet normals and the four
// axis directions.  The contour is located on every x- and y-edge of the
// grid whose end values change sign (phi > 0 at one end only), by linear
// interpolation; edges across a periodic wrap are not used.  The side
// centres, the crystal centre and the side lengths follow on the host from
// these few numbers.
//
// Two passes, as the FP64 diagnostics: per-CTA maxima and point counts into
// a scratch table, then one CTA over the table.  Maxima do not depend on the
// order of reduction, so the result is reproducible bit for bit.

#include "lbpf_internal.cuh"

namespace lbk {
namespace {

constexpr int kBlocks = 152 * 2;
constexpr int kThreads = 256;
constexpr int kSlots = kMaxDirs + 1;  // the maxima, then the point count

__device__ __forceinline__ void take(const FacetDirs& d, double px, double py,
                                     double (&best)[kMaxDirs]) {
#pragma unroll
  for (int j = 0; j < kMaxDirs; ++j)
    if (j < d.n) {
      const double v = __dadd_rn(__dmul_rn(px, d.dx[j]), __dmul_rn(py, d.dy[j]));
      best[j] = v > best[j] ? v : best[j];
    }
}

// reduce best[] and cnt of the CTA into row[0 .. kSlots)
__device__ void block_reduce(double (&best)[kMaxDirs], double cnt, double* row) {
  __shared__ double sh[kSlots][kThreads];
#pragma unroll
  for (int j = 0; j < kMaxDirs; ++j) sh[j][threadIdx.x] = best[j];
  sh[kMaxDirs][threadIdx.x] = cnt;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int j = 0; j < kMaxDirs; ++j) {
        const double o = sh[j][threadIdx.x + w];
        sh[j][threadIdx.x] = o > sh[j][threadIdx.x] ? o : sh[j][threadIdx.x];
      }
      sh[kMaxDirs][threadIdx.x] += sh[kMaxDirs][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x < kSlots) row[threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kThreads)
    facet_support_kernel(const double* __restrict__ phi, int nx, int ny, const FacetDirs d,
                         double* __restrict__ partials) {
  double best[kMaxDirs];
#pragma unroll
  for (int j = 0; j < kMaxDirs; ++j) best[j] = -INFINITY;
  double cnt = 0.0;
  const long long n = (long long)nx * ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = int(i % nx), y = int(i / nx);
    const double a = phi[i];
    const bool pa = a > 0.0;
    if (x + 1 < nx) {  // x-edge to (x + 1, y)
      const double b = phi[i + 1];
      if (pa != (b > 0.0)) {
        take(d, double(x) + a / (a - b), double(y), best);
        cnt += 1.0;
      }
    }
    if (y + 1 < ny) {  // y-edge to (x, y + 1)
      const double b = phi[i + nx];
      if (pa != (b > 0.0)) {
        take(d, double(x), double(y) + a / (a - b), best);
        cnt += 1.0;
      }
    }
  }
  block_reduce(best, cnt, partials + size_t(blockIdx.x) * kSlots);
}

__global__ void __launch_bounds__(kThreads)
    facet_final_kernel(const double* __restrict__ partials, int nblocks, int ndir,
                       double* __restrict__ out) {
  double best[kMaxDirs];
#pragma unroll
  for (int j = 0; j < kMaxDirs; ++j) best[j] = -INFINITY;
  double cnt = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    const double* row = partials + size_t(b) * kSlots;
#pragma unroll
    for (int j = 0; j < kMaxDirs; ++j) best[j] = row[j] > best[j] ? row[j] : best[j];
    cnt += row[kMaxDirs];
  }
  __shared__ double res[kSlots];
  block_reduce(best, cnt, res);
  __syncthreads();
  if (threadIdx.x < ndir) out[threadIdx.x] = res[threadIdx.x];
  if (threadIdx.x == 0) out[ndir] = res[kMaxDirs];
}

}  // namespace

size_t facet_scratch_bytes() { return sizeof(double) * kBlocks * kSlots; }

cudaError_t launch_facet_support(const double* phi, int nx, int ny, const FacetDirs& dirs,
                                 double* scratch, double* out, cudaStream_t s) {
  if (dirs.n < 1 || dirs.n > kMaxDirs || nx < 1 || ny < 1) return cudaErrorInvalidValue;
  facet_support_kernel<<<kBlocks, kThreads, 0, s>>>(phi, nx, ny, dirs, scratch);
  facet_final_kernel<<<1, kThreads, 0, s>>>(scratch, kBlocks, dirs.n, out);
  return cudaGetLastError();
}

}  // namespace lbk
