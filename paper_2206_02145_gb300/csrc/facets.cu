// Crystal-shape measurement on the device (Sec. 3.1.2 and Sec. 3.2): the
// support values of the phi = 0 contour along the facet normals and the four
// axis directions.  The contour is located on every x- and y-edge of the
// grid whose end values change sign (phi > 0 at one end only), by linear
// interpolation in FP64; edges across a periodic wrap are not used.  The side
// centres, the crystal centre and the side lengths follow on the host from
// these few numbers.
//
// One pass over the h populations: persistent CTAs walk 32 x 8 tiles, form
// phi = -1 + sum_a d_a (Eq. 22, in the step's arithmetic and summation order,
// so that it is the phi the field read-out returns) for the tile and a
// one-node halo row and column in shared memory, and test the tile's edges in
// that arithmetic.  Only warps that hold a crossing enter the FP64 part (this
// GPU's FP64 rate is low, and predicated FP64 instructions would still
// issue).  Maxima are kept as order-preserving 64-bit integer keys of the
// doubles, raised by atomicMax in shared memory and then once per CTA in
// global memory; the point count is an integer sum: both exact and
// independent of the order of arrival, so the result is reproducible bit for
// bit.

#include <cstring>

#include "lbpf_device.cuh"
#include "lbpf_internal.cuh"

namespace lbk {
namespace {

constexpr int kThreads = 256;
constexpr int kTx = 32, kTy = 8;   // tile: one node per thread
constexpr int kBlocksPerSm = 6;    // 35 registers x 256 threads, no spills
constexpr unsigned kFull = 0xffffffffu;

// IEEE-754 doubles (not NaN) to unsigned keys of the same order; key 0 lies
// below every double, so zeroed slots mean "no value yet"
__device__ __forceinline__ unsigned long long order_key(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

template <typename T, typename R>
__device__ __forceinline__ R node_phi(const T* __restrict__ ph, long long P, long long j,
                                      R ref_h) {
  R d = R(0);
#pragma unroll
  for (int a = 0; a < 9; ++a) d += Pop<T>::template ld<R>(ph + a * P + j);
  return ref_h + d;
}

// a contour point: raise the CTA's maxima (order keys in shared memory)
__device__ __forceinline__ void take(const FacetDirs& d, double px, double py,
                                     unsigned long long* s_best) {
  for (int j = 0; j < d.n; ++j) {
    const double v = __dadd_rn(__dmul_rn(px, d.dx[j]), __dmul_rn(py, d.dy[j]));
    atomicMax(s_best + j, order_key(v));
  }
}

template <typename T, typename R>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm)
    facet_support_kernel(const Model m, const T* __restrict__ pops, const FacetDirs d,
                         unsigned long long* __restrict__ out) {
  __shared__ R sh[kTy + 1][kTx + 1];
  __shared__ unsigned long long s_best[kMaxDirs];
  __shared__ unsigned s_cnt;
  if (threadIdx.x < kMaxDirs) s_best[threadIdx.x] = 0ull;
  if (threadIdx.x == kMaxDirs) s_cnt = 0u;
  const long long P = m.plane;
  const T* ph = pops + (long long)(m.qf + m.qs) * P;
  const R ref_h = coef<R>(m).ref_h;
  const int nx = m.nx, ny = m.ny, px = m.px;
  const int tx = threadIdx.x % kTx, ty = threadIdx.x / kTx;
  const int ntx = (nx + kTx - 1) / kTx, nty = (ny + kTy - 1) / kTy;
  unsigned cnt = 0;
  for (int tile = blockIdx.x; tile < ntx * nty; tile += gridDim.x) {
    const int x0 = (tile % ntx) * kTx, y0 = (tile / ntx) * kTy;
    const int x = x0 + tx, y = y0 + ty;
    const bool in = x < nx && y < ny;
    if (in) sh[ty][tx] = node_phi<T, R>(ph, P, (long long)y * px + x, ref_h);
    // halo: the row after the tile (threads 0..31), the column after it (32..39)
    if (threadIdx.x < kTx) {
      const int yy = y0 + kTy;
      if (x < nx && yy < ny) sh[kTy][tx] = node_phi<T, R>(ph, P, (long long)yy * px + x, ref_h);
    } else if (threadIdx.x < kTx + kTy) {
      const int xx = x0 + kTx, yy = y0 + threadIdx.x - kTx;
      if (xx < nx && yy < ny)
        sh[yy - y0][kTx] = node_phi<T, R>(ph, P, (long long)yy * px + xx, ref_h);
    }
    __syncthreads();
    {
      const R a = in ? sh[ty][tx] : R(0);
      const bool pa = a > R(0);
      // (tx + 1, ty + 1 stay inside sh; their values count only where in the grid)
      const bool ex = in && x + 1 < nx && (pa != (sh[ty][tx + 1] > R(0)));  // x-edge
      const bool ey = in && y + 1 < ny && (pa != (sh[ty + 1][tx] > R(0)));  // y-edge
      cnt += unsigned(ex) + unsigned(ey);
      if (__any_sync(kFull, ex || ey)) {  // warp-uniform: rare
        const double da = double(a);
        if (ex) {
          const double db = double(sh[ty][tx + 1]);
          take(d, double(x) + da / (da - db), double(y), s_best);
        }
        if (ey) {
          const double db = double(sh[ty + 1][tx]);
          take(d, double(x), double(y) + da / (da - db), s_best);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&s_cnt, cnt);
  __syncthreads();
  if (threadIdx.x < d.n) {
    if (s_best[threadIdx.x]) atomicMax(out + threadIdx.x, s_best[threadIdx.x]);
  } else if (threadIdx.x == kMaxDirs) {
    if (s_cnt) atomicAdd(out + kMaxDirs, (unsigned long long)s_cnt);
  }
}

template <typename T, typename R>
cudaError_t support_t(const Model& m, const void* pops, const FacetDirs& dirs,
                      unsigned long long* out, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int tiles = ((m.nx + kTx - 1) / kTx) * ((m.ny + kTy - 1) / kTy);
  const int cap = sms * kBlocksPerSm;
  const int grid = tiles < cap ? tiles : cap;
  if ((e = cudaMemsetAsync(out, 0, sizeof(unsigned long long) * (kMaxDirs + 1), s)) !=
      cudaSuccess)
    return e;
  facet_support_kernel<T, R><<<grid, kThreads, 0, s>>>(m, static_cast<const T*>(pops), dirs,
                                                       out);
  return cudaGetLastError();
}

}  // namespace

double facet_key_value(unsigned long long k) {
  const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  double v;
  static_assert(sizeof(v) == sizeof(u), "64-bit double");
  std::memcpy(&v, &u, sizeof(v));
  return v;
}

cudaError_t launch_facet_support(const Model& m, const void* pops, const FacetDirs& dirs,
                                 unsigned long long* out, cudaStream_t s) {
  if (m.dim != 2 || dirs.n < 1 || dirs.n > kMaxDirs) return cudaErrorInvalidValue;
  switch (m.storage) {
    case ST_FP64: return support_t<double, double>(m, pops, dirs, out, s);
    case ST_FP16: return support_t<__half, float>(m, pops, dirs, out, s);
    case ST_BF16: return support_t<__nv_bfloat16, float>(m, pops, dirs, out, s);
    default: return support_t<float, float>(m, pops, dirs, out, s);
  }
}

}  // namespace lbk
