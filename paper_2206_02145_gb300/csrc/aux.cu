// Initial state, moment read-out and FP64 diagnostics of liblbpf.so.
#include "lbpf_device.cuh"

namespace lbk {
namespace {

__device__ __forceinline__ void node_xyz(const Model& m, long long i, int& x, int& y, int& z) {
  x = int(i % m.nx);
  long long r = i / m.nx;
  y = int(r % m.ny);
  z = int(r / m.ny);
}
__device__ __forceinline__ long long pitched(const Model& m, int x, int y, int z) {
  return ((long long)z * m.ny + y) * m.px + x;
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): Weyl increment
// 0x9E3779B97F4A7C15 followed by the two xor-shift-multiply rounds.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Equilibrium populations of (rho, u*, U, phi) in FP64 (Eq. 9 at second
// order, Eq. 16, Eq. 21 with N = 0), stored as deviations from w_a M_ref
// (M_ref = 1, U_ref, -1) in the population type; with a per-node g reference
// (2D, 16-bit storage) g relative to w_a U_n, U_n the node's U rounded to the
// FP16 of the reference planes, and both planes of the node set to U_n.
template <typename T>
__device__ void store_equilibrium(const Model& m, T* pops, long long j, double phi, double U,
                                  double rho, double ux, double uy, double uz) {
  const long long P = m.plane;
  const double ph = phi < -1.0 ? -1.0 : (phi > 1.0 ? 1.0 : phi);
  const double mask = m.flow ? 0.5 * (1.0 - ph) : 0.0;
  const double us[3] = {mask * ux, mask * uy, mask * uz};
  const double uu = us[0] * us[0] + us[1] * us[1] + us[2] * us[2];
  const __half Rh = __float2half_rn(float(U));
  const double Rg = m.rel_g ? double(__half2float(Rh)) : m.ref_g;
  T* pf = pops;
  T* pg = pops + (long long)m.qf * P;
  T* ph_ = pops + (long long)(m.qf + m.qs) * P;
  if (m.dim == 2) {
    for (int a = 0; a < 9; ++a) {
      const double w = d2_w<double>(a);
      const double cu = D2_CX[a] * us[0] + D2_CY[a] * us[1];
      if (m.flow)
        Pop<T>::st(pf + a * P + j,
                   w * ((rho - m.ref_f) + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu)));
      Pop<T>::st(pg + a * P + j, w * ((U - Rg) + U * 3.0 * cu));
      Pop<T>::st(ph_ + a * P + j, w * (phi - m.ref_h));
    }
    if (m.rel_g) m.uring[j] = m.uring[P + j] = Rh;
  } else {
    if (m.flow)
      for (int a = 0; a < 19; ++a) {
        const double w = d3q19_w<double>(a);
        const double cu = D3_CX[a] * us[0] + D3_CY[a] * us[1] + D3_CZ[a] * us[2];
        Pop<T>::st(pf + a * P + j,
                   w * ((rho - m.ref_f) + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu)));
      }
    for (int a = 0; a < 7; ++a) {
      const double w = d3q7_w<double>(a);
      const double cu = D3_CX[a] * us[0] + D3_CY[a] * us[1] + D3_CZ[a] * us[2];
      Pop<T>::st(pg + a * P + j, w * ((U - Rg) + U * 4.0 * cu));  // cs^2 = 1/4
      Pop<T>::st(ph_ + a * P + j, w * (phi - m.ref_h));
    }
    if (m.rel_g) m.uring[j] = m.uring[P + j] = Rh;
  }
}

// The same equilibrium in the arithmetic type R (FP32 for the FP32 and 16-bit
// storages): used where a whole state is rebuilt every few steps.
template <typename T, typename R>
__device__ void store_equilibrium_r(const Model& m, T* pops, long long j, R phi, R U, R rho, R ux,
                                    R uy) {
  const long long P = m.plane;
  const Coef<R>& c = coef<R>(m);
  const R ph = phi < R(-1) ? R(-1) : (phi > R(1) ? R(1) : phi);
  const R mask = m.flow ? R(0.5) * (R(1) - ph) : R(0);
  const R us0 = mask * ux, us1 = mask * uy;
  const R uu = us0 * us0 + us1 * us1;
  const __half Rh = __float2half_rn(float(U));
  const R Rg = m.rel_g ? R(__half2float(Rh)) : c.ref_g;
  T* pf = pops;
  T* pg = pops + (long long)m.qf * P;
  T* ph_ = pops + (long long)(m.qf + m.qs) * P;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const R w = d2_w<R>(a);
    const R cu = R(D2_CX[a]) * us0 + R(D2_CY[a]) * us1;
    if (m.flow)
      Pop<T>::st(pf + a * P + j,
                 w * ((rho - c.ref_f) + rho * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu)));
    Pop<T>::st(pg + a * P + j, w * ((U - Rg) + U * R(3) * cu));
    Pop<T>::st(ph_ + a * P + j, w * (phi - c.ref_h));
  }
  if (m.rel_g) m.uring[j] = m.uring[P + j] = Rh;
}

template <typename T, typename R>
__global__ void init_seed_kernel(const Model m, const SeedArgs s, T* pops, R* phi_prev) {
  const long long n = (long long)m.nx * m.ny * m.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    node_xyz(m, i, x, y, z);
    const double dx = x - s.cx, dy = y - s.cy, dz = m.dim == 3 ? z - s.cz : 0.0;
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    double phi = tanh((s.radius - r) / (sqrt(2.0) * m.w0));
    const unsigned long long bits =
        splitmix64(s.seed ^ ((unsigned long long)i * 0x9E3779B97F4A7C15ull));
    const double xi = double(bits >> 11) * 0x1.0p-52 - 1.0;  // [-1, 1)
    phi += s.noise_amp * xi;
    const long long j = pitched(m, x, y, z);
    store_equilibrium<T>(m, pops, j, phi, s.u0, 1.0, m.flow ? m.u_in : 0.0, 0.0, 0.0);
    phi_prev[j] = R(phi - m.ref_h);  // the ring holds phi + 1
  }
}

// Convex polygon seed (2D; the rhombic and hexagonal seeds of Sec. 3.1): the
// signed distance to {x : (x - c).n_i <= d_i} taken as s = max_i [(x - c).n_i
// - d_i] (exact inside and beside the sides), phi0 = tanh(-s / (sqrt(2) W0));
// noise, U, rho and u as for the round seed.
template <typename T, typename R>
__global__ void init_polygon_kernel(const Model m, const PolygonArgs a, T* pops, R* phi_prev) {
  const long long n = (long long)m.nx * m.ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    node_xyz(m, i, x, y, z);
    double sd = -1e300;
    for (int f = 0; f < a.k; ++f) {
      const double v = (x - a.cx) * a.nx[f] + (y - a.cy) * a.ny[f] - a.d[f];
      sd = v > sd ? v : sd;
    }
    double phi = tanh(-sd / (sqrt(2.0) * m.w0));
    const unsigned long long bits =
        splitmix64(a.seed ^ ((unsigned long long)i * 0x9E3779B97F4A7C15ull));
    const double xi = double(bits >> 11) * 0x1.0p-52 - 1.0;  // [-1, 1)
    phi += a.noise_amp * xi;
    const long long j = pitched(m, x, y, z);
    store_equilibrium<T>(m, pops, j, phi, a.u0, 1.0, m.flow ? m.u_in : 0.0, 0.0, 0.0);
    phi_prev[j] = R(phi - m.ref_h);  // the ring holds phi + 1
  }
}

// Solid nodes: buffer c's state copied to buffer c ^ 1.
template <typename T, typename R>
__global__ void solid_sync_kernel(const Model m, const T* src, T* dst, const R* ring_src,
                                  R* ring_dst, const __half* uref_src, __half* uref_dst) {
  const long long n = (long long)m.nx * m.ny * m.nz;
  const int q = m.qf + 2 * m.qs;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    node_xyz(m, i, x, y, z);
    const long long j = pitched(m, x, y, z);
    if (!m.solid[j]) continue;
    for (int a = 0; a < q; ++a) dst[a * m.plane + j] = src[a * m.plane + j];
    ring_dst[j] = ring_src[j];
    if (uref_src) uref_dst[j] = uref_src[j];
  }
}

template <typename T, typename R>
__global__ void init_fields_kernel(const Model m, const double* phi, const double* U,
                                   const double* rho, const double* ux, const double* uy,
                                   const double* uz, T* pops, R* phi_prev) {
  const long long n = (long long)m.nx * m.ny * m.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    node_xyz(m, i, x, y, z);
    const long long j = pitched(m, x, y, z);
    store_equilibrium<T>(m, pops, j, phi[i], U[i], rho ? rho[i] : 1.0, ux ? ux[i] : 0.0,
                         uy ? uy[i] : 0.0, uz ? uz[i] : 0.0);
    phi_prev[j] = R(phi[i] - m.ref_h);
  }
}

// Moments of one node from the stored populations, in the arithmetic type R
// of the step (FP32, or FP64 for FP64 storage).
template <typename T, typename R>
__device__ void node_moments(const Model& m, const T* pops, long long j, R& phi, R& U, R& rho,
                             R u[3], const __half* uref = nullptr) {
  const long long P = m.plane;
  const T* pf = pops;
  const T* pg = pops + (long long)m.qf * P;
  const T* ph_ = pops + (long long)(m.qf + m.qs) * P;
  R dphi = R(0), dU = R(0), drho = R(0);
  R mo[3] = {R(0), R(0), R(0)};
  if (m.dim == 2) {
    for (int a = 0; a < 9; ++a) {
      dU += Pop<T>::template ld<R>(pg + a * P + j);
      dphi += Pop<T>::template ld<R>(ph_ + a * P + j);
    }
    if (m.flow) {
      for (int a = 0; a < 9; ++a) {
        const R v = Pop<T>::template ld<R>(pf + a * P + j);
        drho += v;
        mo[0] += R(D2_CX[a]) * v;
        mo[1] += R(D2_CY[a]) * v;
      }
    }
  } else {
    for (int a = 0; a < 7; ++a) {
      dU += Pop<T>::template ld<R>(pg + a * P + j);
      dphi += Pop<T>::template ld<R>(ph_ + a * P + j);
    }
    if (m.flow) {
      for (int a = 0; a < 19; ++a) {
        const R v = Pop<T>::template ld<R>(pf + a * P + j);
        drho += v;
        mo[0] += R(D3_CX[a]) * v;
        mo[1] += R(D3_CY[a]) * v;
        mo[2] += R(D3_CZ[a]) * v;
      }
    }
  }
  const Coef<R>& c = coef<R>(m);
  phi = c.ref_h + dphi;
  U = (uref ? R(__half2float(uref[j])) : c.ref_g) + dU;  // per-node g reference where it is stored so
  rho = c.ref_f + drho;
  const R ph = phi < R(-1) ? R(-1) : (phi > R(1) ? R(1) : phi);
  const R K = m.flow ? c.kdrag * (R(1) + ph) * (R(1) + ph) * (R(1) - ph) : R(0);
  const R inv = R(1) / (rho + R(0.5) * K);
  for (int d = 0; d < 3; ++d) u[d] = m.flow ? (mo[d] + R(0.5) * c.body[d]) * inv : R(0);
}

template <typename T, typename R, typename O>
__global__ void fields_kernel(const Model m, const T* pops, const R* phi_prev,
                              const __half* uref, unsigned mask, O* out) {
  const long long n = (long long)m.nx * m.ny * m.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    node_xyz(m, i, x, y, z);
    const long long j = pitched(m, x, y, z);
    R phi, U, rho, u[3];
    node_moments<T, R>(m, pops, j, phi, U, rho, u, uref);
    // phi(t-1) = -1 + ring, formed in the output precision
    const O vals[7] = {O(phi), O(U), O(rho), O(u[0]), O(u[1]), O(u[2]),
                       O(m.ref_h) + O(phi_prev[j])};
    int slot = 0;
    for (int b = 0; b < 7; ++b)
      if (mask & (1u << b)) out[(long long)(slot++) * n + i] = vals[b];
  }
}

constexpr int kDiagBlocks = 152 * 4;
constexpr int kDiagThreads = 256;
constexpr int kDiagSlots = 5;  // sum(U + phi_prev), sum(rho), solid, max|u|, nonfinite

template <typename T, typename R>
__global__ void __launch_bounds__(kDiagThreads)
    diag_partial_kernel(const Model m, const T* pops, const R* phi_prev, const __half* uref,
                        double* partials) {
  const long long n = (long long)m.nx * m.ny * m.nz;
  double acc[kDiagSlots] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    node_xyz(m, i, x, y, z);
    const long long j = pitched(m, x, y, z);
    R phi, U, rho, u[3];
    node_moments<T, R>(m, pops, j, phi, U, rho, u, uref);
    // FP64 accumulation of per-node values formed in the step's arithmetic
    const double pp = m.ref_h + double(phi_prev[j]);
    const R ph = phi < R(-1) ? R(-1) : (phi > R(1) ? R(1) : phi);
    acc[0] += double(U) + pp;
    acc[1] += double(rho);
    acc[2] += 0.5 * (1.0 + double(ph));
    const double um = double(sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
    acc[3] = um > acc[3] ? um : acc[3];
    if (!(finite_r(phi) && finite_r(U) && finite_r(rho))) acc[4] += 1.0;
  }
  __shared__ double sh[kDiagSlots][kDiagThreads];
  for (int k = 0; k < kDiagSlots; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < kDiagSlots; ++k) {
        const double o = sh[k][threadIdx.x + w];
        sh[k][threadIdx.x] = k == 3 ? (o > sh[k][threadIdx.x] ? o : sh[k][threadIdx.x])
                                    : sh[k][threadIdx.x] + o;
      }
    __syncthreads();
  }
  if (threadIdx.x < kDiagSlots) partials[blockIdx.x * kDiagSlots + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kDiagThreads)
    diag_final_kernel(const double* partials, int nblocks, double* out) {
  __shared__ double sh[kDiagSlots][kDiagThreads];
  double acc[kDiagSlots] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int k = 0; k < kDiagSlots; ++k) {
      const double v = partials[b * kDiagSlots + k];
      acc[k] = k == 3 ? (v > acc[k] ? v : acc[k]) : acc[k] + v;
    }
  for (int k = 0; k < kDiagSlots; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < kDiagSlots; ++k) {
        const double o = sh[k][threadIdx.x + w];
        sh[k][threadIdx.x] = k == 3 ? (o > sh[k][threadIdx.x] ? o : sh[k][threadIdx.x])
                                    : sh[k][threadIdx.x] + o;
      }
    __syncthreads();
  }
  if (threadIdx.x < kDiagSlots) out[threadIdx.x] = sh[threadIdx.x][0];
}

// phi = 0 crossing along the six axis rays from (icx, icy, icz): the first
// sign change from phi >= 0 to phi < 0, linearly interpolated; -1 if none.
template <typename T, typename R>
__global__ void crossing_kernel(const Model m, const T* pops, int icx, int icy, int icz,
                                double* out) {
  const int r = threadIdx.x;
  if (r >= 6) return;
  const int axis = r / 2, dir = (r & 1) ? -1 : 1;
  double res = -1.0;
  if (axis < m.dim) {
    const int n = axis == 0 ? m.nx : (axis == 1 ? m.ny : m.nz);
    int c[3] = {icx, icy, m.dim == 3 ? icz : 0};
    R phi, U, rho, u[3];
    node_moments<T, R>(m, pops, pitched(m, c[0], c[1], c[2]), phi, U, rho, u);
    double prev = double(phi);
    if (prev >= 0.0) {
      const int limit = m.bc[axis] == BC_PERIODIC ? n / 2 : n;
      const int start = c[axis];
      for (int d = 1; d < limit; ++d) {
        int v = start + dir * d;
        if (m.bc[axis] == BC_PERIODIC) v = ((v % n) + n) % n;
        else if (v < 0 || v >= n) break;
        c[axis] = v;
        node_moments<T, R>(m, pops, pitched(m, c[0], c[1], c[2]), phi, U, rho, u);
        if (double(phi) < 0.0) {
          res = double(d - 1) + prev / (prev - double(phi));
          break;
        }
        prev = double(phi);
      }
    }
  }
  out[5 + r] = res;
}

// Learned block propagator, 2D: the network input (phi, U, ux, uy), each as
// (f - shift) / scale, NHWC with H = ny and W = nx; and the same four fields
// plus rho unnormalised as planes of n values (skipped if F is null).
template <typename T, typename R>
__global__ void surrogate_gather_kernel(const Model m, const T* pops, const __half* uref,
                                        const Vec4 shift,
                                        const Vec4 inv_scale, float* x, float* F) {
  const long long n = (long long)m.nx * m.ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int xx, yy, zz;
    node_xyz(m, i, xx, yy, zz);
    R phi, U, rho, u[3];
    node_moments<T, R>(m, pops, pitched(m, xx, yy, 0), phi, U, rho, u, uref);
    const float f[4] = {float(phi), float(U), float(u[0]), float(u[1])};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      x[i * 4 + c] = (f[c] - shift.v[c]) * inv_scale.v[c];
      if (F) F[c * n + i] = f[c];
    }
    if (F) F[4 * n + i] = float(rho);
  }
}

// Replace the state by the equilibrium of the fields in planes F1 (phi, U,
// ux, uy, phi(t-1)) and rho, as the fields initialisation does.
template <typename T, typename R>
__global__ void surrogate_commit_kernel(const Model m, const float* F1, const float* rho, T* pops,
                                        R* phi_prev) {
  const long long n = (long long)m.nx * m.ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int xx, yy, zz;
    node_xyz(m, i, xx, yy, zz);
    const long long j = pitched(m, xx, yy, 0);
    store_equilibrium_r<T, R>(m, pops, j, R(F1[i]), R(F1[n + i]), R(rho[i]), R(F1[2 * n + i]),
                              R(F1[3 * n + i]));
    phi_prev[j] = R(F1[4 * n + i]) - coef<R>(m).ref_h;
  }
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return int(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

template <typename T, typename R>
cudaError_t init_seed_t(const Model& m, const SeedArgs& a, void* pops, void* pp, cudaStream_t s) {
  const long long n = (long long)m.nx * m.ny * m.nz;
  init_seed_kernel<T, R><<<grid_for(n), 256, 0, s>>>(m, a, static_cast<T*>(pops),
                                                     static_cast<R*>(pp));
  return cudaGetLastError();
}
template <typename T, typename R>
cudaError_t init_polygon_t(const Model& m, const PolygonArgs& a, void* pops, void* pp,
                           cudaStream_t s) {
  const long long n = (long long)m.nx * m.ny;
  init_polygon_kernel<T, R><<<grid_for(n), 256, 0, s>>>(m, a, static_cast<T*>(pops),
                                                        static_cast<R*>(pp));
  return cudaGetLastError();
}
template <typename T, typename R>
cudaError_t solid_sync_t(const Model& m, void* const pops[2], void* const rings[2], int c,
                         cudaStream_t s) {
  const long long n = (long long)m.nx * m.ny * m.nz;
  __half* u = m.rel_g ? m.uring : nullptr;
  solid_sync_kernel<T, R><<<grid_for(n), 256, 0, s>>>(
      m, static_cast<const T*>(pops[c]), static_cast<T*>(pops[c ^ 1]),
      static_cast<const R*>(rings[c]), static_cast<R*>(rings[c ^ 1]),
      u ? u + size_t(c) * size_t(m.plane) : nullptr,
      u ? u + size_t(c ^ 1) * size_t(m.plane) : nullptr);
  return cudaGetLastError();
}
template <typename T, typename R>
cudaError_t init_fields_t(const Model& m, const double* phi, const double* U, const double* rho,
                          const double* ux, const double* uy, const double* uz, void* pops,
                          void* pp, cudaStream_t s) {
  const long long n = (long long)m.nx * m.ny * m.nz;
  init_fields_kernel<T, R><<<grid_for(n), 256, 0, s>>>(m, phi, U, rho, ux, uy, uz,
                                                       static_cast<T*>(pops), static_cast<R*>(pp));
  return cudaGetLastError();
}
template <typename T, typename R>
cudaError_t fields_t(const Model& m, const void* pops, const void* pp, const __half* uref,
                     unsigned mask, int fp64, void* out, cudaStream_t s) {
  const long long n = (long long)m.nx * m.ny * m.nz;
  if (fp64)
    fields_kernel<T, R, double><<<grid_for(n), 256, 0, s>>>(
        m, static_cast<const T*>(pops), static_cast<const R*>(pp), uref, mask,
        static_cast<double*>(out));
  else
    fields_kernel<T, R, float><<<grid_for(n), 256, 0, s>>>(
        m, static_cast<const T*>(pops), static_cast<const R*>(pp), uref, mask,
        static_cast<float*>(out));
  return cudaGetLastError();
}
template <typename T, typename R>
cudaError_t diag_t(const Model& m, const void* pops, const void* pp, const __half* uref,
                   double* partials, double* out, int icx, int icy, int icz, cudaStream_t s) {
  diag_partial_kernel<T, R><<<kDiagBlocks, kDiagThreads, 0, s>>>(
      m, static_cast<const T*>(pops), static_cast<const R*>(pp), uref, partials);
  diag_final_kernel<<<1, kDiagThreads, 0, s>>>(partials, kDiagBlocks, out);
  crossing_kernel<T, R><<<1, 32, 0, s>>>(m, static_cast<const T*>(pops), icx, icy, icz, out);
  return cudaGetLastError();
}

template <typename T, typename R>
cudaError_t gather_t(const Model& m, const void* pops, const __half* uref, const Vec4& shift,
                     const Vec4& inv_scale, float* x, float* F, cudaStream_t s) {
  const long long n = (long long)m.nx * m.ny;
  surrogate_gather_kernel<T, R><<<grid_for(n), 256, 0, s>>>(m, static_cast<const T*>(pops), uref,
                                                            shift, inv_scale, x, F);
  return cudaGetLastError();
}
template <typename T, typename R>
cudaError_t commit_t(const Model& m, const float* F1, const float* rho, void* pops, void* pp,
                     cudaStream_t s) {
  const long long n = (long long)m.nx * m.ny;
  surrogate_commit_kernel<T, R><<<grid_for(n), 256, 0, s>>>(m, F1, rho, static_cast<T*>(pops),
                                                            static_cast<R*>(pp));
  return cudaGetLastError();
}

}  // namespace

#define LBPF_DISPATCH(FN, ...)                                          \
  switch (m.storage) {                                                  \
    case ST_FP64: return FN<double, double>(__VA_ARGS__);               \
    case ST_FP16: return FN<__half, float>(__VA_ARGS__);                \
    case ST_BF16: return FN<__nv_bfloat16, float>(__VA_ARGS__);         \
    default: return FN<float, float>(__VA_ARGS__);                      \
  }

cudaError_t launch_init_seed(const Model& m, const SeedArgs& a, void* pops, void* phi_prev,
                             cudaStream_t s) {
  LBPF_DISPATCH(init_seed_t, m, a, pops, phi_prev, s)
}
cudaError_t launch_init_polygon(const Model& m, const PolygonArgs& a, void* pops,
                                void* phi_prev, cudaStream_t s) {
  if (m.dim != 2 || a.k < 1 || a.k > kMaxFacets) return cudaErrorInvalidValue;
  LBPF_DISPATCH(init_polygon_t, m, a, pops, phi_prev, s)
}
cudaError_t launch_solid_sync(const Model& m, void* const pops[2], void* const rings[2], int c,
                              cudaStream_t s) {
  if (!m.solid) return cudaErrorInvalidValue;
  LBPF_DISPATCH(solid_sync_t, m, pops, rings, c, s)
}
cudaError_t launch_init_fields(const Model& m, const double* phi, const double* U,
                               const double* rho, const double* ux, const double* uy,
                               const double* uz, void* pops, void* phi_prev, cudaStream_t s) {
  LBPF_DISPATCH(init_fields_t, m, phi, U, rho, ux, uy, uz, pops, phi_prev, s)
}
cudaError_t launch_fields(const Model& m, const void* pops, const void* phi_prev, int c,
                          unsigned mask, int fp64, void* out, cudaStream_t s) {
  const __half* uref = uref_plane(m, c);
  LBPF_DISPATCH(fields_t, m, pops, phi_prev, uref, mask, fp64, out, s)
}
cudaError_t launch_surrogate_gather(const Model& m, const void* pops, int c, const Vec4& shift,
                                    const Vec4& scale, float* x, float* F, cudaStream_t s) {
  if (m.dim != 2) return cudaErrorInvalidValue;
  Vec4 inv;
  for (int k = 0; k < 4; ++k) inv.v[k] = 1.0f / scale.v[k];
  const __half* uref = uref_plane(m, c);
  LBPF_DISPATCH(gather_t, m, pops, uref, shift, inv, x, F, s)
}
cudaError_t launch_surrogate_commit(const Model& m, const float* F1, const float* rho, void* pops,
                                    void* phi_prev, cudaStream_t s) {
  if (m.dim != 2) return cudaErrorInvalidValue;
  LBPF_DISPATCH(commit_t, m, F1, rho, pops, phi_prev, s)
}
size_t diag_partials_bytes(const Model&) { return sizeof(double) * kDiagBlocks * kDiagSlots; }
cudaError_t launch_diag(const Model& m, const void* pops, const void* phi_prev, int c,
                        double* partials, double* out, int icx, int icy, int icz, cudaStream_t s) {
  const __half* uref = uref_plane(m, c);
  LBPF_DISPATCH(diag_t, m, pops, phi_prev, uref, partials, out, icx, icy, icz, s)
}

}  // namespace lbk
