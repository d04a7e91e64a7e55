// Device helpers of liblbpf.so: lattice constants, population storage
// codecs and the anisotropy function.  Internal to the CUDA library.
#pragma once

#include "lbpf_internal.cuh"

namespace lbk {

// ---- lattices (direction order of the exported state) ----------------------
// D2Q9: (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
__device__ constexpr int D2_CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ constexpr int D2_CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__device__ constexpr int D2_OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
// Weights.  In FP32 the three values are chosen so that their exact sum
// (w0 + 4 w1 + 4 w2, resp. w0 + 6 w1 + 12 w2) is 1: with the rounded 4/9, 1/9,
// 1/36 the sum is 1 + 7.4e-9, which biases every zeroth moment by that much
// per collision (sum of U + phi(t-1) drifts; phi drifts by ~1e-8 per step).
// FP64 uses the plain fractions.
template <typename R>
__device__ __forceinline__ R d2_w(int a);
template <>
__device__ __forceinline__ double d2_w<double>(int a) {
  return a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}
template <>
__device__ __forceinline__ float d2_w<float>(int a) {
  return a == 0 ? 0x1.c71c72p-2f : (a < 5 ? 0x1.c71c72p-4f : 0x1.c71c70p-6f);
}

// D3Q19: rest, +x, -x, +y, -y, +z, -z, then the 12 edge links; D3Q7 is the
// first seven of these.
__device__ constexpr int D3_CX[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__device__ constexpr int D3_CY[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__device__ constexpr int D3_CZ[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
__device__ constexpr int D3_OPP[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
template <typename R>
__device__ __forceinline__ R d3q19_w(int a);
template <>
__device__ __forceinline__ double d3q19_w<double>(int a) {
  return a == 0 ? 1.0 / 3.0 : (a < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
}
template <>
__device__ __forceinline__ float d3q19_w<float>(int a) {
  return a == 0 ? 0x1.555558p-2f : (a < 7 ? 0x1.c71c72p-5f : 0x1.c71c6ep-6f);
}
template <typename R>
__device__ __forceinline__ R d3q7_w(int a) {
  return a == 0 ? R(0.25) : R(0.125);
}

// ---- arithmetic helpers -------------------------------------------------------
__device__ __forceinline__ float rsqrt_r(float v) { return rsqrtf(v); }
// Reciprocal of the per-node relaxation and velocity denominators (all in
// [0.5, ~10]): in FP32 the hardware approximation (2 ulp) instead of the
// IEEE-exact division sequence; in FP64 the exact division.
__device__ __forceinline__ float rcp_r(float v) { return __fdividef(1.0f, v); }
__device__ __forceinline__ double rcp_r(double v) { return 1.0 / v; }
__device__ __forceinline__ double rsqrt_r(double v) { return rsqrt(v); }
template <typename R>
__device__ __forceinline__ R clamp1(R v) {
  return v < R(-1) ? R(-1) : (v > R(1) ? R(1) : v);
}
__device__ __forceinline__ bool finite_r(float v) { return isfinite(v); }

// Explicitly rounded multiply / add / fused multiply-add.  The values a node
// pushes are written with these so that the compiler cannot fuse them
// differently in different code paths (interior vs edge tiles, single vs
// batched kernels): every path then rounds identically and a node's result
// does not depend on how the grid was tiled.
__device__ __forceinline__ float fma_r(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_r(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_r(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_r(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_r(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_r(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ bool finite_r(double v) { return isfinite(v); }

// ---- population storage ---------------------------------------------------------
// Every lattice stores and updates the deviation of its populations from the
// weights times a reference moment, d_a = p_a - w_a M_ref (M_ref = 1 for f,
// U_ref for g, -1 for h), so that rounding acts on small numbers: the moments
// are M = M_ref + sum d and the equilibria are written as deviations too.
// FP32/FP64 store d as is; the 16-bit modes store d rounded to binary16 or
// bfloat16 and compute in FP32.
template <typename T>
struct Pop;
template <>
struct Pop<float> {
  template <typename R>
  __device__ static __forceinline__ R ld(const float* p) { return R(*p); }
  template <typename R>
  __device__ static __forceinline__ void st(float* p, R v) { *p = float(v); }
};
template <>
struct Pop<double> {
  template <typename R>
  __device__ static __forceinline__ R ld(const double* p) { return R(*p); }
  template <typename R>
  __device__ static __forceinline__ void st(double* p, R v) { *p = double(v); }
};
template <>
struct Pop<__half> {
  template <typename R>
  __device__ static __forceinline__ R ld(const __half* p) { return R(__half2float(*p)); }
  template <typename R>
  __device__ static __forceinline__ void st(__half* p, R v) { *p = __float2half_rn(float(v)); }
};
template <>
struct Pop<__nv_bfloat16> {
  template <typename R>
  __device__ static __forceinline__ R ld(const __nv_bfloat16* p) {
    return R(__bfloat162float(*p));
  }
  template <typename R>
  __device__ static __forceinline__ void st(__nv_bfloat16* p, R v) {
    *p = __float2bfloat16_rn(float(v));
  }
};

// ---- anisotropy (Eq. 3) and flux vector N (Eq. 21) ----------------------------
// n = -grad/|grad| (solid -> liquid).  k-fold: cos/sin(k theta) are the real and
// imaginary parts of (n_x + i n_y)^k, rotated by k theta0, so no atan2 is needed.
// N = fac |grad|^2 a_s d(a_s)/d(grad):
//   k-fold: N = fac k eps a_s sin(k(theta - theta0)) (g_y, -g_x)
//   cubic : N_i = fac 16 eps a_s |grad| (n_i S - n_i^3), S = sum n_j^4
template <typename R>
__device__ __forceinline__ void aniso(const Model& m, R gx, R gy, R gz, R& as, R& Nx, R& Ny,
                                      R& Nz) {
  as = R(1);
  Nx = Ny = Nz = R(0);
  R g2 = gx * gx + gy * gy + gz * gz;
  const Coef<R>& c = coef<R>(m);
  if (!(g2 > R(1e-12)) || c.eps == R(0)) return;
  const R ig = rsqrt_r(g2);
  const R nx = -gx * ig, ny = -gy * ig, nz = -gz * ig;
  const R eps = c.eps, fac = c.aniso_fac;
  if (m.fold > 0) {
    R ck = nx, sk = ny;
    for (int j = 1; j < m.fold; ++j) {
      const R c2 = ck * nx - sk * ny;
      sk = ck * ny + sk * nx;
      ck = c2;
    }
    const R cosd = ck * c.ck0 + sk * c.sk0;
    const R sind = sk * c.ck0 - ck * c.sk0;
    as = R(1) + eps * cosd;
    const R amp = fac * R(m.fold) * eps * as * sind;
    Nx = amp * gy;
    Ny = -amp * gx;
  } else {
    const R nx2 = nx * nx, ny2 = ny * ny, nz2 = nz * nz;
    const R S = nx2 * nx2 + ny2 * ny2 + nz2 * nz2;
    as = R(1) - R(3) * eps + R(4) * eps * S;
    const R amp = fac * R(16) * eps * as * (g2 * ig);
    Nx = amp * nx * (S - nx2);
    Ny = amp * ny * (S - ny2);
    Nz = amp * nz * (S - nz2);
  }
}

// periodic wrap of a coordinate that is at most one period out of range
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
// neighbour coordinate for the gradient stencil: periodic wrap, else copy the
// nearest node (zero normal derivative)
__device__ __forceinline__ int grad_coord(int v, int n, int bc) {
  if (bc == BC_PERIODIC) return wrap1(v, n);
  return v < 0 ? 0 : (v >= n ? n - 1 : v);
}

}  // namespace lbk
