// Fused coupled LB step in 3D: D3Q19 flow f (Eqs. 4-12), D3Q7 solute g
// (Eqs. 13-18) and D3Q7 phase field h (Eqs. 19-23), push streaming (same
// update as the pull form of the equations).  Per node and step the HBM
// traffic is 33 populations read + 33 written + the phi ring read and written
// (272 B in FP32, 140 B with 16-bit populations).  grad(phi) uses the D3Q19
// stencil; phi(t) and the destination's old h of Eq. 19 come from a one-node
// halo in shared memory.  Populations are deviations d_a = p_a - w_a M_ref
// as in 2D; the ring holds phi + 1.
//
// step3d_kernel: one thread per node, one 32 x 4 x 2 tile per CTA (16 x 4 x 2
// in FP64); the tile's own populations and the halo's h are loaded by the CTA,
// then every node collides and pushes (step3d_core.cuh).  A TMA-fed
// persistent variant of the 2D design measured slower in 3D (8.2 vs 13.4
// GLUPS at 256^3): its halo box carries 3.75x the tile's h data, a quarter of
// the tiles touch an x face, and the stage size allows 2 CTAs per SM only.
#include "step3d_core.cuh"

namespace lbk {
namespace {

// ---- the 3D step kernel: one tile per CTA -------------------------------------
template <typename T, typename R, bool FLOW, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX* TY* TZ)
    step3d_kernel(const Model m, const T* __restrict__ src, T* __restrict__ dst,
                  const R* __restrict__ ring_prev, R* __restrict__ ring_cur,
                  unsigned* __restrict__ err) {
  constexpr int SX = TX + 2, SY = TY + 2, SZ = TZ + 2;
  constexpr int QF = FLOW ? 19 : 0;
  constexpr int NT = TX * TY * TZ;
  __shared__ R sh_phi[SZ][SY][SX];
  __shared__ R sh_h[7][SZ][SY][SX];

  const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
  const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
  const int nx = m.nx, ny = m.ny, nz = m.nz, px = m.px;
  const int P = int(m.plane);
  const int slab = ny * px;
  const bool active = x < nx && y < ny && z < nz;
  const int idx = z * slab + y * px + x;

  R f[19], g[7], h[7];
  R dphi_prev = R(0);
  if (active) {
#pragma unroll
    for (int a = 0; a < 19; ++a)
      if (FLOW) f[a] = Pop<T>::template ld<R>(src + (a * P + idx));
#pragma unroll
    for (int a = 0; a < 7; ++a) {
      g[a] = Pop<T>::template ld<R>(src + ((QF + a) * P + idx));
      h[a] = Pop<T>::template ld<R>(src + ((QF + 7 + a) * P + idx));
    }
    dphi_prev = ring_prev[idx];
    R s = R(0);
#pragma unroll
    for (int a = 0; a < 7; ++a) {
      s += h[a];  // Eq. 22: phi = -1 + sum d_h
      sh_h[a][tz + 1][ty + 1][tx + 1] = h[a];
    }
    sh_phi[tz + 1][ty + 1][tx + 1] = s;
  }
  const int tid = (tz * TY + ty) * TX + tx;
  for (int i = tid; i < SX * SY * SZ; i += NT) {
    const int lx = i % SX, ly = (i / SX) % SY, lz = i / (SX * SY);
    int gx = x0 + lx - 1, gy = y0 + ly - 1, gz = z0 + lz - 1;
    if (lx >= 1 && lx <= TX && ly >= 1 && ly <= TY && lz >= 1 && lz <= TZ && gx < nx &&
        gy < ny && gz < nz)
      continue;
    gx = grad_coord(gx, nx, m.bc[0]);
    gy = grad_coord(gy, ny, m.bc[1]);
    gz = grad_coord(gz, nz, m.bc[2]);
    const int j = gz * slab + gy * px + gx;
    R s = R(0);
#pragma unroll
    for (int a = 0; a < 7; ++a) {
      const R v = Pop<T>::template ld<R>(src + ((QF + 7 + a) * P + j));
      sh_h[a][lz][ly][lx] = v;
      s += v;
    }
    sh_phi[lz][ly][lx] = s;
  }
  __syncthreads();
  if (!active) return;
  TileView3<R, R, SX, SX * SY, SX * SY * SZ, 0> hs{&sh_h[0][0][0][0]};
  const bool interior = x0 >= 1 && x0 + TX <= nx - 1 && y0 >= 1 && y0 + TY <= ny - 1 &&
                        z0 >= 1 && z0 + TZ <= nz - 1;
  if (interior)
    collide_push_3d<T, R, FLOW, true, SX, SX * SY>(m, x, y, z, tx + 1, ty + 1, tz + 1, f, g, h,
                                                   sh_phi[tz + 1][ty + 1][tx + 1], dphi_prev,
                                                   &sh_phi[0][0][0], hs, dst, ring_cur, err);
  else
    collide_push_3d<T, R, FLOW, false, SX, SX * SY>(m, x, y, z, tx + 1, ty + 1, tz + 1, f, g, h,
                                                    sh_phi[tz + 1][ty + 1][tx + 1], dphi_prev,
                                                    &sh_phi[0][0][0], hs, dst, ring_cur, err);
}

// ---- host side -------------------------------------------------------------------
template <typename T, typename R, bool FLOW>
cudaError_t launch3_plain_t(const Model& m, const void* src, void* dst, const void* ring_prev,
                            void* ring_cur, unsigned* err, cudaStream_t s) {
  constexpr int TX = sizeof(R) == 8 ? 16 : 32, TY = 4, TZ = 2;
  dim3 block(TX, TY, TZ);
  dim3 grid((m.nx + TX - 1) / TX, (m.ny + TY - 1) / TY, (m.nz + TZ - 1) / TZ);
  step3d_kernel<T, R, FLOW, TX, TY, TZ><<<grid, block, 0, s>>>(
      m, static_cast<const T*>(src), static_cast<T*>(dst), static_cast<const R*>(ring_prev),
      static_cast<R*>(ring_cur), err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_step3d(const Model&, void* const[2], void* const[2], StepMaps* out) {
  out->ready = 0;  // the 3D kernel needs no tensor maps
  return cudaSuccess;
}

cudaError_t launch_step3d(const Model& m, const StepMaps&, int, const void* src, void* dst,
                          const void* ring_prev, void* ring_cur, unsigned* err, cudaStream_t s) {
  switch (m.storage) {
    case ST_FP64:
      return m.flow ? launch3_plain_t<double, double, true>(m, src, dst, ring_prev, ring_cur, err, s)
                    : launch3_plain_t<double, double, false>(m, src, dst, ring_prev, ring_cur, err, s);
    case ST_FP16:
      return m.flow ? launch3_plain_t<__half, float, true>(m, src, dst, ring_prev, ring_cur, err, s)
                    : launch3_plain_t<__half, float, false>(m, src, dst, ring_prev, ring_cur, err, s);
    case ST_BF16:
      return m.flow
                 ? launch3_plain_t<__nv_bfloat16, float, true>(m, src, dst, ring_prev, ring_cur, err, s)
                 : launch3_plain_t<__nv_bfloat16, float, false>(m, src, dst, ring_prev, ring_cur, err, s);
    default:
      return m.flow ? launch3_plain_t<float, float, true>(m, src, dst, ring_prev, ring_cur, err, s)
                    : launch3_plain_t<float, float, false>(m, src, dst, ring_prev, ring_cur, err, s);
  }
}

}  // namespace lbk
