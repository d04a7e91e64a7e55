// Fused coupled LB step in 3D: D3Q19 flow f (Eqs. 4-12), D3Q7 solute g
// (Eqs. 13-18) and D3Q7 phase field h (Eqs. 19-23), push streaming (same
// update as the pull form of the equations).  Per node and step the HBM
// traffic is 33 populations read + 33 written + the phi ring read and written
// (272 B in FP32, 140 B with 16-bit populations).  grad(phi) uses the D3Q19
// stencil; phi(t) and the destination's old h of Eq. 19 come from a one-node
// halo in shared memory.  Populations are deviations d_a = p_a - w_a M_ref
// as in 2D; the ring holds phi + 1.
//
// step3d_march_kernel (FP32 arithmetic: FP32, FP16 and BF16 storage): a CTA
// walks a column of nodes along z with a ring of h / phi planes in shared
// memory (below).  step3d_kernel (FP64): one thread per node, one 16 x 4 x 2
// tile per CTA; the tile's own populations and the halo's h are loaded by the
// CTA, then every node collides and pushes (step3d_core.cuh).  A TMA-fed
// persistent variant of the 2D design measured slower in 3D (8.2 vs 13.4
// GLUPS at 256^3): its halo box carries 3.75x the tile's h data, a quarter of
// the tiles touch an x face, and the stage size allows 2 CTAs per SM only.
#include "step3d_core.cuh"

namespace lbk {
namespace {

// ---- the 3D step kernel: one tile per CTA -------------------------------------
template <typename T, typename R, bool FLOW, bool CHM, int TX, int TY, int TZ>
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
  // with solid nodes every tile takes the general path with the mask (this
  // kernel is the FP64 parity path; the FP32 one keeps per-chunk flags)
  const bool solids = m.solid != nullptr;
  if (solids && m.solid[idx]) {
    ring_cur[idx] = sh_phi[tz + 1][ty + 1][tx + 1];  // a solid node keeps its state
    return;
  }
  HSlab3<R, SX, SX * SY, SX * SY * SZ> hs{&sh_h[0][tz + 1][0][0]};
  PhiSlab3<R, SX, SX * SY> pv{&sh_phi[tz + 1][0][0]};
  const bool interior = x0 >= 1 && x0 + TX <= nx - 1 && y0 >= 1 && y0 + TY <= ny - 1 &&
                        z0 >= 1 && z0 + TZ <= nz - 1;
  if (interior && !solids)
    collide_push_3d<T, R, FLOW, true, CHM>(m, x, y, z, tx + 1, ty + 1, f, g, h,
                                           sh_phi[tz + 1][ty + 1][tx + 1], dphi_prev, pv, hs,
                                           dst, ring_cur, err);
  else
    collide_push_3d<T, R, FLOW, false, CHM, true>(m, x, y, z, tx + 1, ty + 1, f, g, h,
                                                  sh_phi[tz + 1][ty + 1][tx + 1], dphi_prev, pv,
                                                  hs, dst, ring_cur, err, solids);
}

// ---- the z-marching kernel (FP32 arithmetic) --------------------------------------
// One CTA per column of TX x TY nodes and chunk of zc planes.  The CTA walks
// its column along z; a ring of four halo-extended planes of h and phi + 1
// lives in shared memory, so every h plane of the column is read once (the
// x/y halo is (TX + 2)(TY + 2) / (TX TY) of the plane) instead of the
// three-plane-deep halo box of the tile kernel.  Each iteration first issues
// the loads of the node's own f, g and phi(t-1), then loads plane z + 1 into
// the ring, synchronises once and collides / pushes plane z.  With four
// slots, the slot filled at z + 1 is never one another thread may still read.
// MASK: the variant with solid nodes; a chunk whose flag (m.solid_tiles, one
// per column and chunk) says that it or its one-node halo holds a solid node
// takes the general path with the mask.
//
// 16-bit storage keeps g relative to a per-node U (two FP16 planes, as in
// the 2D step): the node's own reference is read from plane c, its new U
// written there, and every pushed g is encoded against the destination's
// reference in plane c ^ 1, carried in a third ring of halo-extended planes.
template <typename T, bool FLOW, bool CHM, int TX, int TY, int MINB, bool MASK>
__global__ void __launch_bounds__(TX* TY, MINB)
    step3d_march_kernel(const Model m, const T* __restrict__ src, T* __restrict__ dst,
                        const float* __restrict__ ring_prev, float* __restrict__ ring_cur,
                        unsigned* __restrict__ err, int zc, int c) {
  using R = float;
  constexpr int SX = TX + 2, SY = TY + 2, PL = SX * SY;
  constexpr int QF = FLOW ? 19 : 0;
  constexpr int NT = TX * TY;
  constexpr bool REL = sizeof(T) == 2;
  __shared__ R sh_phi[4][PL];
  __shared__ R sh_h[4][7 * PL];
  __shared__ __half sh_u[REL ? 4 : 1][REL ? PL : 1];
  const __half* uref_own = REL ? m.uring + size_t(c) * size_t(m.plane) : nullptr;
  const __half* uref_enc = REL ? m.uring + size_t(c ^ 1) * size_t(m.plane) : nullptr;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int nx = m.nx, ny = m.ny, nz = m.nz, px = m.px;
  const int P = int(m.plane);
  const int slab = ny * px;
  const int zs = blockIdx.z * zc;
  const int ze = zs + zc < nz ? zs + zc : nz;
  const int x = x0 + tx, y = y0 + ty;
  const bool active = x < nx && y < ny;
  const bool xy_inner = x0 >= 1 && x0 + TX <= nx - 1 && y0 >= 1 && y0 + TY <= ny - 1;
  const bool solids =
      MASK && m.solid &&
      m.solid_tiles[(size_t(blockIdx.z) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x];

  // the in-plane offsets of this thread's positions of the halo-extended
  // plane (the same on every plane of the column)
  constexpr int NPOS = (PL + NT - 1) / NT;
  int jxy[NPOS];
#pragma unroll
  for (int r = 0; r < NPOS; ++r) {
    const int i = tid + r * NT;
    const int lx = i % SX, ly = i / SX;
    const int gx = grad_coord(x0 + lx - 1, nx, m.bc[0]);
    const int gy = grad_coord(y0 + ly - 1, ny, m.bc[1]);
    jxy[r] = i < PL ? gy * px + gx : 0;
  }
  // h and phi + 1 of plane zz (ghost planes by the gradient rule) into slot
  auto load_plane = [&](int zz, int slot) {
    const int gz = grad_coord(zz, nz, m.bc[2]);
#pragma unroll
    for (int r = 0; r < NPOS; ++r) {
      const int i = tid + r * NT;
      if (i >= PL) break;
      const int j = gz * slab + jxy[r];
      R s = R(0);
#pragma unroll
      for (int a = 0; a < 7; ++a) {
        const R v = Pop<T>::template ld<R>(src + ((QF + 7 + a) * P + j));
        sh_h[slot][a * PL + i] = v;
        s += v;
      }
      sh_phi[slot][i] = s;
      if (REL) sh_u[slot][i] = uref_enc[j];
    }
  };

  load_plane(zs - 1, 0);
  load_plane(zs, 1);
  for (int z = zs; z < ze; ++z) {
    const int k = z - zs;
    const int sm = k & 3, s0 = (k + 1) & 3, sp = (k + 2) & 3;  // planes z - 1, z, z + 1
    const int idx = z * slab + y * px + x;
    R f[19], g[7], h[7];
    R dphi_prev = R(0);
    float uown = 0.f;
    if (active) {
#pragma unroll
      for (int a = 0; a < 19; ++a)
        if (FLOW) f[a] = Pop<T>::template ld<R>(src + (a * P + idx));
#pragma unroll
      for (int a = 0; a < 7; ++a) g[a] = Pop<T>::template ld<R>(src + ((QF + a) * P + idx));
      dphi_prev = ring_prev[idx];
      if (REL) uown = __half2float(uref_own[idx]);
    }
    load_plane(z + 1, sp);
    __syncthreads();
    if (active) {
      const int o = (ty + 1) * SX + tx + 1;
      if (MASK && solids && m.solid[idx]) {
        ring_cur[idx] = sh_phi[s0][o];  // a solid node keeps its state
        continue;
      }
#pragma unroll
      for (int a = 0; a < 7; ++a) h[a] = sh_h[s0][a * PL + o];
      PhiRing3<R, SX> pv{{sh_phi[sm], sh_phi[s0], sh_phi[sp]}};
      HRing3<R, SX, PL> hv{{sh_h[sm], sh_h[s0], sh_h[sp]}};
      // the encoding references of the three planes; uref_own's plane c
      // receives the node's new U (its own value was read above)
      UView3<REL, SX> uh{{sh_u[REL ? sm : 0], sh_u[REL ? s0 : 0], sh_u[REL ? sp : 0]},
                         const_cast<__half*>(uref_own), uown};
      if (!solids && xy_inner && z >= 1 && z <= nz - 2)
        collide_push_3d<T, R, FLOW, true, CHM, false>(m, x, y, z, tx + 1, ty + 1, f, g, h,
                                                      sh_phi[s0][o], dphi_prev, pv, hv, dst,
                                                      ring_cur, err, false, uh);
      else
        collide_push_3d<T, R, FLOW, false, CHM, MASK>(m, x, y, z, tx + 1, ty + 1, f, g, h,
                                                      sh_phi[s0][o], dphi_prev, pv, hv, dst,
                                                      ring_cur, err, solids, uh);
    }
  }
}

// Column 32 x 4, chunks of 8 planes, 4 CTAs per SM: measured at 256^3 FP32
// against 32 x 8 / 32 x 2 columns, chunks of 4 to 64 planes and 1 to 8 CTAs
// per SM (16.7 GLUPS here; 32-plane chunks of 32 x 8 columns 14.6, the tile
// kernel 13.3): short chunks keep enough CTAs in flight, the two extra planes
// per chunk cost less than that gains.
#ifndef LBPF_3D_TY
#define LBPF_3D_TY 4
#endif
#ifndef LBPF_3D_ZC
#define LBPF_3D_ZC 8
#endif
#ifndef LBPF_3D_MINB
#define LBPF_3D_MINB 4
#endif

constexpr int k3TX = 32, k3TY = LBPF_3D_TY, k3ZC = LBPF_3D_ZC;

template <typename T, bool FLOW>
cudaError_t launch3_march_t(const Model& m, int c, const void* src, void* dst,
                            const void* ring_prev, void* ring_cur, unsigned* err,
                            cudaStream_t s) {
  if (sizeof(T) == 2 && !m.uring) return cudaErrorInvalidValue;
  constexpr int TX = k3TX, TY = k3TY;
  const int zc = k3ZC;
  dim3 grid((m.nx + TX - 1) / TX, (m.ny + TY - 1) / TY, (m.nz + zc - 1) / zc);
  auto kern =
      m.solid ? (FLOW && m.chm ? step3d_march_kernel<T, FLOW, FLOW, TX, TY, LBPF_3D_MINB, true>
                               : step3d_march_kernel<T, FLOW, false, TX, TY, LBPF_3D_MINB, true>)
              : (FLOW && m.chm ? step3d_march_kernel<T, FLOW, FLOW, TX, TY, LBPF_3D_MINB, false>
                               : step3d_march_kernel<T, FLOW, false, TX, TY, LBPF_3D_MINB, false>);
  kern<<<grid, TX * TY, 0, s>>>(m, static_cast<const T*>(src), static_cast<T*>(dst),
                                static_cast<const float*>(ring_prev),
                                static_cast<float*>(ring_cur), err, zc, c);
  return cudaGetLastError();
}

// one thread per column chunk of the z-marching kernel: does the chunk or its
// one-node halo (mapped like the gradient stencil) hold a solid node?
__global__ void solid_chunks_kernel(const Model m, unsigned char* flags, int ntx, int nty,
                                    int nzc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntx * nty * nzc) return;
  const int x0 = (t % ntx) * k3TX, y0 = ((t / ntx) % nty) * k3TY, z0 = (t / (ntx * nty)) * k3ZC;
  bool any = false;
  for (int lz = -1; lz <= k3ZC && !any; ++lz)
    for (int ly = -1; ly <= k3TY && !any; ++ly)
      for (int lx = -1; lx <= k3TX && !any; ++lx)
        any = solid_mapped3(m, x0 + lx, y0 + ly, z0 + lz);
  flags[t] = any ? 1 : 0;
}

// ---- host side -------------------------------------------------------------------
template <typename T, typename R, bool FLOW>
cudaError_t launch3_plain_t(const Model& m, const void* src, void* dst, const void* ring_prev,
                            void* ring_cur, unsigned* err, cudaStream_t s) {
  constexpr int TX = sizeof(R) == 8 ? 16 : 32, TY = 4, TZ = 2;
  dim3 block(TX, TY, TZ);
  dim3 grid((m.nx + TX - 1) / TX, (m.ny + TY - 1) / TY, (m.nz + TZ - 1) / TZ);
  auto kern = FLOW && m.chm ? step3d_kernel<T, R, FLOW, FLOW, TX, TY, TZ>
                            : step3d_kernel<T, R, FLOW, false, TX, TY, TZ>;
  kern<<<grid, block, 0, s>>>(m, static_cast<const T*>(src), static_cast<T*>(dst),
                              static_cast<const R*>(ring_prev), static_cast<R*>(ring_cur), err);
  return cudaGetLastError();
}

}  // namespace

size_t solid_chunk_count(const Model& m) {
  return size_t((m.nx + k3TX - 1) / k3TX) * size_t((m.ny + k3TY - 1) / k3TY) *
         size_t((m.nz + k3ZC - 1) / k3ZC);
}

cudaError_t launch_solid_chunks(const Model& m, unsigned char* flags, cudaStream_t s) {
  if (m.dim != 3 || !m.solid) return cudaErrorInvalidValue;
  const int ntx = (m.nx + k3TX - 1) / k3TX, nty = (m.ny + k3TY - 1) / k3TY,
            nzc = (m.nz + k3ZC - 1) / k3ZC;
  const int n = ntx * nty * nzc;
  solid_chunks_kernel<<<(n + 127) / 128, 128, 0, s>>>(m, flags, ntx, nty, nzc);
  return cudaGetLastError();
}

cudaError_t prepare_step3d(const Model&, void* const[2], void* const[2], StepMaps* out) {
  out->ready = 0;  // the 3D kernel needs no tensor maps
  return cudaSuccess;
}

cudaError_t launch_step3d(const Model& m, const StepMaps&, int c, const void* src, void* dst,
                          const void* ring_prev, void* ring_cur, unsigned* err, cudaStream_t s) {
  switch (m.storage) {
    case ST_FP64:
      return m.flow ? launch3_plain_t<double, double, true>(m, src, dst, ring_prev, ring_cur, err, s)
                    : launch3_plain_t<double, double, false>(m, src, dst, ring_prev, ring_cur, err, s);
    case ST_FP16:
      return m.flow ? launch3_march_t<__half, true>(m, c, src, dst, ring_prev, ring_cur, err, s)
                    : launch3_march_t<__half, false>(m, c, src, dst, ring_prev, ring_cur, err, s);
    case ST_BF16:
      return m.flow ? launch3_march_t<__nv_bfloat16, true>(m, c, src, dst, ring_prev, ring_cur, err, s)
                    : launch3_march_t<__nv_bfloat16, false>(m, c, src, dst, ring_prev, ring_cur, err, s);
    default:
      return m.flow ? launch3_march_t<float, true>(m, c, src, dst, ring_prev, ring_cur, err, s)
                    : launch3_march_t<float, false>(m, c, src, dst, ring_prev, ring_cur, err, s);
  }
}

}  // namespace lbk
