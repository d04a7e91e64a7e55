// Fused coupled LB step in 2D: D2Q9 flow f (Eqs. 4-12), D2Q9 solute g
// (Eqs. 13-18) and D2Q9 phase field h (Eqs. 19-23).
//
// Streaming is done in push form: the thread of node s holds its own
// populations, forms every moment locally, collides and writes the
// post-collision value of direction a to s + c_a.  That is the same update
// as the pull form of the paper's equations; it needs no stored macroscopic
// fields, only phi(t-1) for d(phi)/dt.  Per node and step the HBM traffic is
// 27 populations read + 27 written + phi(t-1) read + phi(t) written (224 B in
// FP32 with flow, 152 B without, 116 B with 16-bit populations).
//
// Populations are deviations d_a = p_a - w_a M_ref (M_ref = 1 for f, U_ref
// for g, -1 for h); the phi ring holds phi + 1.
//
// Two parts of the step need neighbour data, both served from shared memory:
// grad(phi) (Eq. 3, 21, 23) needs phi(t) of a one-node halo, summed from the
// halo's h populations, and Eq. 19 writes
// a_s^2 h(r + c, t+1) = h*(r) - (1 - a_s^2(r)) h(r + c, t), i.e. needs the old
// h of the destination node.
//
// step2d_tma_kernel (FP32 and 16-bit storage): persistent CTAs stream 32 x 4
// tiles through a 2-stage shared-memory pipeline, 4 CTAs of 128 threads per SM
// (tile, depth and CTAs per SM chosen by a sweep on GB300).  Per tile one thread issues
// three TMA tensor loads on one mbarrier: f and g of the tile, h of the tile
// plus halo (box starting 16 bytes left of the tile so that its innermost
// coordinate stays aligned), and the phi ring of the tile.  While a tile is
// computed and pushed, the next one is in flight.  Halo positions outside
// the domain (the TMA fills them with zeros) are patched with the mapped
// periodic / zero-gradient values on edge tiles only.
//
// step2d_kernel (FP64 storage): one thread per node, one tile per CTA, the
// same per-node code.
#include "step2d_tile.cuh"
#include "tma_host.h"

namespace lbk {
namespace {

constexpr int kSpin = 1 << 22;  // bound on mbarrier polls before giving up

// ---- FP64 (and reference) kernel: one tile per CTA ------------------------------
template <typename T, typename R, bool FLOW, int TX, int TY, bool CHM>
__global__ void __launch_bounds__(TX* TY)
    step2d_kernel(const Model m, const PopPtrs sp, const PopPtrs dp,
                  const R* __restrict__ ring_prev, R* __restrict__ ring_cur,
                  unsigned* __restrict__ err) {
  constexpr int SX = TX + 2, SY = TY + 2;
  constexpr int QF = FLOW ? 9 : 0;
  constexpr int NT = TX * TY;
  __shared__ R sh_phi[SY][SX];
  __shared__ R sh_h[9][SY][SX];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int x = x0 + tx, y = y0 + ty;
  const int nx = m.nx, ny = m.ny, px = m.px;
  const bool active = x < nx && y < ny;
  const int idx = y * px + x;

  R f[9], g[9], h[9];
  R dphi_prev = R(0);
  if (active) {
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      if (FLOW) f[a] = Pop<T>::template ld<R>(static_cast<const T*>(sp.p[a]) + idx);
      g[a] = Pop<T>::template ld<R>(static_cast<const T*>(sp.p[QF + a]) + idx);
      h[a] = Pop<T>::template ld<R>(static_cast<const T*>(sp.p[QF + 9 + a]) + idx);
    }
    dphi_prev = ring_prev[idx];
  }
  if (active) {
    R s = R(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      s += h[a];
      sh_h[a][ty + 1][tx + 1] = h[a];
    }
    sh_phi[ty + 1][tx + 1] = s;
  }
  // halo ring (and positions of a partial tile): phi and h of the mapped node
  for (int i = tid; i < SX * SY; i += NT) {
    const int lx = i % SX, ly = i / SX;
    int gx = x0 + lx - 1, gy = y0 + ly - 1;
    if (lx >= 1 && lx <= TX && ly >= 1 && ly <= TY && gx < nx && gy < ny) continue;
    gx = grad_coord(gx, nx, m.bc[0]);
    gy = grad_coord(gy, ny, m.bc[1]);
    const int j = gy * px + gx;
    R s = R(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const R v = Pop<T>::template ld<R>(static_cast<const T*>(sp.p[QF + 9 + a]) + j);
      sh_h[a][ly][lx] = v;
      s += v;
    }
    sh_phi[ly][lx] = s;
  }
  __syncthreads();
  const bool solids = m.solid && m.solid_tiles[blockIdx.y * gridDim.x + blockIdx.x];
  if (!active) return;
  if (solids && m.solid[idx]) {
    ring_cur[idx] = sh_phi[ty + 1][tx + 1];  // a solid node keeps its state
    return;
  }
  TileView<R, R, SX, SX * SY, 0> hs{&sh_h[0][0][0]};
  if (!solids && x0 >= 1 && x0 + TX <= nx - 1 && y0 >= 1 && y0 + TY <= ny - 1)
    collide_push_2d<T, R, FLOW, true, SX, true, CHM>(m, x, y, tx + 1, ty + 1, f, g, h,
                                                sh_phi[ty + 1][tx + 1], dphi_prev,
                                                &sh_phi[0][0], hs, NoUView{},
                                                static_cast<T*>(dp.p[0]), ring_cur, err);
  else
    collide_push_2d<T, R, FLOW, false, SX, true, CHM>(m, x, y, tx + 1, ty + 1, f, g, h,
                                                 sh_phi[ty + 1][tx + 1], dphi_prev,
                                                 &sh_phi[0][0], hs, NoUView{},
                                                 static_cast<T*>(dp.p[0]), ring_cur, err, solids);
}

// ---- TMA-pipelined persistent kernel ------------------------------------------

// Pipeline depth and resident CTAs per SM of the persistent kernel.
#ifndef LBPF_2D_STAGES
#define LBPF_2D_STAGES 2
#endif
#ifndef LBPF_2D_MIN_CTAS
#define LBPF_2D_MIN_CTAS 4
#endif
#ifndef LBPF_2D_TY
#define LBPF_2D_TY 4
#endif

// MASK: the variant with the solid-node path (its extra registers held to
// five CTAs per SM, which measured faster than four at more registers); CHM:
// the central Hermite MRT flow collision (likewise).  CUR: how the threads
// learn the origin of their CTA's next tile (below).
template <typename T, bool FLOW, int TX, int TY, int S, bool MASK, bool CHM,
          bool CUR = sizeof(T) == 2>
__global__ void __launch_bounds__(TX* TY, (MASK || CHM) ? 5 : LBPF_2D_MIN_CTAS)
    step2d_tma_kernel(const __grid_constant__ CUtensorMap tm_fg,
                      const __grid_constant__ CUtensorMap tm_h,
                      const __grid_constant__ CUtensorMap tm_ring,
                      const __grid_constant__ CUtensorMap tm_uown,
                      const __grid_constant__ CUtensorMap tm_uhal, const Model m,
                      const T* __restrict__ src, T* __restrict__ dst,
                      float* __restrict__ ring_cur, unsigned* __restrict__ err, int ntx,
                      int ntiles, int c) {
  using R = float;
  using L = Tiles2D<T, FLOW, TX, TY>;
  constexpr int SX = TX + 2, SY = TY + 2;
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[S];
  __shared__ R sh_phi[SY][SX];
  __shared__ int2 org[S];  // !CUR: origin of the tile in each stage
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));

  const int tid = threadIdx.x;
  const int first = blockIdx.x, G = gridDim.x;

  // The CTA's tiles are first, first + G, first + 2G, ...  Their origins
  // reach the threads without a division by ntx in every thread:
  //  - CUR (16-bit storage): every thread steps the tile's column and row by
  //    (G mod ntx, G div ntx) with one carry; thread 0 loads the tile S steps
  //    ahead of the one being computed;
  //  - otherwise (FP32): thread 0 divides once per tile it loads and writes the
  //    origin into the stage's slot of org before it arrives on the stage's
  //    mbarrier, whose completion publishes it to the other threads.
  // Same-box timings of the 1024^2 coupled step (dividing in every thread /
  // cursor / published origin): FP16 39.6 / 38.35 / 38.5 us, FP32 48.7 / 49.05
  // (two more registers) / 48.5 us.
  struct Cursor {
    int tile, col, row;
  };
  const int gcol = G % ntx, grow = G / ntx;
  auto advance = [&](Cursor& q) {
    q.tile += G;
    q.col += gcol;
    q.row += grow;
    if (q.col >= ntx) {
      q.col -= ntx;
      ++q.row;
    }
  };
  auto issue_xy = [&](int x0, int y0, int s) {
    issue_tile_2d<T, FLOW, TX, TY>(&tm_fg, &tm_h, &tm_ring, &tm_uown, &tm_uhal, c, &full[s],
                                   smem + s * L::STAGE, x0, y0);
  };
  auto issue_org = [&](int tile, int s) {  // thread 0, !CUR
    const int2 o = make_int2((tile % ntx) * TX, (tile / ntx) * TY);
    org[s] = o;
    issue_xy(o.x, o.y, s);
  };
  Cursor work{first, first % ntx, first / ntx};

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (tid == 0) {
    if constexpr (CUR) {
      Cursor q = work;
      for (int k = 0; k < S && q.tile < ntiles; ++k) {
        issue_xy(q.col * TX, q.row * TY, k);
        advance(q);
      }
    } else {
      for (int k = 0; k < S; ++k)
        if (first + k * G < ntiles) issue_org(first + k * G, k);
    }
  }

  for (int k = 0;; ++k) {
    const int tile = first + k * G;
    if (tile >= ntiles) break;
    const int s = k % S;
    const bool ok = mbar_wait_bounded(&full[s], uint32_t((k / S) & 1), kSpin);
    if (__syncthreads_or(!ok)) {
      // a tile never arrived: report, let the copies in flight land, stop
      if (tid == 0) {
        atomicOr(err, 2u);
        for (int j = 1; j < S; ++j) {
          const int kk = k + j;
          if (first + kk * G < ntiles)
            mbar_wait_bounded(&full[kk % S], uint32_t((kk / S) & 1), kSpin);
        }
      }
      __syncthreads();
      return;
    }
    int x0, y0;
    if constexpr (CUR) {
      x0 = work.col * TX;
      y0 = work.row * TY;
    } else {
      const int2 o = org[s];
      x0 = o.x;
      y0 = o.y;
    }
    tile_2d<T, FLOW, TX, TY, MASK, CHM>(m, src, dst, ring_cur, err, x0, y0, c,
                                        smem + s * L::STAGE, &sh_phi[0][0]);
    __syncthreads();  // stage s, its origin slot and sh_phi are free again
    if constexpr (CUR) {
      if (tid == 0) {
        Cursor q = work;
        for (int j = 0; j < S; ++j) advance(q);
        if (q.tile < ntiles) {
          fence_proxy_async_smem();
          issue_xy(q.col * TX, q.row * TY, s);
        }
      }
      advance(work);
    } else {
      if (tid == 0 && tile + S * G < ntiles) {
        fence_proxy_async_smem();
        issue_org(tile + S * G, s);
      }
    }
  }
}

// ---- host side: tensor maps and launches -------------------------------------------
constexpr int kTX = 32, kTY = LBPF_2D_TY, kStages = LBPF_2D_STAGES;

// one thread per kTX x kTY tile: does the tile or its one-node halo (mapped
// like the gradient stencil) hold a solid node?
__global__ void solid_tiles_kernel(const Model m, unsigned char* flags, int ntx, int nty) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntx * nty) return;
  const int x0 = (t % ntx) * kTX, y0 = (t / ntx) * kTY;
  bool any = false;
  for (int ly = -1; ly <= kTY; ++ly)
    for (int lx = -1; lx <= kTX; ++lx) any |= solid_mapped(m, x0 + lx, y0 + ly);
  flags[t] = any ? 1 : 0;
}

template <typename T, bool FLOW>
cudaError_t prepare_t(const Model& m, void* const pops[2], void* const rings[2], StepMaps* out) {
  using L = Tiles2D<T, FLOW, kTX, kTY>;
  const CUtensorMapDataType dt = pop_tensor_type(m.storage);
  const uint64_t q = uint64_t(L::QFG + 9);
  for (int b = 0; b < 2; ++b) {
    const uint64_t dims3[3] = {uint64_t(m.nx), uint64_t(m.ny), q};
    const uint64_t str3[2] = {uint64_t(m.px) * sizeof(T), uint64_t(m.plane) * sizeof(T)};
    const uint32_t box_fg[3] = {kTX, kTY, uint32_t(L::QFG)};
    const uint32_t box_h[3] = {uint32_t(L::BXH), kTY + 2, 9};
    const uint64_t dims2[2] = {uint64_t(m.nx), uint64_t(m.ny)};
    const uint64_t str2[1] = {uint64_t(m.px) * 4};
    const uint32_t box_r[2] = {kTX, kTY};
    if (!encode_tiled(&out->fg[b], dt, 3, pops[b], dims3, str3, box_fg) ||
        !encode_tiled(&out->h[b], dt, 3, pops[b], dims3, str3, box_h) ||
        !encode_tiled(&out->ring[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, rings[b], dims2, str2, box_r))
      return cudaErrorInvalidValue;
  }
  if (L::REL) {
    // the two U planes as one 3D tensor; the plane is the third coordinate
    if (!m.uring) return cudaErrorInvalidValue;
    const uint64_t dimsu[3] = {uint64_t(m.nx), uint64_t(m.ny), 2};
    const uint64_t stru[2] = {uint64_t(m.px) * 2, uint64_t(m.plane) * 2};
    const uint32_t box_uo[3] = {kTX, kTY, 1};
    const uint32_t box_uh[3] = {uint32_t(L::BXU), kTY + 2, 1};
    if (!encode_tiled(&out->uown, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, m.uring, dimsu, stru, box_uo) ||
        !encode_tiled(&out->uhal, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, m.uring, dimsu, stru, box_uh))
      return cudaErrorInvalidValue;
  } else {
    out->uown = out->ring[0];  // unused
    out->uhal = out->ring[0];
  }
  const int smem = kStages * L::STAGE + 128;
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  auto setup = [&](auto kern, int* ctas) {
    int per_sm = 0;
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (r == cudaSuccess)
      r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTX * kTY, smem);
    *ctas = sms * (per_sm > 0 ? per_sm : 1);
    return r;
  };
  if ((e = setup(step2d_tma_kernel<T, FLOW, kTX, kTY, kStages, false, false>,
                 &out->ctas_v[0])) != cudaSuccess ||
      (e = setup(step2d_tma_kernel<T, FLOW, kTX, kTY, kStages, true, false>,
                 &out->ctas_v[1])) != cudaSuccess)
    return e;
  if constexpr (FLOW) {  // the central Hermite MRT exists with flow only
    if ((e = setup(step2d_tma_kernel<T, FLOW, kTX, kTY, kStages, false, true>,
                   &out->ctas_v[2])) != cudaSuccess ||
        (e = setup(step2d_tma_kernel<T, FLOW, kTX, kTY, kStages, true, true>,
                   &out->ctas_v[3])) != cudaSuccess)
      return e;
  }
  out->ctas = out->ctas_v[0];
  out->smem = smem;
  out->ready = 1;
  return cudaSuccess;
}

template <typename T, bool FLOW>
cudaError_t launch_tma_t(const Model& m, const StepMaps& maps, int c, const void* src, void* dst,
                         void* ring_cur, unsigned* err, cudaStream_t s) {
  const int ntx = (m.nx + kTX - 1) / kTX, nty = (m.ny + kTY - 1) / kTY;
  const int ntiles = ntx * nty;
  const int v = (m.solid ? 1 : 0) + (FLOW && m.chm ? 2 : 0);
  const int grid = ntiles < maps.ctas_v[v] ? ntiles : maps.ctas_v[v];
  auto go = [&](auto kern) {
    kern<<<grid, kTX * kTY, maps.smem, s>>>(maps.fg[c], maps.h[c], maps.ring[c], maps.uown,
                                            maps.uhal, m, static_cast<const T*>(src),
                                            static_cast<T*>(dst), static_cast<float*>(ring_cur),
                                            err, ntx, ntiles, c);
  };
  if (v == 0) go(step2d_tma_kernel<T, FLOW, kTX, kTY, kStages, false, false>);
  else if (v == 1) go(step2d_tma_kernel<T, FLOW, kTX, kTY, kStages, true, false>);
  if constexpr (FLOW) {
    if (v == 2) go(step2d_tma_kernel<T, FLOW, kTX, kTY, kStages, false, true>);
    else if (v == 3) go(step2d_tma_kernel<T, FLOW, kTX, kTY, kStages, true, true>);
  }
  return cudaGetLastError();
}

template <typename T, typename R, bool FLOW>
cudaError_t launch_plain_t(const Model& m, const void* src, void* dst, const void* ring_prev,
                           void* ring_cur, unsigned* err, cudaStream_t s) {
  dim3 block(kTX, kTY);
  dim3 grid((m.nx + kTX - 1) / kTX, (m.ny + kTY - 1) / kTY);
  const PopPtrs sp = pop_ptrs(m, const_cast<void*>(src), sizeof(T));
  const PopPtrs dp = pop_ptrs(m, dst, sizeof(T));
  if (FLOW && m.chm)
    step2d_kernel<T, R, FLOW, kTX, kTY, FLOW><<<grid, block, 0, s>>>(
        m, sp, dp, static_cast<const R*>(ring_prev), static_cast<R*>(ring_cur), err);
  else
    step2d_kernel<T, R, FLOW, kTX, kTY, false><<<grid, block, 0, s>>>(
        m, sp, dp, static_cast<const R*>(ring_prev), static_cast<R*>(ring_cur), err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_step2d(const Model& m, void* const pops[2], void* const rings[2],
                           StepMaps* out) {
  out->ready = 0;
  if (m.storage == ST_FP64) return cudaSuccess;  // one-tile kernel, no maps
  switch (m.storage) {
    case ST_FP16:
      return m.flow ? prepare_t<__half, true>(m, pops, rings, out)
                    : prepare_t<__half, false>(m, pops, rings, out);
    case ST_BF16:
      return m.flow ? prepare_t<__nv_bfloat16, true>(m, pops, rings, out)
                    : prepare_t<__nv_bfloat16, false>(m, pops, rings, out);
    default:
      return m.flow ? prepare_t<float, true>(m, pops, rings, out)
                    : prepare_t<float, false>(m, pops, rings, out);
  }
}

size_t solid_tile_count(const Model& m) {
  return size_t((m.nx + kTX - 1) / kTX) * size_t((m.ny + kTY - 1) / kTY);
}

cudaError_t launch_solid_tiles(const Model& m, unsigned char* flags, cudaStream_t s) {
  if (m.dim != 2 || !m.solid) return cudaErrorInvalidValue;
  const int ntx = (m.nx + kTX - 1) / kTX, nty = (m.ny + kTY - 1) / kTY;
  solid_tiles_kernel<<<(ntx * nty + 127) / 128, 128, 0, s>>>(m, flags, ntx, nty);
  return cudaGetLastError();
}

cudaError_t launch_step2d(const Model& m, const StepMaps& maps, int c, const void* src, void* dst,
                          const void* ring_prev, void* ring_cur, unsigned* err, cudaStream_t s) {
  if (m.storage == ST_FP64)
    return m.flow ? launch_plain_t<double, double, true>(m, src, dst, ring_prev, ring_cur, err, s)
                  : launch_plain_t<double, double, false>(m, src, dst, ring_prev, ring_cur, err, s);
  if (!maps.ready) return cudaErrorNotReady;
  switch (m.storage) {
    case ST_FP16:
      return m.flow ? launch_tma_t<__half, true>(m, maps, c, src, dst, ring_cur, err, s)
                    : launch_tma_t<__half, false>(m, maps, c, src, dst, ring_cur, err, s);
    case ST_BF16:
      return m.flow ? launch_tma_t<__nv_bfloat16, true>(m, maps, c, src, dst, ring_cur, err, s)
                    : launch_tma_t<__nv_bfloat16, false>(m, maps, c, src, dst, ring_cur, err, s);
    default:
      return m.flow ? launch_tma_t<float, true>(m, maps, c, src, dst, ring_cur, err, s)
                    : launch_tma_t<float, false>(m, maps, c, src, dst, ring_cur, err, s);
  }
}

}  // namespace lbk
