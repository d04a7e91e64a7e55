// One tile of the TMA-fed 2D step, shared by the single-grid and the batched
// persistent kernels: shared-memory layout of a pipeline stage, the three TMA
// loads that fill it, and the work on a filled stage (edge patching, phi + 1
// of the halo-extended tile, per-node collide and push).
#pragma once

#include "step2d_core.cuh"
#include "tma.cuh"

namespace lbk {

template <typename T, bool FLOW, int TX, int TY>
struct Tiles2D {
  static constexpr int QFG = (FLOW ? 9 : 0) + 9;   // f and g arrays
  static constexpr int HX = 16 / int(sizeof(T));   // halo box starts HX left of the tile
  static constexpr int BXH = TX + 2 * HX;          // h box width
  static constexpr int FG_BYTES = QFG * TY * TX * int(sizeof(T));
  static constexpr int H_BYTES = 9 * (TY + 2) * BXH * int(sizeof(T));
  static constexpr int RING_BYTES = TY * TX * 4;
  static constexpr int al(int b) { return (b + 127) / 128 * 128; }
  static constexpr int OFF_H = al(FG_BYTES);
  static constexpr int OFF_RING = OFF_H + al(H_BYTES);
  static constexpr int STAGE = OFF_RING + al(RING_BYTES);
  static constexpr int TX_BYTES = FG_BYTES + H_BYTES + RING_BYTES;
};

// Fill one stage: f and g of the tile, h with its halo, the phi ring.
template <typename T, bool FLOW, int TX, int TY>
__device__ __forceinline__ void issue_tile_2d(const CUtensorMap* tm_fg, const CUtensorMap* tm_h,
                                              const CUtensorMap* tm_ring, uint64_t* bar,
                                              unsigned char* st, int x0, int y0) {
  using L = Tiles2D<T, FLOW, TX, TY>;
  mbar_arrive_expect_tx(bar, L::TX_BYTES);
  tma_load_3d(st, tm_fg, bar, x0, y0, 0);
  tma_load_3d(st + L::OFF_H, tm_h, bar, x0 - L::HX, y0 - 1, L::QFG);
  tma_load_2d(st + L::OFF_RING, tm_ring, bar, x0, y0);
}

// Work on a filled stage `st` for the tile at (x0, y0).  Called by all
// threads of the CTA; contains CTA barriers.  sh_phi: (TY + 2) x (TX + 2).
template <typename T, bool FLOW, int TX, int TY>
__device__ __forceinline__ void tile_2d(const Model& m, const T* __restrict__ src,
                                        T* __restrict__ dst, float* __restrict__ ring_cur,
                                        unsigned* __restrict__ err, int x0, int y0,
                                        unsigned char* st, float* sh_phi_flat) {
  using R = float;
  using L = Tiles2D<T, FLOW, TX, TY>;
  constexpr int NT = TX * TY, SX = TX + 2, SY = TY + 2;
  constexpr int QF = FLOW ? 9 : 0;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int nx = m.nx, ny = m.ny, px = m.px;
  R(*sh_phi)[SX] = reinterpret_cast<R(*)[SX]>(sh_phi_flat);
    const T* fgs = reinterpret_cast<const T*>(st);
    T* hsm = reinterpret_cast<T*>(st + L::OFF_H);
    const float* rings = reinterpret_cast<const float*>(st + L::OFF_RING);
    constexpr int HPLANE = SY * L::BXH;

    if (x0 == 0 || y0 == 0 || x0 + TX >= nx || y0 + TY >= ny) {
      // halo positions outside the domain: periodic wrap or nearest node
      for (int i = tid; i < SX * SY; i += NT) {
        const int lx = i % SX, ly = i / SX;
        int gx = x0 + lx - 1, gy = y0 + ly - 1;
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) continue;
        gx = grad_coord(gx, nx, m.bc[0]);
        gy = grad_coord(gy, ny, m.bc[1]);
        const int j = gy * px + gx;
        const int P = int(m.plane);
#pragma unroll
        for (int a = 0; a < 9; ++a)
          hsm[a * HPLANE + ly * L::BXH + lx + L::HX - 1] = src[(QF + 9 + a) * P + j];
      }
      __syncthreads();
    }
    // phi + 1 of the halo-extended tile
    for (int i = tid; i < SX * SY; i += NT) {
      const int lx = i % SX, ly = i / SX;
      const T* hp = hsm + ly * L::BXH + lx + L::HX - 1;
      R sum = R(0);
#pragma unroll
      for (int a = 0; a < 9; ++a) sum += Pop<T>::template ld<R>(hp + a * HPLANE);
      sh_phi[ly][lx] = sum;
    }
    __syncthreads();

    const int x = x0 + tx, y = y0 + ty;
    if (x < nx && y < ny) {
      R f[9], g[9], h[9];
      const int o = ty * TX + tx;
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        if (FLOW) f[a] = Pop<T>::template ld<R>(fgs + a * (TY * TX) + o);
        g[a] = Pop<T>::template ld<R>(fgs + (QF + a) * (TY * TX) + o);
        h[a] = Pop<T>::template ld<R>(hsm + a * HPLANE + (ty + 1) * L::BXH + tx + L::HX);
      }
      TileView<T, R, L::BXH, HPLANE, L::HX - 1> hs{hsm};
      if (x0 >= 1 && x0 + TX <= nx - 1 && y0 >= 1 && y0 + TY <= ny - 1)
        collide_push_2d<T, R, FLOW, true, SX>(m, x, y, tx + 1, ty + 1, f, g, h,
                                              sh_phi[ty + 1][tx + 1], rings[o], &sh_phi[0][0], hs,
                                              dst, ring_cur, err);
      else
        collide_push_2d<T, R, FLOW, false, SX>(m, x, y, tx + 1, ty + 1, f, g, h,
                                               sh_phi[ty + 1][tx + 1], rings[o], &sh_phi[0][0],
                                               hs, dst, ring_cur, err);
    }
}

}  // namespace lbk
