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
  // 16-bit storage: g relative to a per-node U (the own reference of the tile
  // and a halo box of the encoding reference, FP16, starting 8 left of the
  // tile so that the box starts on a 16-byte boundary)
  static constexpr bool REL = sizeof(T) == 2;
  static constexpr int HXU = 8, BXU = TX + 2 * HXU;
  static constexpr int UOWN_BYTES = REL ? TY * TX * 2 : 0;
  static constexpr int UHAL_BYTES = REL ? (TY + 2) * BXU * 2 : 0;
  static constexpr int al(int b) { return (b + 127) / 128 * 128; }
  static constexpr int OFF_H = al(FG_BYTES);
  static constexpr int OFF_RING = OFF_H + al(H_BYTES);
  static constexpr int OFF_UOWN = OFF_RING + al(RING_BYTES);
  static constexpr int OFF_UHAL = OFF_UOWN + al(UOWN_BYTES);
  static constexpr int STAGE = OFF_UHAL + al(UHAL_BYTES);
  static constexpr int TX_BYTES = FG_BYTES + H_BYTES + RING_BYTES + UOWN_BYTES + UHAL_BYTES;
};

// Fill one stage: f and g of the tile, h with its halo, the phi ring; with
// 16-bit storage also the tile's U reference (plane c) and the halo of the
// encoding reference (plane c ^ 1).
template <typename T, bool FLOW, int TX, int TY>
__device__ __forceinline__ void issue_tile_2d(const CUtensorMap* tm_fg, const CUtensorMap* tm_h,
                                              const CUtensorMap* tm_ring,
                                              const CUtensorMap* tm_uown,
                                              const CUtensorMap* tm_uhal, int c, uint64_t* bar,
                                              unsigned char* st, int x0, int y0) {
  using L = Tiles2D<T, FLOW, TX, TY>;
  mbar_arrive_expect_tx(bar, L::TX_BYTES);
  tma_load_3d(st, tm_fg, bar, x0, y0, 0);
  tma_load_3d(st + L::OFF_H, tm_h, bar, x0 - L::HX, y0 - 1, L::QFG);
  tma_load_2d(st + L::OFF_RING, tm_ring, bar, x0, y0);
  if (L::REL) {
    tma_load_3d(st + L::OFF_UOWN, tm_uown, bar, x0, y0, c);
    tma_load_3d(st + L::OFF_UHAL, tm_uhal, bar, x0 - L::HXU, y0 - 1, c ^ 1);
  }
}

// Work on a filled stage `st` for the tile at (x0, y0).  Called by all
// threads of the CTA; contains CTA barriers.  sh_phi: (TY + 2) x (TX + 2).
// MASK: solid nodes are handled (flag of the tile from m.solid_tiles).  CHM:
// the flow collides by the central Hermite MRT.
template <typename T, bool FLOW, int TX, int TY, bool MASK, bool CHM>
__device__ __forceinline__ void tile_2d(const Model& m, const T* __restrict__ src,
                                        T* __restrict__ dst, float* __restrict__ ring_cur,
                                        unsigned* __restrict__ err, int x0, int y0, int c,
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
    const __half* uown = reinterpret_cast<const __half*>(st + L::OFF_UOWN);
    __half* uhal = reinterpret_cast<__half*>(st + L::OFF_UHAL);
    constexpr int HPLANE = SY * L::BXH;
    // tiles next to solid nodes take the general path with the mask (the
    // flag is loaded first, so that its latency overlaps the phi sums)
    const bool solids =
        MASK && m.solid && m.solid_tiles[(y0 / TY) * ((nx + TX - 1) / TX) + x0 / TX];

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
        if (L::REL) uhal[ly * L::BXU + lx + L::HXU - 1] = m.uring[size_t(c ^ 1) * m.plane + j];
      }
      __syncthreads();
    }
    // phi + 1 of the halo-extended tile: each thread's own position from the
    // h it keeps for the collision, the ring around the tile by a pass
    R h[9];
    {
      R sum = R(0);
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        h[a] = Pop<T>::template ld<R>(hsm + a * HPLANE + (ty + 1) * L::BXH + tx + L::HX);
        sum += h[a];
      }
      sh_phi[ty + 1][tx + 1] = sum;
    }
    constexpr int NRING = 2 * SX + 2 * TY;
    for (int i = tid; i < NRING; i += NT) {
      int lx, ly;
      if (i < 2 * SX) {
        lx = i % SX;
        ly = i < SX ? 0 : SY - 1;
      } else {
        lx = (i - 2 * SX) & 1 ? SX - 1 : 0;
        ly = 1 + (i - 2 * SX) / 2;
      }
      const T* hp = hsm + ly * L::BXH + lx + L::HX - 1;
      R sum = R(0);
#pragma unroll
      for (int a = 0; a < 9; ++a) sum += Pop<T>::template ld<R>(hp + a * HPLANE);
      sh_phi[ly][lx] = sum;
    }
    __syncthreads();

    const int x = x0 + tx, y = y0 + ty;
    if (x < nx && y < ny && solids && m.solid[y * px + x]) {
      ring_cur[y * px + x] = sh_phi[ty + 1][tx + 1];  // a solid node keeps its state
    } else if (x < nx && y < ny) {
      R f[9], g[9];
      const int o = ty * TX + tx;
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        if (FLOW) f[a] = Pop<T>::template ld<R>(fgs + a * (TY * TX) + o);
        g[a] = Pop<T>::template ld<R>(fgs + (QF + a) * (TY * TX) + o);
      }
      // g stored relative to the node's own U reference, the collision
      // takes the deviations from it as they are
      UView<L::REL, L::BXU> uh{uhal + L::HXU - 1,
                               L::REL ? m.uring + size_t(c) * m.plane : nullptr,
                               L::REL ? __half2float(uown[o]) : 0.f};
      TileView<T, R, L::BXH, HPLANE, L::HX - 1> hs{hsm};
      if (!solids && x0 >= 1 && x0 + TX <= nx - 1 && y0 >= 1 && y0 + TY <= ny - 1)
        collide_push_2d<T, R, FLOW, true, SX, MASK, CHM>(m, x, y, tx + 1, ty + 1, f, g, h,
                                                    sh_phi[ty + 1][tx + 1], rings[o],
                                                    &sh_phi[0][0], hs, uh, dst, ring_cur, err);
      else
        collide_push_2d<T, R, FLOW, false, SX, MASK, CHM>(m, x, y, tx + 1, ty + 1, f, g, h,
                                                     sh_phi[ty + 1][tx + 1], rings[o],
                                                     &sh_phi[0][0], hs, uh, dst, ring_cur, err,
                                                     solids);
    }
}

}  // namespace lbk
