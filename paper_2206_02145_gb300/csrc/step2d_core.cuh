// Per-node part of the 2D coupled step, shared by the step kernels: moments,
// anisotropy, collisions of f, g and h, and the push of every direction to
// its destination (Eqs. 3-23).  The caller has the node's own population
// deviations in registers and the tile's phi + 1 and h deviations (with a
// one-node halo) in shared memory.
#pragma once

#include "lbpf_device.cuh"

namespace lbk {

// Shared-memory view of the halo-extended tile: value of lattice direction a
// at local position (lx, ly) (lx, ly in [0, TX + 1] x [0, TY + 1]).  The
// shape is compile-time, so every access is one load with an immediate
// offset from a per-thread base.
template <typename T, typename R, int ROW, int PLANE, int XOFF>
struct TileView {
  const T* base;
  __device__ __forceinline__ R at(int a, int ly, int lx) const {
    return Pop<T>::template ld<R>(base + a * PLANE + ly * ROW + lx + XOFF);
  }
};

// The per-node g reference around a node (2D, 16-bit storage): `own` the
// reference of the node's own populations, at(ly, lx) the encoding reference
// of the node at local (ly, lx) (halo box of row pitch ROW, the pointer
// offset so that lx = 0 is the tile's left halo column), `out` the plane that
// receives each node's new U.  With REL = false (FP32 and FP64 storage) g is
// relative to the global U_ref and every member is unused.
template <bool REL, int ROW>
struct UView {
  static constexpr bool kRel = REL;
  const __half* hal;
  __half* out;
  float own;
  __device__ __forceinline__ float at(int ly, int lx) const {
    return REL ? __half2float(hal[ly * ROW + lx]) : 0.f;
  }
};
using NoUView = UView<false, 1>;

// Solid nodes (2D mask): is the node at (x, y), mapped like a gradient
// neighbour (periodic wrap, else nearest node), solid?
__device__ __forceinline__ bool solid_mapped(const Model& m, int x, int y) {
  x = grad_coord(x, m.nx, m.bc[0]);
  y = grad_coord(y, m.ny, m.bc[1]);
  return m.solid[y * m.px + x] != 0;
}

// Central Hermite MRT of the flow populations (2D; the collision of the
// paper's flow solver, read as the C ABI documents for LBPF_COLL_CHM).
// d: pre-collision deviations f - w; drho, rho, (mx, my): their zeroth and
// first moments; (vx, vy) = u*; F the force; wf, wb, wh the rates.  The
// moments are formed from the deviations with the weights' own moments
// (1, 0, 0, 1/3, 1/3, 0, 0, 0, 1/9) taken out analytically, so that FP32
// keeps the small quantities: raw moments e_pq -> central Hermite moments
// about u* -> relaxation by order -> raw moments -> populations through the
// inverse of the D2Q9 raw-moment matrix.  out: post-collision deviations.
template <typename R>
__device__ __forceinline__ void chm_post_2d(const R (&d)[9], R drho, R rho, R mx, R my, R vx,
                                            R vy, R Fx, R Fy, R wf, R wb, R wh, R (&out)[9]) {
  const R t3 = R(1.0 / 3.0), t9 = R(1.0 / 9.0);
  // raw moments of the deviations
  const R e00 = drho, e10 = mx, e01 = my;
  const R dd = (d[5] + d[6]) + (d[7] + d[8]);
  const R e20 = (d[1] + d[3]) + dd, e02 = (d[2] + d[4]) + dd;
  const R e11 = (d[5] - d[6]) + (d[7] - d[8]);
  const R e21 = (d[5] + d[6]) - (d[7] + d[8]);
  const R e12 = (d[5] - d[6]) - (d[7] - d[8]);
  const R e22 = dd;
  const R vxx = vx * vx, vyy = vy * vy, vxy = vx * vy;
  // central Hermite moments about (vx, vy)
  const R h1 = e10 - vx * rho, h2 = e01 - vy * rho;
  const R hxx = e20 - t3 * e00 - R(2) * vx * e10 + vxx * rho;
  const R hyy = e02 - t3 * e00 - R(2) * vy * e01 + vyy * rho;
  const R hxy = e11 - vx * e01 - vy * e10 + vxy * rho;
  const R hxxy = e21 - R(2) * vx * e11 + vxx * e01 - vy * e20 + R(2) * vxy * e10 -
                 vxx * vy * rho - t3 * e01 + t3 * vy * e00;
  const R hxyy = e12 - R(2) * vy * e11 + vyy * e10 - vx * e02 + R(2) * vxy * e01 -
                 vx * vyy * rho - t3 * e10 + t3 * vx * e00;
  const R hxxyy = e22 - R(2) * vx * e12 - R(2) * vy * e21 + vxx * e02 + vyy * e20 +
                  R(4) * vxy * e11 - R(2) * vxy * vy * e10 - R(2) * vxy * vx * e01 +
                  vxx * vyy * rho - t3 * (e20 + e02) + R(2) * t3 * (vx * e10 + vy * e01) -
                  t3 * (vxx + vyy) * e00 + t9 * e00;
  // relaxation towards rho and zeros; the force in the first order
  const R kf = R(1) - wf, gf = R(1) - R(0.5) * wf, kh = R(1) - wh;
  const R h1s = kf * h1 + gf * Fx, h2s = kf * h2 + gf * Fy;
  const R tr = (R(1) - wb) * (hxx + hyy), dv = kf * (hxx - hyy);
  const R hxxs = R(0.5) * (tr + dv), hyys = R(0.5) * (tr - dv);
  const R hxys = kf * hxy;
  const R hxxys = kh * hxxy, hxyys = kh * hxyy, hxxyys = kh * hxxyy;
  // central (raw) moments after collision, then raw moments of the deviations
  const R k20 = hxxs + t3 * rho, k02 = hyys + t3 * rho;
  const R k21 = hxxys + t3 * h2s, k12 = hxyys + t3 * h1s;
  const R f10 = h1s + vx * rho, f01 = h2s + vy * rho;
  const R f20 = hxxs + t3 * e00 + R(2) * vx * h1s + vxx * rho;
  const R f02 = hyys + t3 * e00 + R(2) * vy * h2s + vyy * rho;
  const R f11 = hxys + vx * h2s + vy * h1s + vxy * rho;
  const R f21 = k21 + R(2) * vx * hxys + vxx * h2s + vy * k20 + R(2) * vxy * h1s + vxx * vy * rho;
  const R f12 = k12 + R(2) * vy * hxys + vyy * h1s + vx * k02 + R(2) * vxy * h2s + vx * vyy * rho;
  const R f22 = hxxyys + t3 * (hxxs + hyys) + t9 * e00 + R(2) * vx * k12 + R(2) * vy * k21 +
                vxx * k02 + vyy * k20 + R(4) * vxy * hxys + R(2) * vxy * vy * h1s +
                R(2) * vxy * vx * h2s + vxx * vyy * rho;
  // populations (D2Q9 order: rest, +x, +y, -x, -y, ++, -+, --, +-)
  out[0] = e00 - f20 - f02 + f22;
  out[1] = R(0.5) * (f10 + f20 - f12 - f22);
  out[3] = R(0.5) * (-f10 + f20 + f12 - f22);
  out[2] = R(0.5) * (f01 + f02 - f21 - f22);
  out[4] = R(0.5) * (-f01 + f02 + f21 - f22);
  out[5] = R(0.25) * (f11 + f21 + f12 + f22);
  out[6] = R(0.25) * (-f11 + f21 - f12 + f22);
  out[7] = R(0.25) * (f11 - f21 - f12 + f22);
  out[8] = R(0.25) * (-f11 - f21 + f12 + f22);
}

// dphi_prev: phi(t-1) + 1 of this node; ring_cur: where phi(t) + 1 goes.
// phi_s: the tile's phi + 1 with halo ([ly][lx], row pitch PROW).
// dst: the destination population buffer (array a at dst + a * plane).
// INTERIOR: the caller guarantees 1 <= x <= nx - 2 and 1 <= y <= ny - 2 for
// every node of the tile, so every destination is an ordinary node (no wrap,
// wall or ghost) and the push needs no boundary logic.  MASK: the code for
// solid nodes is compiled in; `solids` (the tile holds or borders a solid
// node) switches it on.  CHM: the flow collides by the central Hermite MRT.
template <typename T, typename R, bool FLOW, bool INTERIOR, int PROW, bool MASK, bool CHM,
          typename HV, typename UV>
__device__ __forceinline__ void collide_push_2d(const Model& m, int x, int y, int lx, int ly,
                                                const R (&f)[9], const R (&g)[9],
                                                const R (&h)[9], R dphi, R dphi_prev,
                                                const R* phi_s, const HV& hs, const UV& uh,
                                                T* __restrict__ dst, R* __restrict__ ring_cur,
                                                unsigned* __restrict__ err,
                                                bool solids = false) {
  constexpr int QF = FLOW ? 9 : 0;
  const int nx = m.nx, ny = m.ny, px = m.px;
  const int P = int(m.plane);  // fits: checked at creation
  const int idx = y * px + x;
  T* const pd = dst + idx;  // this node in array 0; the offsets below are uniform
  const Coef<R>& c = coef<R>(m);

  // ---- local moments (Eqs. 11, 12, 17, 22) ----------------------------------
  const R phi = dphi - R(1);
  R dU = R(0);
#pragma unroll
  for (int a = 0; a < 9; ++a) dU += g[a];
  // g deviations are taken from w_a Rg; the collision (Eqs. 13-16) is linear
  // in them, so any per-node Rg gives the same populations
  const R Rg = UV::kRel ? R(uh.own) : c.ref_g;
  const R U = Rg + dU;
  R drho = R(0), mx = R(0), my = R(0);
  if (FLOW) {
#pragma unroll
    for (int a = 0; a < 9; ++a) drho += f[a];
    mx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    my = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
  }
  const R rho = R(1) + drho;
  const R ph = clamp1(phi);
  const R mask = R(0.5) * (R(1) - ph);  // (1 - phi)/2 of Eq. 7 and q(phi) of Eq. 18
  R ux = R(0), uy = R(0), Fx = R(0), Fy = R(0);
  if (FLOW) {
    // Eq. 6: F = b - K u, K = h tau_f (1+phi)^2 (1-phi) / (4 W0^2); the Guo
    // half-force velocity u = (m + F/2)/rho solved in closed form.
    const R K = c.kdrag * (R(1) + ph) * (R(1) + ph) * (R(1) - ph);
    const R inv = rcp_r(rho + R(0.5) * K);
    ux = (mx + R(0.5) * c.body[0]) * inv;
    uy = (my + R(0.5) * c.body[1]) * inv;
    Fx = c.body[0] - K * ux;
    Fy = c.body[1] - K * uy;
  }
  const R usx = mask * ux, usy = mask * uy;  // u* (Eq. 7)
  R fchm[9];
  if (FLOW && CHM)
    chm_post_2d<R>(f, drho, rho, mx, my, usx, usy, Fx, Fy, c.omega_f, c.chm_wb, c.chm_wh, fchm);
  const R omega_U = rcp_r(R(0.5) + c.tauU_slope * mask);  // Eq. 18
  const R dphidt = dphi - dphi_prev;
  ring_cur[idx] = dphi;
  if (UV::kRel) uh.out[idx] = __float2half_rn(float(U));
  if (!(finite_r(phi) && finite_r(U) && finite_r(rho))) atomicOr(err, 1u);
  // a g deviation pushed to the node at local (dly, dlx), taken from its
  // reference there instead of this node's
  auto genc = [&](R v, R w, int dly, int dlx) -> R {
    return UV::kRel ? fma_r(-w, R(uh.at(dly, dlx)) - Rg, v) : v;
  };

  // ---- gradient, anisotropy, phase-field coefficients (Eqs. 3, 20, 21, 23) --
  const R* pc = phi_s + ly * PROW + lx;
  R pE = pc[1], pW = pc[-1], pN = pc[PROW], pS = pc[-PROW];
  R pNE = pc[PROW + 1], pNW = pc[PROW - 1], pSE = pc[-PROW + 1], pSW = pc[-PROW - 1];
  if (MASK && !INTERIOR && solids) {
    // a solid neighbour counts as the first fluid node among (x + c_x, y),
    // (x, y + c_y) and (x, y): zero normal derivative at walls and obstacles
    auto sv = [&](int cx, int cy, R v) -> R {
      if (!solid_mapped(m, x + cx, y + cy)) return v;
      if (cx != 0 && !solid_mapped(m, x + cx, y)) return pc[cx];
      if (cy != 0 && !solid_mapped(m, x, y + cy)) return pc[cy * PROW];
      return pc[0];
    };
    pE = sv(1, 0, pE);
    pW = sv(-1, 0, pW);
    pN = sv(0, 1, pN);
    pS = sv(0, -1, pS);
    pNE = sv(1, 1, pNE);
    pNW = sv(-1, 1, pNW);
    pSE = sv(1, -1, pSE);
    pSW = sv(-1, -1, pSW);
  }
  // grad = 3 sum_a w_a c_a phi(x + c_a) over D2Q9
  const R gxv = R(1.0 / 3.0) * (pE - pW) + R(1.0 / 12.0) * ((pNE + pSE) - (pNW + pSW));
  const R gyv = R(1.0 / 3.0) * (pN - pS) + R(1.0 / 12.0) * ((pNE + pNW) - (pSE + pSW));
  R as, Nx, Ny, Nz;
  aniso<R>(m, gxv, gyv, R(0), as, Nx, Ny, Nz);
  const R a2 = as * as;
  const R inv_a2 = rcp_r(a2);
  const R omega_phi = rcp_r(a2 * c.tpc + R(0.5));  // Eq. 23
  const R phi2m = R(1) - phi * phi;
  const R Qs = (phi - phi * phi * phi + c.lambda * U * phi2m * phi2m) * c.inv_tau0;  // Eq. 20
  // Node constants of the collisions, so that each direction costs a few FMAs:
  //   f*: (1 - w_f) d + w_f w [E0 + cu (E1 + E2 cu)] + guo w [cF (3 + 9 cu) - 3 u*.F]
  //       (Eq. 4, 5, 8, 9 with c_s^2 = 1/3, d = f - w)
  //   g*: (1 - w_U) d + w (K0 + K1 cu)            (Eqs. 13-16, d = g - w U_ref)
  //   h*: (1 - w_phi) d + w (H0 - c.H)            (Eqs. 19-21, d = h + w)
  const R uu = usx * usx + usy * usy, uF = usx * Fx + usy * Fy;
  const R omega_f = c.omega_f, keep_f = R(1) - c.omega_f, guo = c.guo;
  const R E0 = omega_f * (drho - R(1.5) * rho * uu);
  const R E1 = omega_f * R(3) * rho, E2 = omega_f * R(4.5) * rho;
  const R G0 = -R(3) * uF;
  const R keep_U = R(1) - omega_U;
  const R K0 = omega_U * dU - dphidt, K1 = R(3) * omega_U * U;
  const R keep_phi = R(1) - omega_phi;
  const R H0 = omega_phi * dphi + Qs;
  const R Hx = omega_phi * c.tpc * Nx, Hy = omega_phi * c.tpc * Ny;
  const R keep_old = R(1) - inv_a2;  // Eq. 19: h_new = h* / a_s^2 + (1 - 1/a_s^2) h_old

  // array of direction a: f at a * P, g at (QF + a) * P, h at (QF + 9 + a) * P
#define LBPF_DF(a) (dst + (a) * P)
#define LBPF_DG(a) (dst + (QF + (a)) * P)
#define LBPF_DH(a) (dst + (QF + 9 + (a)) * P)
  const int bcx = m.bc[0], bcy = m.bc[1];

#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const int cx = D2_CX[a], cy = D2_CY[a];
    const R w = d2_w<R>(a);
    const R cu = R(cx) * usx + R(cy) * usy;
    // post-collision deviations at this node
    R fp = R(0);
    if (FLOW && CHM) {
      fp = fchm[a];
    } else if (FLOW) {
      const R cF = R(cx) * Fx + R(cy) * Fy;
      const R feq = fma_r(cu, fma_r(E2, cu, E1), E0);
      const R guo_t = mul_r(guo, fma_r(cF, fma_r(R(9), cu, R(3)), G0));
      fp = fma_r(keep_f, f[a], mul_r(w, add_r(feq, guo_t)));
    }
    const R gp = fma_r(keep_U, g[a], mul_r(w, fma_r(K1, cu, K0)));
    const R hp = fma_r(keep_phi, h[a], mul_r(w, add_r(H0, -add_r(R(cx) * Hx, R(cy) * Hy))));
    if (INTERIOR) {
      const int off = cy * px + cx;  // uniform
      const R hold = hs.at(a, ly + cy, lx + cx);  // h_a(s + c_a, t)
      if (FLOW) Pop<T>::st(pd + (a * P + off), fp);
      Pop<T>::st(pd + ((QF + a) * P + off), genc(gp, w, ly + cy, lx + cx));
      Pop<T>::st(pd + ((QF + 9 + a) * P + off), fma_r(inv_a2, hp, mul_r(keep_old, hold)));  // Eq. 19
      continue;
    }
    // destination s + c_a
    int xd = x + cx, yd = y + cy;
    bool bounce = false, drop = false;
    if (yd < 0 || yd >= ny) {
      if (bcy == BC_PERIODIC) yd = wrap1(yd, ny);
      else bounce = true;
    }
    if (xd < 0 || xd >= nx) {
      if (bcx == BC_PERIODIC) xd = wrap1(xd, nx);
      else if (bcx == BC_WALL) bounce = true;
      else drop = true;
    }
    if (MASK && solids && !bounce && !drop && m.solid[yd * px + xd]) bounce = true;  // obstacle
    if (bounce) {
      // half-way bounce-back: comes back to this node reversed
      const int b = D2_OPP[a];
      if (FLOW) Pop<T>::st(LBPF_DF(b) + idx, fp);
      Pop<T>::st(LBPF_DG(b) + idx, genc(gp, w, ly, lx));
      Pop<T>::st(LBPF_DH(b) + idx, fma_r(inv_a2, hp, mul_r(keep_old, h[b])));
    } else if (!drop) {
      const int jd = yd * px + xd;
      const R hold = hs.at(a, ly + cy, lx + cx);  // h_a(s + c_a, t)
      if (FLOW) Pop<T>::st(LBPF_DF(a) + jd, fp);
      Pop<T>::st(LBPF_DG(a) + jd, genc(gp, w, ly + cy, lx + cx));
      Pop<T>::st(LBPF_DH(a) + jd, fma_r(inv_a2, hp, mul_r(keep_old, hold)));  // Eq. 19
    }
    if (bcx == BC_INOUT) {
      if (cx == -1 && x == nx - 1) {
        // outflow ghost x = nx repeats this column: its post-collision value
        // arrives at (nx - 1, y + c_y)
        int yo = y + cy;
        bool ok = true;
        if (yo < 0 || yo >= ny) {
          if (bcy == BC_PERIODIC) yo = wrap1(yo, ny);
          else ok = false;
        }
        if (ok) {
          const int jo = yo * px + x;
          const R hold = hs.at(a, ly + cy, lx);
          if (FLOW) Pop<T>::st(LBPF_DF(a) + jo, fp);
          Pop<T>::st(LBPF_DG(a) + jo, genc(gp, w, ly + cy, lx));
          Pop<T>::st(LBPF_DH(a) + jo, fma_r(inv_a2, hp, mul_r(keep_old, hold)));
        }
      }
      if (cx == 1 && x == 0) {
        // inflow ghost x = -1: equilibrium at rho = 1, u = u_in e_x, U = U_in,
        // phi = -1 (a_s = 1; its h deviation is 0), unless behind a wall
        const int ys = y - cy;
        if (!((ys < 0 || ys >= ny) && bcy == BC_WALL)) {
          const R uin = c.u_in, cui = uin;
          if (FLOW)
            Pop<T>::st(LBPF_DF(a) + idx,
                       w * (R(3) * cui + R(4.5) * cui * cui - R(1.5) * uin * uin));
          const R gu = FLOW ? cui : R(0);
          const R Uin = c.U_in;
          Pop<T>::st(LBPF_DG(a) + idx, genc(w * ((Uin - Rg) + Uin * R(3) * gu), w, ly, lx));
          Pop<T>::st(LBPF_DH(a) + idx, R(0));
        }
      }
    }
  }
#undef LBPF_DF
#undef LBPF_DG
#undef LBPF_DH
}

}  // namespace lbk
