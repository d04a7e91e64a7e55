// Per-node part of the 3D coupled step, shared by the 3D step kernels:
// D3Q19 flow f (Eqs. 4-12), D3Q7 solute g (Eqs. 13-18) and D3Q7 phase field
// h (Eqs. 19-23, cubic anisotropy of Eq. 3), push streaming.  The caller has
// the node's own population deviations in registers and phi + 1 and the h
// deviations around the node (one node in x, y and z) in shared memory.
#pragma once

#include "lbpf_device.cuh"

namespace lbk {

// Shared-memory views of the node's neighbourhood, indexed by the plane
// offset dz in {-1, 0, 1} from the node's plane and the local (ly, lx) of a
// halo-extended tile.  PhiSlab3 / HSlab3: a contiguous [z][y][x] tile (plane
// of the node at lz); PhiRing3 / HRing3: three separately stored planes.
template <typename R, int ROW, int SLAB>
struct PhiSlab3 {
  const R* base;  // plane of the node
  __device__ __forceinline__ R at(int dz, int ly, int lx) const {
    return base[dz * SLAB + ly * ROW + lx];
  }
};
template <typename R, int ROW, int SLAB, int PLANE>
struct HSlab3 {
  const R* base;  // direction 0, plane of the node
  __device__ __forceinline__ R at(int a, int dz, int ly, int lx) const {
    return base[a * PLANE + dz * SLAB + ly * ROW + lx];
  }
};
template <typename R, int ROW>
struct PhiRing3 {
  const R* p[3];  // planes dz = -1, 0, 1
  __device__ __forceinline__ R at(int dz, int ly, int lx) const { return p[dz + 1][ly * ROW + lx]; }
};
template <typename R, int ROW, int PLANE>
struct HRing3 {
  const R* p[3];  // planes dz = -1, 0, 1 (direction 0; direction a at + a * PLANE)
  __device__ __forceinline__ R at(int a, int dz, int ly, int lx) const {
    return p[dz + 1][a * PLANE + ly * ROW + lx];
  }
};

// ---- central Hermite MRT of the D3Q19 flow lattice (Sec. 2.2 after Eq. 9) ----
// The nineteen moments are the products H_i(X) H_j(Y) H_k(Z) (H_0 = 1,
// H_1 = X, H_2 = X^2 - 1/3; i, j, k <= 2, at most two non-zero) about u*.
// Every one involves at most two axes, and the weights' moments over an axis
// pair are those of D2Q9 (1, 1/3, 1/3, 1/9), so each pair (p, q) takes the
// 2D transform of its nine raw moments; the pairs share the moments of one
// axis.  Raw moments of the stored deviations -> central Hermite moments ->
// relaxation by order -> raw moments -> populations through the inverse of
// the D3Q19 raw-moment matrix (rest, faces and each pair's four edges in
// closed form).

// central Hermite moments XY, X^2 Y, X Y^2, X^2 Y^2 of the pair (p, q) from
// the raw deviation moments e_ij of p^i q^j
template <typename R>
struct ChmPair {
  R hpq, hppq, hpqq, hppqq;
};

template <typename R>
__device__ __forceinline__ ChmPair<R> chm_pair_central(R e00, R e10, R e01, R e20, R e02, R e11,
                                                      R e21, R e12, R e22, R vp, R vq, R rho) {
  const R t3 = R(1.0 / 3.0), t9 = R(1.0 / 9.0);
  const R vpp = vp * vp, vqq = vq * vq, vpq = vp * vq;
  ChmPair<R> h;
  h.hpq = e11 - vp * e01 - vq * e10 + vpq * rho;
  h.hppq = e21 - R(2) * vp * e11 + vpp * e01 - vq * e20 + R(2) * vpq * e10 - vpp * vq * rho -
           t3 * e01 + t3 * vq * e00;
  h.hpqq = e12 - R(2) * vq * e11 + vqq * e10 - vp * e02 + R(2) * vpq * e01 - vp * vqq * rho -
           t3 * e10 + t3 * vp * e00;
  h.hppqq = e22 - R(2) * vp * e12 - R(2) * vq * e21 + vpp * e02 + vqq * e20 + R(4) * vpq * e11 -
            R(2) * vpq * vq * e10 - R(2) * vpq * vp * e01 + vpp * vqq * rho -
            t3 * (e20 + e02) + R(2) * t3 * (vp * e10 + vq * e01) - t3 * (vpp + vqq) * e00 +
            t9 * e00;
  return h;
}

// raw deviation moments f11, f21 (p^2 q), f12 (p q^2), f22 of the pair after
// collision, from its relaxed central Hermite moments (s: first and
// diagonal second order of p and q, m: the pair's own)
template <typename R>
__device__ __forceinline__ void chm_pair_raw(const ChmPair<R>& m, R hp, R hq, R hpp, R hqq, R vp,
                                             R vq, R rho, R e00, R& f11, R& f21, R& f12,
                                             R& f22) {
  const R t3 = R(1.0 / 3.0), t9 = R(1.0 / 9.0);
  const R vpp = vp * vp, vqq = vq * vq, vpq = vp * vq;
  const R kpp = hpp + t3 * rho, kqq = hqq + t3 * rho;
  const R k21 = m.hppq + t3 * hq, k12 = m.hpqq + t3 * hp;
  f11 = m.hpq + vp * hq + vq * hp + vpq * rho;
  f21 = k21 + R(2) * vp * m.hpq + vpp * hq + vq * kpp + R(2) * vpq * hp + vpp * vq * rho;
  f12 = k12 + R(2) * vq * m.hpq + vqq * hp + vp * kqq + R(2) * vpq * hq + vp * vqq * rho;
  f22 = m.hppqq + t3 * (hpp + hqq) + t9 * e00 + R(2) * vp * k12 + R(2) * vq * k21 + vpp * kqq +
        vqq * kpp + R(4) * vpq * m.hpq + R(2) * vpq * vq * hp + R(2) * vpq * vp * hq +
        vpp * vqq * rho;
}

// d: the node's f deviations (D3Q19 order: rest, +x, -x, +y, -y, +z, -z, then
// the pairs xy, xz, yz with four edges each, (+,+), (-,-), (+,-), (-,+));
// mo: their first moments; v: u*; F: the force.  out: post-collision
// deviations.
template <typename R>
__device__ __forceinline__ void chm_post_3d(const R (&d)[19], R drho, R rho, const R (&mo)[3],
                                            const R (&v)[3], const R (&F)[3], R wf, R wb, R wh,
                                            R (&out)[19]) {
  const R t3 = R(1.0 / 3.0);
  const R e00 = drho;
  // raw moments of each pair: p^2 q^2, p q, p^2 q, p q^2
  R e22[3], e11[3], e21[3], e12[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int b = 7 + 4 * k;
    e22[k] = (d[b] + d[b + 1]) + (d[b + 2] + d[b + 3]);
    e11[k] = (d[b] + d[b + 1]) - (d[b + 2] + d[b + 3]);
    e21[k] = (d[b] - d[b + 1]) - (d[b + 2] - d[b + 3]);
    e12[k] = (d[b] - d[b + 1]) + (d[b + 2] - d[b + 3]);
  }
  // pairs: 0 = (x, y), 1 = (x, z), 2 = (y, z)
  const R e2[3] = {(d[1] + d[2]) + (e22[0] + e22[1]), (d[3] + d[4]) + (e22[0] + e22[2]),
                   (d[5] + d[6]) + (e22[1] + e22[2])};
  // central Hermite moments, first and diagonal second order
  R h1[3], h2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    h1[a] = mo[a] - v[a] * rho;
    h2[a] = e2[a] - t3 * e00 - R(2) * v[a] * mo[a] + v[a] * v[a] * rho;
  }
  constexpr int PP[3] = {0, 0, 1}, QQ[3] = {1, 2, 2};
  ChmPair<R> hp[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int p = PP[k], q = QQ[k];
    hp[k] = chm_pair_central<R>(e00, mo[p], mo[q], e2[p], e2[q], e11[k], e21[k], e12[k], e22[k],
                                v[p], v[q], rho);
  }
  // relaxation towards rho and zeros; the force in the first order; the
  // trace of the second order at wb, its deviatoric part and the mixed
  // moments at wf, third and fourth order at wh
  const R kf = R(1) - wf, gf = R(1) - R(0.5) * wf, kh = R(1) - wh;
  const R mean = (h2[0] + h2[1] + h2[2]) * t3;
  const R kb = (R(1) - wb) * mean;
  R s1[3], s2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    s1[a] = kf * h1[a] + gf * F[a];
    s2[a] = kb + kf * (h2[a] - mean);
  }
  R f11[3], f21[3], f12[3], f22[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int p = PP[k], q = QQ[k];
    ChmPair<R> m;
    m.hpq = kf * hp[k].hpq;
    m.hppq = kh * hp[k].hppq;
    m.hpqq = kh * hp[k].hpqq;
    m.hppqq = kh * hp[k].hppqq;
    chm_pair_raw<R>(m, s1[p], s1[q], s2[p], s2[q], v[p], v[q], rho, e00, f11[k], f21[k], f12[k],
                    f22[k]);
  }
  // raw moments of one axis after collision
  R f1[3], f2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    f1[a] = s1[a] + v[a] * rho;
    f2[a] = s2[a] + t3 * e00 + R(2) * v[a] * s1[a] + v[a] * v[a] * rho;
  }
  // populations: rest, faces, edges
  out[0] = e00 - (f2[0] + f2[1] + f2[2]) + (f22[0] + f22[1] + f22[2]);
  {
    // faces of x: x y^2 and x z^2 are the p q^2 of pairs xy and xz; of y:
    // x^2 y (pair xy, p^2 q) and y z^2 (pair yz, p q^2); of z: x^2 z and y^2 z
    const R sx = f2[0] - f22[0] - f22[1], ax = f1[0] - f12[0] - f12[1];
    const R sy = f2[1] - f22[0] - f22[2], ay = f1[1] - f21[0] - f12[2];
    const R sz = f2[2] - f22[1] - f22[2], az = f1[2] - f21[1] - f21[2];
    out[1] = R(0.5) * (sx + ax);
    out[2] = R(0.5) * (sx - ax);
    out[3] = R(0.5) * (sy + ay);
    out[4] = R(0.5) * (sy - ay);
    out[5] = R(0.5) * (sz + az);
    out[6] = R(0.5) * (sz - az);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int b = 7 + 4 * k;
    out[b] = R(0.25) * (f22[k] + f12[k] + f21[k] + f11[k]);
    out[b + 1] = R(0.25) * (f22[k] - f12[k] - f21[k] + f11[k]);
    out[b + 2] = R(0.25) * (f22[k] + f12[k] - f21[k] - f11[k]);
    out[b + 3] = R(0.25) * (f22[k] - f12[k] + f21[k] - f11[k]);
  }
}

// The per-node g reference around a node (3D, 16-bit storage), as UView of
// the 2D step: `own` the reference of the node's own populations, at(dz, ly,
// lx) the encoding reference of the node at plane offset dz and local (ly,
// lx) (three halo-extended planes of row pitch ROW), `out` the plane that
// receives each node's new U.  REL = false: every member unused.
template <bool REL, int ROW>
struct UView3 {
  static constexpr bool kRel = REL;
  const __half* p[3];
  __half* out;
  float own;
  __device__ __forceinline__ float at(int dz, int ly, int lx) const {
    return REL ? __half2float(p[dz + 1][ly * ROW + lx]) : 0.f;
  }
};
using NoUView3 = UView3<false, 1>;

// Solid nodes (3D mask): is the node at (x, y, z), mapped like a gradient
// neighbour (periodic wrap, else nearest node), solid?
__device__ __forceinline__ bool solid_mapped3(const Model& m, int x, int y, int z) {
  x = grad_coord(x, m.nx, m.bc[0]);
  y = grad_coord(y, m.ny, m.bc[1]);
  z = grad_coord(z, m.nz, m.bc[2]);
  return m.solid[(size_t(z) * m.ny + y) * m.px + x] != 0;
}

// pv: phi + 1 around the node, hv: the h deviations around it (views above).
// INTERIOR: every node of the tile is at least one node away from every
// domain face, so every destination is an ordinary node.  CHM: the flow
// collides by the central Hermite MRT.  MASK: the code for solid nodes is
// compiled in; `solids` (the tile or column chunk holds or borders a solid
// node) switches it on: a solid gradient neighbour counts as the first fluid
// node among the single-axis steps of its direction (x, y, z order) and the
// node itself, and a push towards a solid node comes back reversed.
template <typename T, typename R, bool FLOW, bool INTERIOR, bool CHM, bool MASK = false,
          typename PV, typename HV, typename UV = NoUView3>
__device__ __forceinline__ void collide_push_3d(const Model& m, int x, int y, int z, int lx,
                                                int ly, const R (&f)[19], const R (&g)[7],
                                                const R (&h)[7], R dphi, R dphi_prev,
                                                const PV& pv, const HV& hs,
                                                T* __restrict__ dst, R* __restrict__ ring_cur,
                                                unsigned* __restrict__ err,
                                                bool solids = false, const UV& uh = UV()) {
  constexpr int QF = FLOW ? 19 : 0;
  const int nx = m.nx, ny = m.ny, nz = m.nz, px = m.px;
  const int P = int(m.plane);  // fits: checked at creation
  const int slab = ny * px;
  const int idx = z * slab + y * px + x;
  T* const pd = dst + idx;
  const Coef<R>& c = coef<R>(m);

  // ---- local moments (Eqs. 11, 12, 17, 22) ----------------------------------
  const R phi = dphi - R(1);
  R dU = R(0);
#pragma unroll
  for (int a = 0; a < 7; ++a) dU += g[a];
  // g deviations are taken from w_a Rg; the collision (Eqs. 13-16) is linear
  // in them, so any per-node Rg gives the same populations
  const R Rg = UV::kRel ? R(uh.own) : c.ref_g;
  const R U = Rg + dU;
  R drho = R(0), mo[3] = {R(0), R(0), R(0)};
  if (FLOW) {
#pragma unroll
    for (int a = 0; a < 19; ++a) {
      drho += f[a];
      if (D3_CX[a]) mo[0] += R(D3_CX[a]) * f[a];
      if (D3_CY[a]) mo[1] += R(D3_CY[a]) * f[a];
      if (D3_CZ[a]) mo[2] += R(D3_CZ[a]) * f[a];
    }
  }
  const R rho = R(1) + drho;
  const R ph = clamp1(phi);
  const R mask = R(0.5) * (R(1) - ph);  // (1 - phi)/2 of Eq. 7 and q(phi) of Eq. 18
  R u[3] = {R(0), R(0), R(0)}, F[3] = {R(0), R(0), R(0)};
  if (FLOW) {
    const R K = c.kdrag * (R(1) + ph) * (R(1) + ph) * (R(1) - ph);  // Eq. 6
    const R inv = rcp_r(rho + R(0.5) * K);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      u[d] = (mo[d] + R(0.5) * c.body[d]) * inv;
      F[d] = c.body[d] - K * u[d];
    }
  }
  const R us[3] = {mask * u[0], mask * u[1], mask * u[2]};  // Eq. 7
  R fchm[19];
  if (FLOW && CHM) chm_post_3d<R>(f, drho, rho, mo, us, F, c.omega_f, c.chm_wb, c.chm_wh, fchm);
  const R omega_U = rcp_r(R(0.5) + c.tauU_slope * mask);  // Eq. 18
  const R dphidt = dphi - dphi_prev;
  ring_cur[idx] = dphi;
  if (UV::kRel) uh.out[idx] = __float2half_rn(float(U));
  if (!(finite_r(phi) && finite_r(U) && finite_r(rho))) atomicOr(err, 1u);
  // a g deviation pushed to the node at (dz, dly, dlx), taken from its
  // reference there instead of this node's
  auto genc = [&](R v, R w, int dz, int dly, int dlx) -> R {
    return UV::kRel ? fma_r(-w, R(uh.at(dz, dly, dlx)) - Rg, v) : v;
  };

  // ---- grad = 3 sum_a w_a c_a phi(x + c_a) over D3Q19 ---------------------------
  R gr[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int a = 1; a < 19; ++a) {
    const int gcx = D3_CX[a], gcy = D3_CY[a], gcz = D3_CZ[a];
    R pn = pv.at(gcz, ly + gcy, lx + gcx);
    if (MASK && !INTERIOR && solids && solid_mapped3(m, x + gcx, y + gcy, z + gcz)) {
      if (gcx != 0 && !solid_mapped3(m, x + gcx, y, z)) pn = pv.at(0, ly, lx + gcx);
      else if (gcy != 0 && !solid_mapped3(m, x, y + gcy, z)) pn = pv.at(0, ly + gcy, lx);
      else if (gcz != 0 && !solid_mapped3(m, x, y, z + gcz)) pn = pv.at(gcz, ly, lx);
      else pn = pv.at(0, ly, lx);
    }
    const R v = pn * (a < 7 ? R(1.0 / 6.0) : R(1.0 / 12.0));
    if (D3_CX[a]) gr[0] += R(D3_CX[a]) * v;
    if (D3_CY[a]) gr[1] += R(D3_CY[a]) * v;
    if (D3_CZ[a]) gr[2] += R(D3_CZ[a]) * v;
  }
  R as, N[3];
  aniso<R>(m, gr[0], gr[1], gr[2], as, N[0], N[1], N[2]);
  const R a2 = as * as;
  const R inv_a2 = rcp_r(a2);
  const R omega_phi = rcp_r(a2 * c.tpc + R(0.5));  // Eq. 23
  const R phi2m = R(1) - phi * phi;
  const R Qs = (phi - phi * phi * phi + c.lambda * U * phi2m * phi2m) * c.inv_tau0;  // Eq. 20

  // node constants of the collisions (see the 2D core); D3Q7 has c_s^2 = 1/4
  const R uu = us[0] * us[0] + us[1] * us[1] + us[2] * us[2];
  const R uF = us[0] * F[0] + us[1] * F[1] + us[2] * F[2];
  const R omega_f = c.omega_f, keep_f = R(1) - c.omega_f, guo = c.guo;
  const R E0 = omega_f * (drho - R(1.5) * rho * uu);
  const R E1 = omega_f * R(3) * rho, E2 = omega_f * R(4.5) * rho;
  const R G0 = -R(3) * uF;
  const R keep_U = R(1) - omega_U;
  const R K0 = omega_U * dU - dphidt, K1 = R(4) * omega_U * U;
  const R keep_phi = R(1) - omega_phi;
  const R H0 = omega_phi * dphi + Qs;
  const R Hx = omega_phi * c.tpc * N[0], Hy = omega_phi * c.tpc * N[1],
          Hz = omega_phi * c.tpc * N[2];
  const R keep_old = R(1) - inv_a2;  // Eq. 19: h_new = h* / a_s^2 + (1 - 1/a_s^2) h_old
  const int bcx = m.bc[0], bcy = m.bc[1], bcz = m.bc[2];

#pragma unroll
  for (int a = 0; a < 19; ++a) {
    if (!FLOW && a >= 7) break;
    const int cx = D3_CX[a], cy = D3_CY[a], cz = D3_CZ[a];
    const R cu = R(cx) * us[0] + R(cy) * us[1] + R(cz) * us[2];
    const bool sc = a < 7;  // also a direction of the D3Q7 lattices
    R fp = R(0), gp = R(0), hp = R(0);
    if (FLOW) {
      const R wf = d3q19_w<R>(a);
      const R cF = R(cx) * F[0] + R(cy) * F[1] + R(cz) * F[2];
      const R feq = fma_r(cu, fma_r(E2, cu, E1), E0);
      const R guo_t = mul_r(guo, fma_r(cF, fma_r(R(9), cu, R(3)), G0));
      fp = CHM ? fchm[a] : fma_r(keep_f, f[a], mul_r(wf, add_r(feq, guo_t)));
    }
    if (sc) {
      const R ws = d3q7_w<R>(a);
      gp = fma_r(keep_U, g[a], mul_r(ws, fma_r(K1, cu, K0)));
      hp = fma_r(keep_phi, h[a],
                 mul_r(ws, add_r(H0, -add_r(add_r(R(cx) * Hx, R(cy) * Hy), R(cz) * Hz))));
    }
    if (INTERIOR) {
      const int off = cz * slab + cy * px + cx;
      if (FLOW) Pop<T>::st(pd + (a * P + off), fp);
      if (sc) {
        const R hold = hs.at(a, cz, ly + cy, lx + cx);
        Pop<T>::st(pd + ((QF + a) * P + off), genc(gp, d3q7_w<R>(a), cz, ly + cy, lx + cx));
        Pop<T>::st(pd + ((QF + 7 + a) * P + off), fma_r(inv_a2, hp, mul_r(keep_old, hold)));  // Eq. 19
      }
      continue;
    }
    int xd = x + cx, yd = y + cy, zd = z + cz;
    bool bounce = false, drop = false;
    if (yd < 0 || yd >= ny) {
      if (bcy == BC_PERIODIC) yd = wrap1(yd, ny);
      else bounce = true;
    }
    if (zd < 0 || zd >= nz) {
      if (bcz == BC_PERIODIC) zd = wrap1(zd, nz);
      else bounce = true;
    }
    if (xd < 0 || xd >= nx) {
      if (bcx == BC_PERIODIC) xd = wrap1(xd, nx);
      else if (bcx == BC_WALL) bounce = true;
      else drop = true;
    }
    if (MASK && solids && !bounce && !drop && m.solid[zd * slab + yd * px + xd])
      bounce = true;  // obstacle
    if (bounce) {
      // half-way bounce-back: comes back to this node reversed
      const int b = D3_OPP[a];
      if (FLOW) Pop<T>::st(dst + (b * P + idx), fp);
      if (sc) {
        Pop<T>::st(dst + ((QF + b) * P + idx), genc(gp, d3q7_w<R>(a), 0, ly, lx));
        Pop<T>::st(dst + ((QF + 7 + b) * P + idx), fma_r(inv_a2, hp, mul_r(keep_old, h[b])));
      }
    } else if (!drop) {
      const int jd = zd * slab + yd * px + xd;
      if (FLOW) Pop<T>::st(dst + (a * P + jd), fp);
      if (sc) {
        const R hold = hs.at(a, cz, ly + cy, lx + cx);
        Pop<T>::st(dst + ((QF + a) * P + jd), genc(gp, d3q7_w<R>(a), cz, ly + cy, lx + cx));
        Pop<T>::st(dst + ((QF + 7 + a) * P + jd), fma_r(inv_a2, hp, mul_r(keep_old, hold)));  // Eq. 19
      }
    }
    if (bcx == BC_INOUT) {
      if (cx == -1 && x == nx - 1) {
        // outflow ghost x = nx repeats this column
        int yo = y + cy, zo = z + cz;
        bool ok = true;
        if (yo < 0 || yo >= ny) {
          if (bcy == BC_PERIODIC) yo = wrap1(yo, ny);
          else ok = false;
        }
        if (zo < 0 || zo >= nz) {
          if (bcz == BC_PERIODIC) zo = wrap1(zo, nz);
          else ok = false;
        }
        if (ok) {
          const int jo = zo * slab + yo * px + x;
          if (FLOW) Pop<T>::st(dst + (a * P + jo), fp);
          if (sc) {
            const R hold = hs.at(a, cz, ly + cy, lx);
            Pop<T>::st(dst + ((QF + a) * P + jo), genc(gp, d3q7_w<R>(a), cz, ly + cy, lx));
            Pop<T>::st(dst + ((QF + 7 + a) * P + jo), fma_r(inv_a2, hp, mul_r(keep_old, hold)));
          }
        }
      }
      if (cx == 1 && x == 0) {
        // inflow ghost x = -1 (equilibrium, phi = -1), unless behind a wall
        const int ys = y - cy, zs = z - cz;
        const bool behind_wall = ((ys < 0 || ys >= ny) && bcy == BC_WALL) ||
                                 ((zs < 0 || zs >= nz) && bcz == BC_WALL);
        if (!behind_wall) {
          const R uin = c.u_in, cui = uin;
          if (FLOW)
            Pop<T>::st(dst + (a * P + idx),
                       d3q19_w<R>(a) * (R(3) * cui + R(4.5) * cui * cui - R(1.5) * uin * uin));
          if (sc) {
            const R ws = d3q7_w<R>(a);
            const R gu = FLOW ? cui : R(0);
            Pop<T>::st(dst + ((QF + a) * P + idx),
                       genc(ws * ((c.U_in - Rg) + c.U_in * R(4) * gu), ws, 0, ly, lx));
            Pop<T>::st(dst + ((QF + 7 + a) * P + idx), R(0));  // phi = -1: zero deviation
          }
        }
      }
    }
  }
}

}  // namespace lbk
