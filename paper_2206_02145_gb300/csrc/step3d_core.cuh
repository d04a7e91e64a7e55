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

// pv: phi + 1 around the node, hv: the h deviations around it (views above).
// INTERIOR: every node of the tile is at least one node away from every
// domain face, so every destination is an ordinary node.
template <typename T, typename R, bool FLOW, bool INTERIOR, typename PV, typename HV>
__device__ __forceinline__ void collide_push_3d(const Model& m, int x, int y, int z, int lx,
                                                int ly, const R (&f)[19], const R (&g)[7],
                                                const R (&h)[7], R dphi, R dphi_prev,
                                                const PV& pv, const HV& hs,
                                                T* __restrict__ dst, R* __restrict__ ring_cur,
                                                unsigned* __restrict__ err) {
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
  const R U = c.ref_g + dU;
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
  const R omega_U = rcp_r(R(0.5) + c.tauU_slope * mask);  // Eq. 18
  const R dphidt = dphi - dphi_prev;
  ring_cur[idx] = dphi;
  if (!(finite_r(phi) && finite_r(U) && finite_r(rho))) atomicOr(err, 1u);

  // ---- grad = 3 sum_a w_a c_a phi(x + c_a) over D3Q19 ---------------------------
  R gr[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int a = 1; a < 19; ++a) {
    const R v = pv.at(D3_CZ[a], ly + D3_CY[a], lx + D3_CX[a]) * (a < 7 ? R(1.0 / 6.0) : R(1.0 / 12.0));
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
      fp = fma_r(keep_f, f[a], mul_r(wf, add_r(feq, guo_t)));
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
        Pop<T>::st(pd + ((QF + a) * P + off), gp);
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
    if (bounce) {
      // half-way bounce-back: comes back to this node reversed
      const int b = D3_OPP[a];
      if (FLOW) Pop<T>::st(dst + (b * P + idx), fp);
      if (sc) {
        Pop<T>::st(dst + ((QF + b) * P + idx), gp);
        Pop<T>::st(dst + ((QF + 7 + b) * P + idx), fma_r(inv_a2, hp, mul_r(keep_old, h[b])));
      }
    } else if (!drop) {
      const int jd = zd * slab + yd * px + xd;
      if (FLOW) Pop<T>::st(dst + (a * P + jd), fp);
      if (sc) {
        const R hold = hs.at(a, cz, ly + cy, lx + cx);
        Pop<T>::st(dst + ((QF + a) * P + jd), gp);
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
            Pop<T>::st(dst + ((QF + a) * P + jo), gp);
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
            Pop<T>::st(dst + ((QF + a) * P + idx), ws * ((c.U_in - c.ref_g) + c.U_in * R(4) * gu));
            Pop<T>::st(dst + ((QF + 7 + a) * P + idx), R(0));  // phi = -1: zero deviation
          }
        }
      }
    }
  }
}

}  // namespace lbk
