// Fused coupled LB step in 2D: D2Q9 flow f (Eqs. 4-12), D2Q9 solute g
// (Eqs. 13-18) and D2Q9 phase field h (Eqs. 19-23), one thread per node.
//
// Streaming is done in push form: the thread of node s loads its own
// populations (aligned, coalesced), forms every moment locally, collides and
// writes the post-collision value of direction a to s + c_a.  That is the
// same update as the pull form of the paper's equations; it needs no stored
// macroscopic fields, only phi(t-1) for d(phi)/dt.  Per node and step the
// HBM traffic is 27 populations read + 27 written + phi(t-1) read + phi(t)
// written (224 B in FP32 with flow, 152 B without).
//
// Populations are handled as deviations d_a = p_a - w_a M_ref (M_ref = 1 for
// f, U_ref for g, -1 for h); the phi ring holds phi + 1.
//
// Two parts of the step need neighbour data, both served from shared memory:
//   - grad(phi) for the normal and anisotropy (Eq. 3, Eq. 21, Eq. 23): phi(t)
//     of the tile plus a one-node halo, summed from the h populations;
//   - Eq. 19 writes a_s^2 h(r + c, t+1) = h*(r) - (1 - a_s^2(r)) h(r + c, t):
//     the old h of the destination node, which is the tile's own h or the
//     halo's, staged in shared memory next to phi.
// The halo ring is loaded in the same round trip as the tile's own
// populations (one ring node per thread of the first 2 (TX + TY) + 4).
#include "lbpf_device.cuh"

namespace lbk {
namespace {

template <typename T, typename R, bool FLOW, int TX, int TY>
__global__ void __launch_bounds__(TX* TY)
    step2d_kernel(const Model m, const T* __restrict__ src, T* __restrict__ dst,
                  const R* __restrict__ ring_prev, R* __restrict__ ring_cur,
                  unsigned* __restrict__ err) {
  constexpr int SX = TX + 2, SY = TY + 2;
  constexpr int QF = FLOW ? 9 : 0;
  constexpr int NT = TX * TY;
  constexpr int RING = 2 * SX + 2 * TY;
  static_assert(RING <= NT, "one ring node per thread");
  __shared__ R sh_phi[SY][SX];  // phi + 1 of tile and halo
  __shared__ R sh_h[9][SY][SX];  // h deviations of tile and halo

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int x = x0 + tx, y = y0 + ty;
  const int nx = m.nx, ny = m.ny, px = m.px;
  const long long P = m.plane;
  const bool active = x < nx && y < ny;
  const bool full = x0 + TX <= nx && y0 + TY <= ny;
  const long long idx = (long long)y * px + x;

  const T* sf = src;
  const T* sg = src + (long long)QF * P;
  const T* shp = src + (long long)(QF + 9) * P;

  // ---- one round trip: own populations, phi ring, and (full tiles) the halo
  R f[9], g[9], h[9];
  R dphi_prev = R(0);
  if (active) {
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      if (FLOW) f[a] = Pop<T>::template ld<R>(sf + a * P + idx);
      g[a] = Pop<T>::template ld<R>(sg + a * P + idx);
      h[a] = Pop<T>::template ld<R>(shp + a * P + idx);
    }
    dphi_prev = ring_prev[idx];
  }
  R hv[9];
  int rlx = 0, rly = 0;
  const bool ring_thread = full && tid < RING;
  if (ring_thread) {
    if (tid < SX) {
      rlx = tid;
      rly = 0;
    } else if (tid < 2 * SX) {
      rlx = tid - SX;
      rly = SY - 1;
    } else if (tid < 2 * SX + TY) {
      rlx = 0;
      rly = 1 + tid - 2 * SX;
    } else {
      rlx = SX - 1;
      rly = 1 + tid - 2 * SX - TY;
    }
    const int gx = grad_coord(x0 + rlx - 1, nx, m.bc[0]);
    const int gy = grad_coord(y0 + rly - 1, ny, m.bc[1]);
    const long long j = (long long)gy * px + gx;
#pragma unroll
    for (int a = 0; a < 9; ++a) hv[a] = Pop<T>::template ld<R>(shp + a * P + j);
  }
  R dphi = R(0);
  if (active) {
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      dphi += h[a];  // Eq. 22: phi = -1 + sum d_h
      sh_h[a][ty + 1][tx + 1] = h[a];
    }
    sh_phi[ty + 1][tx + 1] = dphi;
  }
  if (ring_thread) {
    R s = R(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      s += hv[a];
      sh_h[a][rly][rlx] = hv[a];
    }
    sh_phi[rly][rlx] = s;
  }
  if (!full) {
    // edge tile: every position not owned by an active thread, mapped
    for (int i = tid; i < SX * SY; i += NT) {
      const int lx = i % SX, ly = i / SX;
      int gx = x0 + lx - 1, gy = y0 + ly - 1;
      if (lx >= 1 && lx <= TX && ly >= 1 && ly <= TY && gx < nx && gy < ny) continue;
      gx = grad_coord(gx, nx, m.bc[0]);
      gy = grad_coord(gy, ny, m.bc[1]);
      const long long j = (long long)gy * px + gx;
      R s = R(0);
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        const R v = Pop<T>::template ld<R>(shp + a * P + j);
        sh_h[a][ly][lx] = v;
        s += v;
      }
      sh_phi[ly][lx] = s;
    }
  }
  __syncthreads();
  if (!active) return;

  // ---- local moments (Eqs. 11, 12, 17, 22) ----------------------------------
  const R phi = dphi - R(1);
  R dU = R(0);
#pragma unroll
  for (int a = 0; a < 9; ++a) dU += g[a];
  const R U = R(m.ref_g) + dU;
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
    const R K = R(m.kdrag) * (R(1) + ph) * (R(1) + ph) * (R(1) - ph);
    const R inv = R(1) / (rho + R(0.5) * K);
    ux = (mx + R(0.5) * R(m.body[0])) * inv;
    uy = (my + R(0.5) * R(m.body[1])) * inv;
    Fx = R(m.body[0]) - K * ux;
    Fy = R(m.body[1]) - K * uy;
  }
  const R usx = mask * ux, usy = mask * uy;  // u* (Eq. 7)
  const R omega_U = R(1) / (R(0.5) + R(m.tauU_slope) * mask);  // Eq. 18
  const R dphidt = dphi - dphi_prev;
  ring_cur[idx] = dphi;
  if (!(finite_r(phi) && finite_r(U) && finite_r(rho))) atomicOr(err, 1u);

  // ---- gradient, anisotropy, phase-field coefficients (Eqs. 3, 20, 21, 23) --
  const int lx = tx + 1, ly = ty + 1;
  const R pE = sh_phi[ly][lx + 1], pW = sh_phi[ly][lx - 1];
  const R pN = sh_phi[ly + 1][lx], pS = sh_phi[ly - 1][lx];
  const R pNE = sh_phi[ly + 1][lx + 1], pNW = sh_phi[ly + 1][lx - 1];
  const R pSE = sh_phi[ly - 1][lx + 1], pSW = sh_phi[ly - 1][lx - 1];
  // grad = 3 sum_a w_a c_a phi(x + c_a) over D2Q9
  const R gxv = R(1.0 / 3.0) * (pE - pW) + R(1.0 / 12.0) * ((pNE + pSE) - (pNW + pSW));
  const R gyv = R(1.0 / 3.0) * (pN - pS) + R(1.0 / 12.0) * ((pNE + pNW) - (pSE + pSW));
  R as, Nx, Ny, Nz;
  aniso<R>(m, gxv, gyv, R(0), as, Nx, Ny, Nz);
  const R a2 = as * as;
  const R inv_a2 = R(1) / a2;
  const R omega_phi = R(1) / (a2 * R(m.tpc) + R(0.5));  // Eq. 23
  const R phi2m = R(1) - phi * phi;
  const R Qs = (phi - phi * phi * phi + R(m.lambda) * U * phi2m * phi2m) * R(m.inv_tau0);  // Eq. 20
  const R tpc = R(m.tpc);
  const R uu = usx * usx + usy * usy, uF = usx * Fx + usy * Fy;
  const R omega_f = R(m.omega_f), guo = R(m.guo);

  T* df = dst;
  T* dg = dst + (long long)QF * P;
  T* dh = dst + (long long)(QF + 9) * P;
  const int bcx = m.bc[0], bcy = m.bc[1];

#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const int cx = D2_CX[a], cy = D2_CY[a];
    const R w = d2_w<R>(a);
    const R cu = R(cx) * usx + R(cy) * usy;
    // post-collision deviations at this node
    R fp = R(0);
    if (FLOW) {
      const R cF = R(cx) * Fx + R(cy) * Fy;
      const R feq = w * (drho + rho * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu));  // Eq. 9
      const R G = w * guo * (R(3) * cF + R(9) * cu * cF - R(3) * uF);               // Eq. 5
      fp = f[a] - omega_f * (f[a] - feq) + G;                                       // Eq. 4, 8
    }
    const R geq = w * (dU + U * R(3) * cu);                    // Eq. 16
    const R gp = g[a] - omega_U * (g[a] - geq) - w * dphidt;   // Eqs. 13-15
    const R heq = w * (dphi - tpc * (R(cx) * Nx + R(cy) * Ny)); // Eq. 21
    const R hp = h[a] - omega_phi * (h[a] - heq) + w * Qs;     // Eq. 19 (right side)

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
    if (bounce) {
      // half-way bounce-back: comes back to this node reversed
      const int b = D2_OPP[a];
      if (FLOW) Pop<T>::st(df + b * P + idx, fp);
      Pop<T>::st(dg + b * P + idx, gp);
      Pop<T>::st(dh + b * P + idx, hp * inv_a2 - (inv_a2 - R(1)) * h[b]);
    } else if (!drop) {
      const long long jd = (long long)yd * px + xd;
      const R hold = sh_h[a][ly + cy][lx + cx];  // h_a(s + c_a, t)
      if (FLOW) Pop<T>::st(df + a * P + jd, fp);
      Pop<T>::st(dg + a * P + jd, gp);
      Pop<T>::st(dh + a * P + jd, hp * inv_a2 - (inv_a2 - R(1)) * hold);  // Eq. 19
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
          const long long jo = (long long)yo * px + x;
          const R hold = sh_h[a][ly + cy][lx];
          if (FLOW) Pop<T>::st(df + a * P + jo, fp);
          Pop<T>::st(dg + a * P + jo, gp);
          Pop<T>::st(dh + a * P + jo, hp * inv_a2 - (inv_a2 - R(1)) * hold);
        }
      }
      if (cx == 1 && x == 0) {
        // inflow ghost x = -1: equilibrium at rho = 1, u = u_in e_x, U = U_in,
        // phi = -1 (a_s = 1; its h deviation is 0), unless behind a wall
        const int ys = y - cy;
        if (!((ys < 0 || ys >= ny) && bcy == BC_WALL)) {
          const R uin = R(m.u_in), cui = uin;
          if (FLOW)
            Pop<T>::st(df + a * P + idx,
                       w * (R(3) * cui + R(4.5) * cui * cui - R(1.5) * uin * uin));
          const R gu = FLOW ? cui : R(0);
          const R Uin = R(m.U_in);
          Pop<T>::st(dg + a * P + idx, w * ((Uin - R(m.ref_g)) + Uin * R(3) * gu));
          Pop<T>::st(dh + a * P + idx, R(0));
        }
      }
    }
  }
}

template <typename T, typename R, bool FLOW>
cudaError_t launch_t(const Model& m, const void* src, void* dst, const void* ring_prev,
                     void* ring_cur, unsigned* err, cudaStream_t s) {
  constexpr int TX = 32, TY = 8;
  dim3 block(TX, TY);
  dim3 grid((m.nx + TX - 1) / TX, (m.ny + TY - 1) / TY);
  step2d_kernel<T, R, FLOW, TX, TY><<<grid, block, 0, s>>>(
      m, static_cast<const T*>(src), static_cast<T*>(dst), static_cast<const R*>(ring_prev),
      static_cast<R*>(ring_cur), err);
  return cudaGetLastError();
}

template <typename T, typename R>
cudaError_t launch_flow(const Model& m, const void* src, void* dst, const void* pp, void* pc,
                        unsigned* err, cudaStream_t s) {
  return m.flow ? launch_t<T, R, true>(m, src, dst, pp, pc, err, s)
                : launch_t<T, R, false>(m, src, dst, pp, pc, err, s);
}

}  // namespace

cudaError_t launch_step2d(const Model& m, const void* src, void* dst, const void* ring_prev,
                          void* ring_cur, unsigned* err, cudaStream_t s) {
  switch (m.storage) {
    case ST_FP64: return launch_flow<double, double>(m, src, dst, ring_prev, ring_cur, err, s);
    case ST_FP16: return launch_flow<__half, float>(m, src, dst, ring_prev, ring_cur, err, s);
    case ST_BF16: return launch_flow<__nv_bfloat16, float>(m, src, dst, ring_prev, ring_cur, err, s);
    default: return launch_flow<float, float>(m, src, dst, ring_prev, ring_cur, err, s);
  }
}

}  // namespace lbk
