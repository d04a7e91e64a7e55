// Populations are deviations d_a = p_a - w_a M_ref as in 2D; the ring holds phi + 1.
// Fused coupled LB step in 3D: D3Q19 flow f (Eqs. 4-12), D3Q7 solute g
// (Eqs. 13-18) and D3Q7 phase field h (Eqs. 19-23), one thread per node,
// push streaming (same update as the pull form of the equations).  Per node
// and step the HBM traffic is 33 populations read + 33 written + phi(t-1)
// read + phi(t) written (272 B in FP32).  grad(phi) uses the D3Q19
// stencil; phi(t) and the destination's old h of Eq. 19 come from a
// one-node halo staged in shared memory, as in 2D.
#include "lbpf_device.cuh"

namespace lbk {
namespace {

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
  const long long P = m.plane;
  const long long rowz = (long long)ny * px;
  const bool active = x < nx && y < ny && z < nz;
  const long long idx = z * rowz + (long long)y * px + x;

  const Coef<R>& c = coef<R>(m);
  const T* sf = src;
  const T* sg = src + (long long)QF * P;
  const T* shp = src + (long long)(QF + 7) * P;

  R f[FLOW ? 19 : 1], g[7], h[7];
  R dphi = R(0);
  if (active) {
    if (FLOW) {
#pragma unroll
      for (int a = 0; a < 19; ++a) f[a] = Pop<T>::template ld<R>(sf + a * P + idx);
    }
#pragma unroll
    for (int a = 0; a < 7; ++a) {
      g[a] = Pop<T>::template ld<R>(sg + a * P + idx);
      h[a] = Pop<T>::template ld<R>(shp + a * P + idx);
    }
#pragma unroll
    for (int a = 0; a < 7; ++a) {
      dphi += h[a];  // Eq. 22: phi = -1 + sum d_h
      sh_h[a][tz + 1][ty + 1][tx + 1] = h[a];
    }
    sh_phi[tz + 1][ty + 1][tx + 1] = dphi;
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
    const long long j = gz * rowz + (long long)gy * px + gx;
    R s = R(0);
#pragma unroll
    for (int a = 0; a < 7; ++a) {
      const R v = Pop<T>::template ld<R>(shp + a * P + j);
      sh_h[a][lz][ly][lx] = v;
      s += v;
    }
    sh_phi[lz][ly][lx] = s;
  }
  __syncthreads();
  if (!active) return;

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
  const R mask = R(0.5) * (R(1) - ph);
  R u[3] = {R(0), R(0), R(0)}, F[3] = {R(0), R(0), R(0)};
  if (FLOW) {
    const R K = c.kdrag * (R(1) + ph) * (R(1) + ph) * (R(1) - ph);  // Eq. 6
    const R inv = R(1) / (rho + R(0.5) * K);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      u[d] = (mo[d] + R(0.5) * c.body[d]) * inv;
      F[d] = c.body[d] - K * u[d];
    }
  }
  const R us[3] = {mask * u[0], mask * u[1], mask * u[2]};  // Eq. 7
  const R omega_U = R(1) / (R(0.5) + c.tauU_slope * mask);  // Eq. 18
  const R dphidt = dphi - ring_prev[idx];
  ring_cur[idx] = dphi;
  if (!(finite_r(phi) && finite_r(U) && finite_r(rho))) atomicOr(err, 1u);

  // grad = 3 sum_a w_a c_a phi(x + c_a) over D3Q19
  const int lx = tx + 1, ly = ty + 1, lz = tz + 1;
  R gr[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int a = 1; a < 19; ++a) {
    const R v = sh_phi[lz + D3_CZ[a]][ly + D3_CY[a]][lx + D3_CX[a]] * (R(3) * d3q19_w<R>(a));
    if (D3_CX[a]) gr[0] += R(D3_CX[a]) * v;
    if (D3_CY[a]) gr[1] += R(D3_CY[a]) * v;
    if (D3_CZ[a]) gr[2] += R(D3_CZ[a]) * v;
  }
  R as, N[3];
  aniso<R>(m, gr[0], gr[1], gr[2], as, N[0], N[1], N[2]);
  const R a2 = as * as;
  const R inv_a2 = R(1) / a2;
  const R omega_phi = R(1) / (a2 * c.tpc + R(0.5));  // Eq. 23
  const R phi2m = R(1) - phi * phi;
  const R Qs = (phi - phi * phi * phi + c.lambda * U * phi2m * phi2m) * c.inv_tau0;
  const R tpc = c.tpc;
  const R uu = us[0] * us[0] + us[1] * us[1] + us[2] * us[2];
  const R uF = us[0] * F[0] + us[1] * F[1] + us[2] * F[2];

  T* df = dst;
  T* dg = dst + (long long)QF * P;
  T* dh = dst + (long long)(QF + 7) * P;
  const int bcx = m.bc[0], bcy = m.bc[1], bcz = m.bc[2];

#pragma unroll
  for (int a = 0; a < 19; ++a) {
    if (!FLOW && a >= 7) break;
    const int cx = D3_CX[a], cy = D3_CY[a], cz = D3_CZ[a];
    const R cu = R(cx) * us[0] + R(cy) * us[1] + R(cz) * us[2];
    R fp = R(0), gp = R(0), hp = R(0);
    const R wf = d3q19_w<R>(a);
    if (FLOW) {
      const R cF = R(cx) * F[0] + R(cy) * F[1] + R(cz) * F[2];
      const R feq = wf * (drho + rho * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu));  // Eq. 9
      const R G = wf * c.guo * (R(3) * cF + R(9) * cu * cF - R(3) * uF);           // Eq. 5
      fp = f[a] - c.omega_f * (f[a] - feq) + G;
    }
    const bool sc = a < 7;  // direction of the D3Q7 lattices too
    const R ws = d3q7_w<R>(a);
    if (sc) {
      gp = g[a] - omega_U * (g[a] - ws * (dU + U * R(4) * cu)) - ws * dphidt;  // Eqs. 13-16
      const R heq = ws * (dphi - tpc * (R(cx) * N[0] + R(cy) * N[1] + R(cz) * N[2]));  // Eq. 21
      hp = h[a] - omega_phi * (h[a] - heq) + ws * Qs;                                 // Eq. 19
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
      const int b = D3_OPP[a];
      if (FLOW) Pop<T>::st(df + b * P + idx, fp);
      if (sc) {
        Pop<T>::st(dg + b * P + idx, gp);
        Pop<T>::st(dh + b * P + idx, hp * inv_a2 - (inv_a2 - R(1)) * h[b]);
      }
    } else if (!drop) {
      const long long jd = zd * rowz + (long long)yd * px + xd;
      if (FLOW) Pop<T>::st(df + a * P + jd, fp);
      if (sc) {
        const R hold = sh_h[a][lz + cz][ly + cy][lx + cx];
        Pop<T>::st(dg + a * P + jd, gp);
        Pop<T>::st(dh + a * P + jd, hp * inv_a2 - (inv_a2 - R(1)) * hold);
      }
    }
    if (bcx == BC_INOUT) {
      if (cx == -1 && x == nx - 1) {
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
          const long long jo = zo * rowz + (long long)yo * px + x;
          if (FLOW) Pop<T>::st(df + a * P + jo, fp);
          if (sc) {
            const R hold = sh_h[a][lz + cz][ly + cy][lx];
            Pop<T>::st(dg + a * P + jo, gp);
            Pop<T>::st(dh + a * P + jo, hp * inv_a2 - (inv_a2 - R(1)) * hold);
          }
        }
      }
      if (cx == 1 && x == 0) {
        const int ys = y - cy, zs = z - cz;
        const bool behind_wall = ((ys < 0 || ys >= ny) && bcy == BC_WALL) ||
                                 ((zs < 0 || zs >= nz) && bcz == BC_WALL);
        if (!behind_wall) {
          const R uin = c.u_in, cui = uin;
          if (FLOW)
            Pop<T>::st(df + a * P + idx,
                       wf * (R(3) * cui + R(4.5) * cui * cui - R(1.5) * uin * uin));
          if (sc) {
            const R gu = FLOW ? cui : R(0);
            const R Uin = c.U_in;
            Pop<T>::st(dg + a * P + idx, ws * ((Uin - c.ref_g) + Uin * R(4) * gu));
            Pop<T>::st(dh + a * P + idx, R(0));  // phi = -1: zero deviation
          }
        }
      }
    }
  }
}

template <typename T, typename R, bool FLOW>
cudaError_t launch_t(const Model& m, const void* src, void* dst, const void* phi_prev,
                     void* phi_cur, unsigned* err, cudaStream_t s) {
  constexpr int TX = sizeof(R) == 8 ? 16 : 32, TY = 4, TZ = 2;
  dim3 block(TX, TY, TZ);
  dim3 grid((m.nx + TX - 1) / TX, (m.ny + TY - 1) / TY, (m.nz + TZ - 1) / TZ);
  step3d_kernel<T, R, FLOW, TX, TY, TZ><<<grid, block, 0, s>>>(
      m, static_cast<const T*>(src), static_cast<T*>(dst), static_cast<const R*>(phi_prev),
      static_cast<R*>(phi_cur), err);
  return cudaGetLastError();
}

template <typename T, typename R>
cudaError_t launch_flow(const Model& m, const void* src, void* dst, const void* pp, void* pc,
                        unsigned* err, cudaStream_t s) {
  return m.flow ? launch_t<T, R, true>(m, src, dst, pp, pc, err, s)
                : launch_t<T, R, false>(m, src, dst, pp, pc, err, s);
}

}  // namespace

cudaError_t launch_step3d(const Model& m, const void* src, void* dst, const void* phi_prev,
                          void* phi_cur, unsigned* err, cudaStream_t s) {
  switch (m.storage) {
    case ST_FP64: return launch_flow<double, double>(m, src, dst, phi_prev, phi_cur, err, s);
    case ST_FP16: return launch_flow<__half, float>(m, src, dst, phi_prev, phi_cur, err, s);
    case ST_BF16: return launch_flow<__nv_bfloat16, float>(m, src, dst, phi_prev, phi_cur, err, s);
    default: return launch_flow<float, float>(m, src, dst, phi_prev, phi_cur, err, s);
  }
}

}  // namespace lbk
