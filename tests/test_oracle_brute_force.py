"""Brute-force check of one oracle step on tiny periodic grids (4 x 4, 8 x 8).

The step is expanded here node by node and direction by direction in plain
Python, from the model's equations as the paper states them (Sec. 2.2,
Eqs. 3-23) and the readings the oracle documents, in the pull form: every
population of node x at t + 1 is computed from its source node x - c_a.  The
expansion shares nothing with the oracle but the direction order of its
exported populations.  It differs from the oracle's route where the
mathematics allows: the anisotropic flux N of Eq. 21 comes from the
definition N = (1/2) |grad phi|^2 d(a_s^2)/d(grad phi), differentiated by the
complex step (exact to rounding for an analytic function) of a_s written as a
polynomial in the normal, where the oracle uses atan2 and a closed form.

The state the step starts from is the oracle's own after a few steps from
random fields (so that every population is off equilibrium and phi(t-1)
differs from phi(t)); the check is that the oracle's map of that state equals
this expansion to 1e-14.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import Params

# direction order of the exported populations (D2Q9)
C = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
W = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
CS2 = 1.0 / 3.0


def a_s_poly(gx, gy, k, eps, theta0):
    """Eq. 3 with n = -grad/|grad| and theta the angle of n:
    a_s = 1 + eps cos(k (theta - theta0)), with cos(k theta) and sin(k theta)
    written as the real and imaginary parts of (n_x + i n_y)^k expanded by the
    binomial theorem, so that a_s is a polynomial in (n_x, n_y) and analytic in
    (g_x, g_y) away from 0 (complex arguments allowed)."""
    r = (gx * gx + gy * gy) ** 0.5
    nx, ny = -gx / r, -gy / r
    ck = sum(math.comb(k, 2 * j) * (-1) ** j * nx ** (k - 2 * j) * ny ** (2 * j)
             for j in range(k // 2 + 1))
    sk = sum(math.comb(k, 2 * j + 1) * (-1) ** j * nx ** (k - 2 * j - 1) * ny ** (2 * j + 1)
             for j in range((k - 1) // 2 + 1))
    return 1.0 + eps * (ck * math.cos(k * theta0) + sk * math.sin(k * theta0))


def flux_N(gx, gy, k, eps, theta0, literal):
    """N = fac |grad|^2 a_s d(a_s)/d(grad) (reading of Eq. 21; fac = 2 for the
    literal |grad|^2 d(a_s^2)/d(grad)), the derivative by the complex step."""
    h = 1e-30
    a = a_s_poly(gx, gy, k, eps, theta0)
    dax = a_s_poly(complex(gx, h), gy, k, eps, theta0).imag / h
    day = a_s_poly(gx, complex(gy, h), k, eps, theta0).imag / h
    g2 = gx * gx + gy * gy
    fac = 2.0 if literal else 1.0
    return fac * g2 * a * dax, fac * g2 * a * day


def brute_step(p, f, g, h, phi_prev):
    """One coupled step of the whole grid, pull form, periodic in x and y.
    f, g, h: [q][ny][nx] populations at t; phi_prev: phi(t-1).  Returns the
    populations at t + 1."""
    ny, nx = h.shape[1:]
    tau0 = p.w0 ** 2 / (CS2 * (p.tau_phi0 - 0.5))            # Eq. 23 at a_s = 1
    D = CS2 * (p.tau_u_liquid - 0.5)                         # Eq. 18 in the liquid
    lam = p.lambda_ if p.lambda_ >= 0 else D * tau0 / (0.6267 * p.w0 ** 2)
    # per-node quantities at t
    node = {}
    phi = np.zeros((ny, nx))
    for y in range(ny):
        for x in range(nx):
            phi[y, x] = sum(h[a, y, x] for a in range(9))     # Eq. 22
    for y in range(ny):
        for x in range(nx):
            U = sum(g[a, y, x] for a in range(9))             # Eq. 17
            ph = phi[y, x]
            phh = min(1.0, max(-1.0, ph))
            if p.flow:
                rho = sum(f[a, y, x] for a in range(9))       # Eq. 11
                mx = sum(C[a][0] * f[a, y, x] for a in range(9))  # Eq. 12
                my = sum(C[a][1] * f[a, y, x] for a in range(9))
                K = p.h_drag * p.tau_f * (1 + phh) ** 2 * (1 - phh) / (4 * p.w0 ** 2)  # Eq. 6
                # Guo's velocity u = (m + F/2)/rho with F = b - K u, solved for u
                ux = (mx + 0.5 * p.body[0]) / (rho + 0.5 * K)
                uy = (my + 0.5 * p.body[1]) / (rho + 0.5 * K)
                Fx, Fy = p.body[0] - K * ux, p.body[1] - K * uy
            else:
                rho, ux, uy, Fx, Fy = 1.0, 0.0, 0.0, 0.0, 0.0
            mask = 0.5 * (1 - phh)
            usx, usy = mask * ux, mask * uy                  # Eq. 7
            # isotropic gradient: (1/cs^2) sum_a w_a c_a phi(x + c_a)
            gx = sum(W[a] * C[a][0] * phi[(y + C[a][1]) % ny, (x + C[a][0]) % nx]
                     for a in range(9)) / CS2
            gy = sum(W[a] * C[a][1] * phi[(y + C[a][1]) % ny, (x + C[a][0]) % nx]
                     for a in range(9)) / CS2
            if gx * gx + gy * gy <= 1e-12:
                a_s, Nx, Ny = 1.0, 0.0, 0.0
            else:
                a_s = a_s_poly(gx, gy, p.fold, p.eps, p.theta0)
                Nx, Ny = flux_N(gx, gy, p.fold, p.eps, p.theta0, p.aniso_literal)
            node[y, x] = dict(
                U=U, phi=ph, rho=rho, usx=usx, usy=usy, Fx=Fx, Fy=Fy, a2=a_s * a_s,
                tau_phi=a_s * a_s * p.w0 ** 2 / (CS2 * tau0) + 0.5,            # Eq. 23
                tau_U=0.5 + (p.tau_u_liquid - 0.5) * mask,                     # Eq. 18
                Q=ph - ph ** 3 + lam * U * (1 - ph * ph) ** 2,                 # Eq. 20
                dphidt=ph - phi_prev[y, x], Nx=Nx, Ny=Ny)
    fn, gn, hn = np.zeros_like(f), np.zeros_like(g), np.zeros_like(h)
    for y in range(ny):
        for x in range(nx):
            for a in range(9):
                cx, cy = C[a]
                sy, sx = (y - cy) % ny, (x - cx) % nx
                s = node[sy, sx]
                cu = cx * s["usx"] + cy * s["usy"]
                uu = s["usx"] ** 2 + s["usy"] ** 2
                if p.flow:
                    cF = cx * s["Fx"] + cy * s["Fy"]
                    uF = s["usx"] * s["Fx"] + s["usy"] * s["Fy"]
                    feq = W[a] * s["rho"] * (1 + cu / CS2 + cu * cu / (2 * CS2 ** 2)
                                             - uu / (2 * CS2))           # Eq. 9
                    G = (1 - 1 / (2 * p.tau_f)) * W[a] * (
                        cF / CS2 + (cu * cF) / CS2 ** 2 - uF / CS2)      # Eq. 5
                    fn[a, y, x] = f[a, sy, sx] - (f[a, sy, sx] - feq) / p.tau_f + G  # Eq. 4, 8
                geq = W[a] * s["U"] * (1 + cu / CS2)                      # Eq. 16
                gn[a, y, x] = (g[a, sy, sx] - (g[a, sy, sx] - geq) / s["tau_U"]
                               - W[a] * s["dphidt"])                      # Eqs. 13-15
                heq = W[a] * (s["phi"] - (cx * s["Nx"] + cy * s["Ny"]) * p.w0 ** 2
                              / (CS2 * tau0))                             # Eq. 21
                hstar = (h[a, sy, sx] - (h[a, sy, sx] - heq) / s["tau_phi"]
                         + W[a] * s["Q"] / tau0)
                # Eq. 19: a_s^2(r) h(r + c, t + 1) = h*(r) - (1 - a_s^2(r)) h(r + c, t)
                hn[a, y, x] = (hstar - (1 - s["a2"]) * h[a, y, x]) / s["a2"]
    return fn, gn, hn


@pytest.mark.parametrize("n", [4, 8])
@pytest.mark.parametrize("case", ["coupled_5fold", "no_flow_4fold_literal"])
def test_one_step_by_brute_force(oracle_mod, n, case):
    if case == "coupled_5fold":
        p = Params(nx=n, ny=n, flow=1, fold=5, eps=0.04, theta0=0.3, body=(2e-5, -1e-5, 0.0))
    else:
        p = Params(nx=n, ny=n, flow=0, fold=4, eps=0.05, theta0=-0.2, aniso_literal=1,
                   lambda_=2.0)
    rng = np.random.default_rng(100 + n)
    nn = p.nodes
    phi0 = np.tanh(rng.normal(0.0, 1.5, nn))
    o = O.Oracle(p)
    o.init_fields(phi0, 0.3 + 0.05 * rng.random(nn), 1 + 0.01 * rng.standard_normal(nn),
                  0.01 * rng.standard_normal(nn), 0.01 * rng.standard_normal(nn))
    o.step(3)
    f, g, h = (o.pops(k) for k in ("f", "g", "h"))
    fn, gn, hn = brute_step(p, f, g, h, o.phi_prev())
    o.step(1)
    if p.flow:
        np.testing.assert_allclose(o.pops("f"), fn, rtol=0, atol=1e-14)
    np.testing.assert_allclose(o.pops("g"), gn, rtol=0, atol=1e-14)
    np.testing.assert_allclose(o.pops("h"), hn, rtol=0, atol=1e-14)
    # the state is far from equilibrium and the step does something
    assert np.abs(hn - h).max() > 1e-3 and np.abs(gn - g).max() > 1e-4
