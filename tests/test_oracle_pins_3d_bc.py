"""Pins of the 3D lattices (D3Q19 flow, D3Q7 solute and phase field), of the
inlet/outlet boundary and of the default coupling constant."""
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import Params, PERIODIC, INLET_OUTLET

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def p3(**kw):
    base = dict(dim=3, nx=24, ny=24, nz=24, fold=0, flow=0, eps=0.0, lambda_=0.0)
    base.update(kw)
    return Params(**base)


def test_gaussian_diffusion_d3q7(oracle_mod):
    # D3Q7 with cs^2 = 1/4: D = (tau - 1/2) / 4
    n, s0, steps, tau = 32, 3.0, 60, 0.9
    p = p3(nx=n, ny=n, nz=n, tau_u_liquid=tau)
    z, y, x = np.mgrid[0:n, 0:n, 0:n].astype(float)
    c = n / 2
    r2 = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2
    A = 0.1
    o = O.Oracle(p)
    o.init_fields(-np.ones(n ** 3), 0.2 + A * np.exp(-r2 / (2 * s0 ** 2)))
    o.step(steps, threads=4)
    D = (tau - 0.5) / 4.0
    s2 = s0 ** 2 + 2 * D * steps
    exact = 0.2 + A * (s0 ** 2 / s2) ** 1.5 * np.exp(-r2 / (2 * s2))
    err = np.abs(o.fields()["U"] - exact).max() / A
    assert err < 1e-2, err


def test_taylor_green_d3q19(oracle_mod):
    # a 2D vortex in a 3D periodic box, in each of the three planes
    n, u0, tau = 24, 0.01, 0.6
    k = 2 * math.pi / n
    nu = (tau - 0.5) / 3.0
    for plane in range(3):
        p = p3(nx=n, ny=n, nz=n, flow=1, tau_f=tau)
        g = np.mgrid[0:n, 0:n, 0:n].astype(float)[::-1]  # x, y, z
        a, b = [(0, 1), (1, 2), (2, 0)][plane]
        u = [np.zeros((n, n, n)) for _ in range(3)]
        u[a] = -u0 * np.cos(k * g[a]) * np.sin(k * g[b])
        u[b] = u0 * np.sin(k * g[a]) * np.cos(k * g[b])
        rho = 1 - 3 * (u0 ** 2 / 4) * (np.cos(2 * k * g[a]) + np.cos(2 * k * g[b]))
        o = O.Oracle(p)
        o.init_fields(-np.ones(n ** 3), np.zeros(n ** 3), rho, *u)
        o.step(20, threads=4)
        f = o.fields()
        e1 = sum((f[c] ** 2).sum() for c in ("ux", "uy", "uz"))
        o.step(100, threads=4)
        f = o.fields()
        e2 = sum((f[c] ** 2).sum() for c in ("ux", "uy", "uz"))
        rate = -math.log(e2 / e1) / 100
        assert abs(rate / (4 * nu * k * k) - 1) < 2e-3, (plane, rate / (4 * nu * k * k))


def test_uniform_recurrence_3d(oracle_mod):
    p = p3(nx=3, ny=3, nz=3, lambda_=2.0, tau_phi0=0.8, w0=2.0, eps=0.04)
    o = O.Oracle(p)
    n = p.nodes
    phi, U = 0.1, 0.2
    o.init_fields(np.full(n, phi), np.full(n, U))
    t0 = 4.0 / (0.25 * 0.3)  # Eq. 23 with the D3Q7 cs^2 = 1/4
    prev = phi
    for _ in range(30):
        Q = phi - phi ** 3 + 2.0 * U * (1 - phi ** 2) ** 2
        prev, phi, U = phi, phi + Q / t0, U - (phi - prev)
        o.step(1)
        f = o.fields()
        assert abs(f["phi"][1, 1, 1] - phi) < 1e-13 and abs(f["U"][1, 1, 1] - U) < 1e-13


def test_conservation_and_cubic_symmetry_3d(oracle_mod):
    n = 24
    p = p3(nx=n, ny=n, nz=n, flow=1, eps=0.04, lambda_=-1.0)
    o = O.Oracle(p)
    o.init_seed(n / 2, n / 2, n / 2, 6.0, 0.5, 0.0, 1)
    d0 = o.diag(n // 2, n // 2, n // 2)
    o.step(60, threads=4)
    d1 = o.diag(n // 2, n // 2, n // 2)
    assert d1["solid_volume"] > 1.02 * d0["solid_volume"]
    assert abs(d1["solute_total"] / d0["solute_total"] - 1) < 1e-12
    assert abs(d1["mass_total"] / d0["mass_total"] - 1) < 1e-12
    phi = o.fields()["phi"]  # [z, y, x]
    for other in (np.transpose(phi, (0, 2, 1)), np.transpose(phi, (2, 1, 0)),
                  np.roll(phi[:, :, ::-1], 1, axis=2), np.roll(phi[::-1], 1, axis=0)):
        assert np.abs(phi - other).max() < 1e-12
    pos = d1["iface_pos"]
    assert np.ptp(pos) < 1e-9 and pos[0] > 6.0


@pytest.mark.parametrize("dim", [2, 3])
def test_inlet_outlet_uniform_inflow_is_stationary(oracle_mod, dim):
    # liquid at the inlet state (rho = 1, u = u_in e_x, U = U_in) is a fixed
    # point of the inlet ghost, the outlet copy and the periodic sides
    kw = dict(nx=12, ny=6, nz=4 if dim == 3 else 1, dim=dim, fold=0 if dim == 3 else 5,
              flow=1, eps=0.04, bc=(INLET_OUTLET, PERIODIC, PERIODIC),
              u_inlet=0.02, u0_inlet=0.3)
    p = Params(**kw)
    o = O.Oracle(p)
    n = p.nodes
    o.init_fields(-np.ones(n), np.full(n, 0.3), np.ones(n), np.full(n, 0.02), np.zeros(n),
                  np.zeros(n))
    before = {k: o.pops(k).copy() for k in "fgh"}
    o.step(30)
    for k in "fgh":
        np.testing.assert_allclose(o.pops(k), before[k], rtol=0, atol=1e-15)


def test_inlet_feeds_solute(oracle_mod):
    # a liquid at U = 0 fills with the inlet supersaturation from the left
    p = Params(nx=64, ny=4, flow=1, eps=0.0, lambda_=0.0, bc=(INLET_OUTLET, PERIODIC, PERIODIC),
               u_inlet=0.05, u0_inlet=0.3)
    o = O.Oracle(p)
    n = p.nodes
    o.init_fields(-np.ones(n), np.zeros(n), np.ones(n), np.full(n, 0.05), np.zeros(n))
    o.step(400)
    U = o.fields()["U"][0]
    assert abs(U[0] - 0.3) < 0.02 and U[-1] < 0.05
    assert np.all(np.diff(U) <= 1e-12)  # monotone front moving right


def test_default_lambda_matches_paper(oracle_mod):
    vals = {}
    with open(os.path.join(GOLDEN, "paper_lambda.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    # the paper's run in lattice units for an arbitrary time step dt
    dt = 0.2
    w0 = vals["W0_mm"] / vals["dr_mm"]
    tau0 = vals["tau0_s"] / dt
    D = vals["D_mm2_per_s"] * dt / vals["dr_mm"] ** 2
    p = Params(w0=w0, tau_phi0=w0 ** 2 / (tau0 / 3.0) + 0.5, tau_u_liquid=3.0 * D + 0.5)
    assert abs(O.tau0(p) - tau0) < 1e-12
    assert abs(O.coupling(p) - vals["lambda"]) < 5e-3
