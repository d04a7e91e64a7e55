"""Pins of the oracle's central Hermite MRT collision of the flow lattice.

Pinned against: the BGK collision with the product-form equilibrium (a
different formula: with every rate equal and no force the two coincide, since
the product form is the population whose nine central Hermite moments are
rho and zeros); the shear-wave (Taylor-Green) decay rate 2 nu k^2 with
nu = cs^2 (tau_f - 1/2) whatever the other rates; exact mass conservation and
momentum gain N F per step; and the stability the paper adopts it for, at a
viscosity where BGK fails.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import Params

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


@pytest.fixture(scope="module")
def orc(oracle_mod):
    return oracle_mod


def liquid(**kw):
    base = dict(dim=2, nx=24, ny=20, flow=1, eps=0.0, lambda_=0.0, collision=1)
    base.update(kw)
    return Params(**base)


def product_equilibrium(rho, ux, uy):
    def psi(c, u):
        return np.where(c == 0, 2.0 / 3.0 - u * u, 1.0 / 6.0 + 0.5 * c * u + 0.5 * u * u)
    return np.stack([rho * psi(cx, ux) * psi(cy, uy) for cx, cy in zip(CX, CY)])


def test_equal_rates_give_bgk_with_the_product_equilibrium(orc):
    tau = 0.7
    p = liquid(tau_f=tau, omega_bulk=1.0 / tau, omega_high=1.0 / tau)
    rng = np.random.default_rng(1)
    shape = (p.ny, p.nx)
    ux, uy = 0.05 * rng.uniform(-1, 1, shape), 0.05 * rng.uniform(-1, 1, shape)
    rho = 1.0 + 0.02 * rng.uniform(-1, 1, shape)
    o = O.Oracle(p)
    o.init_fields(-np.ones(shape), np.full(shape, 0.2), rho, ux, uy)
    f = o.pops("f").copy()  # second-order Hermite equilibrium: not the product form
    for _ in range(3):
        r = f.sum(axis=0)
        vx = (CX[:, None, None] * f).sum(axis=0) / r
        vy = (CY[:, None, None] * f).sum(axis=0) / r
        post = f - (f - product_equilibrium(r, vx, vy)) / tau
        f = np.stack([np.roll(post[a], (CY[a], CX[a]), axis=(0, 1)) for a in range(9)])
    o.step(3)
    assert np.abs(o.pops("f") - f).max() < 1e-14, np.abs(o.pops("f") - f).max()


@pytest.mark.parametrize("wb,wh", [(0.0, 0.0), (1.3, 1.7)])
def test_shear_wave_decay_follows_the_viscosity(orc, wb, wh):
    n, tau, u0 = 64, 0.62, 1e-4
    p = liquid(nx=n, ny=n, tau_f=tau, omega_bulk=wb, omega_high=wh)
    o = O.Oracle(p)
    y = np.arange(n, dtype=float)[:, None] * np.ones((1, n))
    k = 2 * math.pi / n
    o.init_fields(-np.ones((n, n)), np.zeros((n, n)), None, u0 * np.sin(k * y), None)
    steps = 600
    o.step(steps)
    amp = np.abs(o.fields()["ux"]).max()
    nu = (tau - 0.5) / 3.0
    assert abs(amp / (u0 * math.exp(-nu * k * k * steps)) - 1) < 2e-3


def test_mass_conserved_and_momentum_gains_the_force(orc):
    b = (3e-6, -2e-6, 0.0)
    p = liquid(tau_f=0.55, body=b)
    rng = np.random.default_rng(2)
    shape = (p.ny, p.nx)
    o = O.Oracle(p)
    o.init_fields(-np.ones(shape), np.full(shape, 0.1), 1 + 0.01 * rng.uniform(-1, 1, shape),
                  0.03 * rng.uniform(-1, 1, shape), 0.03 * rng.uniform(-1, 1, shape))

    def totals():
        f = o.pops("f")
        return f.sum(), (CX[:, None, None] * f).sum(), (CY[:, None, None] * f).sum()
    m0, px0, py0 = totals()
    o.step(40)
    m1, px1, py1 = totals()
    N = p.nx * p.ny
    assert abs(m1 / m0 - 1) < 1e-13
    assert abs(px1 - px0 - 40 * N * b[0]) < 1e-11 and abs(py1 - py0 - 40 * N * b[1]) < 1e-11


def test_stable_where_bgk_fails(orc):
    # a double shear layer at tau_f = 0.5005 (viscosity 1.7e-4, Re about 4e4
    # on this grid): BGK diverges within 500 steps; the central Hermite MRT
    # with its default rates (trace and higher orders at 1) stays bounded;
    # with the trace at 1/tau_f instead it diverges too (by step 1500)
    n = 64
    y, x = np.mgrid[0:n, 0:n].astype(float)
    ux = 0.1 * np.tanh(80 * (np.minimum(y, n - y) / n - 0.25))
    uy = 0.005 * np.sin(2 * math.pi * x / n)

    def run(collision, wb=0.0):
        p = liquid(nx=n, ny=n, tau_f=0.5005, collision=collision, omega_bulk=wb)
        o = O.Oracle(p)
        o.init_fields(-np.ones((n, n)), np.zeros((n, n)), None, ux, uy)
        for _ in range(6):
            o.step(500)
            f = o.fields()
            m = np.abs(np.stack([f["ux"], f["uy"]])).max()
            if not np.isfinite(m) or m > 1.0:
                return m
        return m
    bgk, chm, chm_wf = run(0), run(1), run(1, 1.0 / 0.5005)
    assert not np.isfinite(bgk) or bgk > 1.0, bgk
    assert np.isfinite(chm) and chm < 0.2, chm
    assert not np.isfinite(chm_wf) or chm_wf > 1.0, chm_wf
