"""Pins of the oracle's central Hermite MRT collision of the flow lattice.

Pinned against: the BGK collision with the product-form equilibrium (a
different formula: with every rate equal and no force the two coincide, since
the product form is the population whose nine central Hermite moments are
rho and zeros); the shear-wave (Taylor-Green) decay rate 2 nu k^2 with
nu = cs^2 (tau_f - 1/2) whatever the other rates; exact mass conservation and
momentum gain N F per step; and the stability the paper adopts it for, at a
viscosity where BGK fails.

In 3D (D3Q19) the same pins: BGK with the D3Q19 population whose raw moments
1, x, ..., x^2 y^2 (the nineteen monomials of exponents <= 2 in at most two
axes) are those of the Maxwellian, rho prod_d mu_k(u_d) with mu_0 = 1,
mu_1 = u, mu_2 = u^2 + cs^2 (built from raw monomials by a linear solve, no
Hermite polynomials and no shift); the shear-wave decay for each of the three
mixed second-order moments; mass and momentum.

The trace rate omega_bulk is pinned, in 2D and 3D, by the damping of a sound
wave: the acoustic energy of a standing density wave decays as
exp(-nu_L k^2 t) with the longitudinal viscosity nu_L = (2 - 2/D) nu + zeta,
zeta = (2/D) cs^2 (1/omega_bulk - 1/2) the bulk viscosity of a trace relaxed
at omega_bulk (for BGK, omega_bulk = 1/tau_f, the known zeta = 2 nu / D).
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


# ---- D3Q19 --------------------------------------------------------------------
C3 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
               [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1],
               [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
W3 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
EXPS = [(i, j, k) for i in range(3) for j in range(3) for k in range(3)
        if sum(e > 0 for e in (i, j, k)) <= 2]


def maxwell_d3q19(rho, u):
    """The D3Q19 populations whose raw moments prod_d c_d^e_d (the nineteen
    exponent triples) equal the Maxwellian's; rho: (n,), u: (3, n)."""
    assert len(EXPS) == 19
    M0 = np.array([[np.prod(c ** np.array(e)) for c in C3] for e in EXPS], dtype=float)
    mu = lambda k, v: np.ones_like(v) if k == 0 else (v if k == 1 else v * v + 1 / 3)
    rhs = np.stack([rho * mu(e[0], u[0]) * mu(e[1], u[1]) * mu(e[2], u[2]) for e in EXPS])
    return np.linalg.solve(M0, rhs)


def liquid3(**kw):
    base = dict(dim=3, nx=6, ny=5, nz=4, fold=0, flow=1, eps=0.0, lambda_=0.0, collision=1)
    base.update(kw)
    return Params(**base)


def test_d3q19_maxwell_equilibrium_at_rest_is_the_weights():
    rho = np.array([1.0, 0.9])
    f = maxwell_d3q19(rho, np.zeros((3, 2)))
    assert np.abs(f - W3[:, None] * rho).max() < 1e-15


def test_3d_equal_rates_give_bgk_with_the_maxwell_moments(orc):
    tau = 0.7
    p = liquid3(tau_f=tau, omega_bulk=1.0 / tau, omega_high=1.0 / tau)
    rng = np.random.default_rng(5)
    shape = (p.nz, p.ny, p.nx)
    u = 0.05 * rng.uniform(-1, 1, (3,) + shape)
    rho = 1.0 + 0.02 * rng.uniform(-1, 1, shape)
    o = O.Oracle(p)
    o.init_fields(-np.ones(shape), np.full(shape, 0.2), rho, u[0], u[1], u[2])
    f = o.pops("f").copy()
    for _ in range(3):
        r = f.sum(axis=0)
        v = np.stack([(C3[:, d, None, None, None] * f).sum(axis=0) / r for d in range(3)])
        feq = maxwell_d3q19(r.reshape(-1), v.reshape(3, -1)).reshape(f.shape)
        post = f - (f - feq) / tau
        f = np.stack([np.roll(post[a], (C3[a, 2], C3[a, 1], C3[a, 0]), axis=(0, 1, 2))
                      for a in range(19)])
    o.step(3)
    assert np.abs(o.pops("f") - f).max() < 1e-14, np.abs(o.pops("f") - f).max()


@pytest.mark.parametrize("comp,axis", [(0, 2), (1, 0), (2, 1)])
def test_3d_shear_wave_decay_follows_the_viscosity(orc, comp, axis):
    # u_comp = u0 sin(k x_axis): decays through the mixed moment of the pair
    # (BGK on this grid is off the continuum rate by the same 1e-3)
    n, tau, u0 = 64, 0.62, 1e-4
    dims = [4, 4, 4]
    dims[axis] = n
    p = liquid3(nx=dims[0], ny=dims[1], nz=dims[2], tau_f=tau, omega_bulk=1.3, omega_high=1.7)
    shape = (p.nz, p.ny, p.nx)
    coord = np.indices(shape)[2 - axis].astype(float)
    k = 2 * math.pi / n
    vel = [np.zeros(shape) for _ in range(3)]
    vel[comp] = u0 * np.sin(k * coord)
    o = O.Oracle(p)
    o.init_fields(-np.ones(shape), np.zeros(shape), None, *vel)
    steps = 600
    o.step(steps, 4)
    amp = np.abs(o.fields()[("ux", "uy", "uz")[comp]]).max()
    nu = (tau - 0.5) / 3.0
    assert abs(amp / (u0 * math.exp(-nu * k * k * steps)) - 1) < 2e-3


def test_3d_mass_conserved_and_momentum_gains_the_force(orc):
    b = (3e-6, -2e-6, 1e-6)
    p = liquid3(tau_f=0.55, body=b, omega_bulk=1.2, omega_high=1.4)
    rng = np.random.default_rng(6)
    shape = (p.nz, p.ny, p.nx)
    o = O.Oracle(p)
    o.init_fields(-np.ones(shape), np.full(shape, 0.1), 1 + 0.01 * rng.uniform(-1, 1, shape),
                  *(0.03 * rng.uniform(-1, 1, (3,) + shape)))

    def totals():
        f = o.pops("f")
        return [f.sum()] + [(C3[:, d, None, None, None] * f).sum() for d in range(3)]
    t0 = totals()
    o.step(40)
    t1 = totals()
    N = p.nodes
    assert abs(t1[0] / t0[0] - 1) < 1e-13
    for d in range(3):
        assert abs(t1[1 + d] - t0[1 + d] - 40 * N * b[d]) < 1e-11, d


@pytest.mark.parametrize("dim,wb", [(2, 1.0), (2, 1.4), (3, 1.0), (3, 1.4)])
def test_sound_wave_damping_follows_the_bulk_rate(orc, dim, wb):
    n, tau, steps = 64, 0.62, 600
    kw = dict(nx=4, ny=4, nz=n, fold=0) if dim == 3 else dict(nx=4, ny=n)
    p = (liquid3 if dim == 3 else liquid)(tau_f=tau, omega_bulk=wb, **kw)
    shape = p.shape
    k = 2 * math.pi / n
    o = O.Oracle(p)
    o.init_fields(-np.ones(shape), np.zeros(shape),
                  1 + 1e-4 * np.sin(k * np.indices(shape)[0].astype(float)))
    comp = "uz" if dim == 3 else "uy"
    energy = []
    for t in range(steps + 1):
        f = o.fields()
        energy.append(((f["rho"] - 1) ** 2 / 3 + f[comp] ** 2).sum())
        if t < steps:
            o.step(1)
    rate = -np.polyfit(np.arange(steps + 1), np.log(energy), 1)[0]
    nu = (tau - 0.5) / 3
    nu_l = (2 - 2 / dim) * nu + (2 / dim) * (1 / 3) * (1 / wb - 0.5)
    assert abs(rate / (nu_l * k * k) - 1) < 5e-3, rate / (nu_l * k * k)
