"""Pins of the FP64 oracle against what the model and mathematics fix.

Every test here runs on the CPU.  None re-types the oracle's update: each
checks a closed form, an invariant or a special case that reduces to a known
result, chosen so that a dropped term, a wrong sign, index or factor in the
oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import Params, PERIODIC, WALL


def liquid_params(**kw):
    base = dict(dim=2, nx=64, ny=64, flow=0, eps=0.0, lambda_=0.0)
    base.update(kw)
    return Params(**base)


# ---------------------------------------------------------------------------
# P6: uniform liquid and uniform solid are fixed points of the whole step.
@pytest.mark.parametrize("flow", [0, 1])
@pytest.mark.parametrize("phi0", [-1.0, 1.0])
def test_uniform_fixed_points(oracle_mod, flow, phi0):
    p = Params(nx=8, ny=8, flow=flow, eps=0.05, fold=5)
    o = O.Oracle(p)
    n = p.nodes
    o.init_fields(np.full(n, phi0), np.full(n, 0.3), np.ones(n), np.zeros(n), np.zeros(n))
    before = {k: o.pops(k).copy() for k in ("f", "g", "h")}
    o.step(25)
    for k in ("f", "g", "h"):
        np.testing.assert_allclose(o.pops(k), before[k], rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------
# P1: the solute lattice with phi = -1, u = 0 is pure diffusion with
# D = cs^2 (tau_U - 1/2) (Eq. 18); a Gaussian spreads as
# U = Uinf + A (s0^2 / s^2) exp(-r^2 / 2 s^2), s^2 = s0^2 + 2 D t.
def _gaussian_error(n, sigma0, steps, tau=0.8, u=(0.0, 0.0)):
    flow = 1 if any(u) else 0
    p = liquid_params(nx=n, ny=n, tau_u_liquid=tau, flow=flow)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    c = n / 2
    A, Uinf = 0.1, 0.2
    U0 = Uinf + A * np.exp(-((x - c) ** 2 + (y - c) ** 2) / (2 * sigma0 ** 2))
    o = O.Oracle(p)
    o.init_fields(-np.ones(n * n), U0, np.ones(n * n),
                  np.full(n * n, u[0]), np.full(n * n, u[1]))
    o.step(steps)
    D = (tau - 0.5) / 3.0
    s2 = sigma0 ** 2 + 2 * D * steps
    cx, cy = c + u[0] * steps, c + u[1] * steps
    exact = Uinf + A * (sigma0 ** 2 / s2) * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * s2))
    return np.abs(o.fields()["U"] - exact).max() / A


def test_gaussian_diffusion(oracle_mod):
    err = _gaussian_error(64, 4.0, 100)
    assert err < 4e-3, err
    # a diffusivity off by the 1/2 of Eq. 18 would be a 60 % error here;
    # halving dx / sigma cuts the error by 4 (second order in space)
    err_ref = _gaussian_error(128, 8.0, 400)
    assert err_ref < 1e-3, err_ref
    assert 3.5 < err / err_ref < 4.5, err / err_ref


def test_advected_gaussian(oracle_mod):
    # with phi = -1 the mask of Eq. 7 is the identity and the uniform flow is
    # stationary, so U is advected by u (Eq. 16) and diffuses
    err = _gaussian_error(64, 4.0, 200, u=(0.02, -0.01))
    assert err < 3e-3, err


# ---------------------------------------------------------------------------
# P3: Taylor-Green vortex in the liquid decays as exp(-2 nu k^2 t),
# nu = cs^2 (tau_f - 1/2) (Eq. 10).
def test_taylor_green_decay(oracle_mod):
    n, u0, tau = 64, 0.01, 0.6
    k = 2 * math.pi / n
    p = liquid_params(nx=n, ny=n, flow=1, tau_f=tau)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    ux = -u0 * np.cos(k * x) * np.sin(k * y)
    uy = u0 * np.sin(k * x) * np.cos(k * y)
    rho = 1.0 - 3.0 * (u0 ** 2 / 4.0) * (np.cos(2 * k * x) + np.cos(2 * k * y))
    o = O.Oracle(p)
    o.init_fields(-np.ones(n * n), np.zeros(n * n), rho, ux, uy)
    o.step(100)
    f1 = o.fields()
    e1 = (f1["ux"] ** 2 + f1["uy"] ** 2).sum()
    o.step(400)
    f2 = o.fields()
    e2 = (f2["ux"] ** 2 + f2["uy"] ** 2).sum()
    rate = -math.log(e2 / e1) / 400.0
    nu = (tau - 0.5) / 3.0
    assert abs(rate / (4 * nu * k * k) - 1.0) < 1e-3, rate / (4 * nu * k * k)


# ---------------------------------------------------------------------------
# P4: Poiseuille flow between half-way bounce-back walls driven by a body
# force (Guo forcing, Eq. 5): u(y) = b/(2 nu) (y+1/2)(H - y - 1/2), exact for
# BGK at tau_f = 1/2 + sqrt(3/16).
@pytest.mark.parametrize("tau,tol", [(0.5 + math.sqrt(3.0 / 16.0), 1e-6), (0.6, 4e-2)])
def test_poiseuille(oracle_mod, tau, tol):
    H, b = 16, 1e-6
    p = liquid_params(nx=4, ny=H, flow=1, tau_f=tau, bc=(PERIODIC, WALL, PERIODIC),
                      body=(b, 0.0, 0.0))
    o = O.Oracle(p)
    n = p.nodes
    o.init_fields(-np.ones(n), np.zeros(n), np.ones(n), np.zeros(n), np.zeros(n))
    o.step(25000)
    nu = (tau - 0.5) / 3.0
    y = np.arange(H) + 0.5
    exact = b / (2 * nu) * y * (H - y)
    got = o.fields()["ux"][:, 0]
    assert np.abs(got / exact - 1).max() < tol, np.abs(got / exact - 1).max()


# ---------------------------------------------------------------------------
# P2: with U = 0 and lambda = 0, Eq. 1 is Allen-Cahn; a planar interface is
# stationary with profile tanh(s / (sqrt(2) W0 a_s)).  With anisotropy the
# gradient term of Eq. 1 has width W0 a_s(n) while the flux N is divergence
# free for a planar front, so the width follows a_s of the front's normal.
def _slab_error(w0, eps=0.0, diag=False, steps=1500):
    n = 128
    p = Params(nx=n, ny=4 if not diag else n, flow=0, eps=eps, fold=4, lambda_=0.0, w0=w0)
    y, x = np.mgrid[0:p.ny, 0:n].astype(float)
    if not diag:
        s = (n / 4 - np.abs(x - n / 2))
        a = 1.0 + eps  # normal along x: theta = 0 or pi
    else:
        xi = (x + y) % n
        s = (n / 4 - np.abs(xi - n / 2)) / math.sqrt(2.0)
        a = 1.0 - eps  # normal along the diagonal: cos(4 * pi/4) = -1
    o = O.Oracle(p)
    exact = np.tanh(s / (math.sqrt(2.0) * w0 * a))
    iso = np.tanh(s / (math.sqrt(2.0) * w0))
    o.init_fields(iso.reshape(-1), np.zeros(p.nodes))
    o.step(steps, threads=4)
    phi = o.fields()["phi"]
    return np.abs(phi - exact).max(), np.abs(phi - iso).max()


def test_tanh_interface_stationary(oracle_mod):
    e2, _ = _slab_error(2.0)
    e4, _ = _slab_error(4.0)
    assert e2 < 2e-2, e2
    assert e4 < e2 / 3.5, (e2, e4)  # second order in dx / W0


@pytest.mark.parametrize("diag", [False, True])
def test_anisotropic_planar_width(oracle_mod, diag):
    err, err_iso = _slab_error(4.0, eps=0.05, diag=diag, steps=4000)
    assert err < 5e-3, err
    assert err_iso > 4 * err  # the width really changed to W0 a_s


# ---------------------------------------------------------------------------
# Uniform states reduce Eqs. 13-23 to scalar recurrences: summing Eq. 19 over
# the directions with a_s = 1, N = 0 gives the forward-Euler step of
# tau0 dphi/dt = Q (Eq. 1 without gradients), and summing Eq. 13 with Eq. 14
# gives U(t+1) = U(t) - (phi(t) - phi(t-1)) (Eq. 2 without transport).
def test_uniform_phase_solute_recurrence(oracle_mod):
    p = Params(nx=4, ny=4, flow=0, eps=0.05, lambda_=2.5, tau_phi0=0.9, w0=1.5)
    o = O.Oracle(p)
    n = p.nodes
    phi, U = -0.2, 0.35
    o.init_fields(np.full(n, phi), np.full(n, U))
    t0 = 1.5 ** 2 / ((1.0 / 3.0) * (0.9 - 0.5))  # Eq. 23 at a_s = 1
    phi_prev = phi
    for _ in range(60):
        Q = phi - phi ** 3 + 2.5 * U * (1 - phi ** 2) ** 2
        dphi = phi - phi_prev
        phi_prev, phi, U = phi, phi + Q / t0, U - dphi
        o.step(1)
        f = o.fields()
        assert abs(f["phi"][0, 0] - phi) < 1e-13
        assert abs(f["U"][0, 0] - U) < 1e-13
    assert phi > 0.2  # the supersaturated liquid solidifies towards phi = 1


# The flow lattice at uniform phi = 0 with a uniform velocity: the moments of
# Eq. 4 with Eq. 5-9 give m(t+1) = m - (m - rho u*)/tau + (1 - 1/(2 tau)) F,
# u = m / (rho + K/2), F = -K u, u* = u/2, K = h tau (1+0)^2 (1-0)/(4 W0^2).
# The central Hermite MRT (collision = 1) relaxes the first-order moments
# about u* at the same rate with the same force term: the same recurrence.
@pytest.mark.parametrize("collision", [0, 1])
def test_uniform_drag_recurrence(oracle_mod, collision):
    p = Params(nx=4, ny=4, flow=1, eps=0.0, lambda_=0.0, tau_f=0.7, w0=2.0,
               collision=collision)
    o = O.Oracle(p)
    n = p.nodes
    u0 = np.array([0.03, -0.02])
    o.init_fields(np.zeros(n), np.zeros(n), np.ones(n), np.full(n, u0[0]), np.full(n, u0[1]))
    K = 2.757 * 0.7 / (4 * 4.0)
    m = 0.5 * u0  # initial populations are at equilibrium with u* = u/2
    for _ in range(40):
        u = m / (1.0 + K / 2)
        F = -K * u
        m = m - (m - 0.5 * u) / 0.7 + (1 - 1 / 1.4) * F
        o.step(1)
        f = o.fields()
        np.testing.assert_allclose([f["ux"][1, 1], f["uy"][1, 1]], m / (1 + K / 2),
                                   rtol=0, atol=1e-15)
        assert abs(f["phi"][1, 1]) < 1e-15 and abs(f["rho"][1, 1] - 1) < 1e-14


# The same recurrence on the D3Q19 lattice with a three-component velocity.
@pytest.mark.parametrize("collision", [0, 1])
def test_uniform_drag_recurrence_3d(oracle_mod, collision):
    p = Params(dim=3, nx=4, ny=4, nz=4, fold=0, flow=1, eps=0.0, lambda_=0.0, tau_f=0.7,
               w0=2.0, collision=collision)
    o = O.Oracle(p)
    n = p.nodes
    u0 = np.array([0.03, -0.02, 0.015])
    o.init_fields(np.zeros(n), np.zeros(n), np.ones(n), *(np.full(n, v) for v in u0))
    K = 2.757 * 0.7 / (4 * 4.0)
    m = 0.5 * u0
    for _ in range(40):
        u = m / (1.0 + K / 2)
        F = -K * u
        m = m - (m - 0.5 * u) / 0.7 + (1 - 1 / 1.4) * F
        o.step(1)
        f = o.fields()
        np.testing.assert_allclose([f["ux"][1, 2, 3], f["uy"][1, 2, 3], f["uz"][1, 2, 3]],
                                   m / (1 + K / 2), rtol=0, atol=1e-15)
        assert abs(f["phi"][1, 2, 3]) < 1e-15 and abs(f["rho"][1, 2, 3] - 1) < 1e-14


# ---------------------------------------------------------------------------
# P5: periodic domain: sum_x [U(t) + phi(t-1)] and sum rho are invariants.
@pytest.mark.parametrize("flow", [0, 1])
def test_conservation(oracle_mod, flow):
    p = Params(nx=48, ny=40, flow=flow, eps=0.05, fold=5, u_inlet=0.0)
    o = O.Oracle(p)
    o.init_seed(20.0, 21.0, 0.0, 6.0, 0.4, 0.01, 7)
    if flow:  # stir the liquid so that the drag and mask are exercised
        f = o.fields()
        y, x = np.mgrid[0:40, 0:48].astype(float)
        o.init_fields(f["phi"], f["U"], np.ones(p.nodes),
                      0.02 * np.sin(2 * np.pi * y / 40), 0.01 * np.cos(2 * np.pi * x / 48))
    d0 = o.diag(20, 21)
    o.step(150)
    d1 = o.diag(20, 21)
    assert d1["solid_volume"] > d0["solid_volume"] * 1.02  # it really grew
    assert abs(d1["solute_total"] / d0["solute_total"] - 1) < 1e-12
    assert abs(d1["mass_total"] / d0["mass_total"] - 1) < 1e-12


# ---------------------------------------------------------------------------
# P7: k-fold symmetry of a noiseless centred seed.
def test_fourfold_symmetry(oracle_mod):
    n = 48
    p = Params(nx=n, ny=n, flow=0, eps=0.05, fold=4)
    o = O.Oracle(p)
    o.init_seed(n / 2, n / 2, 0, 6.0, 0.4, 0.0, 1)
    o.step(200)
    phi = o.fields()["phi"]
    # node i <-> n - i (mod n) keeps the centre n/2 fixed
    mirror_x = np.roll(phi[:, ::-1], 1, axis=1)
    mirror_y = np.roll(phi[::-1, :], 1, axis=0)
    rot = np.roll(np.rot90(phi), 1, axis=0)
    for other in (mirror_x, mirror_y, rot, phi.T):
        assert np.abs(phi - other).max() < 1e-12


def test_fivefold_mirror(oracle_mod):
    n = 48
    p = Params(nx=n, ny=n, flow=0, eps=0.05, fold=5)
    o = O.Oracle(p)
    o.init_seed(n / 2, n / 2, 0, 6.0, 0.4, 0.0, 1)
    o.step(300)
    phi = o.fields()["phi"]
    assert np.abs(phi - np.roll(phi[::-1, :], 1, axis=0)).max() < 1e-12
    # and not mirror symmetric in x: 5-fold has no x -> -x symmetry
    assert np.abs(phi - np.roll(phi[:, ::-1], 1, axis=1)).max() > 1e-4


# P11: integer shifts of the initial state commute with the step.
def test_translation_invariance(oracle_mod):
    p = Params(nx=32, ny=24, flow=1, eps=0.05, fold=5)
    rng = np.random.default_rng(3)
    y, x = np.mgrid[0:24, 0:32].astype(float)
    phi = np.tanh((6 - np.hypot(x - 12, y - 10)) / (2 * math.sqrt(2))) + 0.01 * rng.uniform(-1, 1, x.shape)
    U = 0.3 + 0.01 * rng.uniform(-1, 1, x.shape)
    ux = 0.01 * rng.uniform(-1, 1, x.shape)
    uy = 0.01 * rng.uniform(-1, 1, x.shape)
    sh = (5, 7)
    a = O.Oracle(p)
    a.init_fields(phi, U, None, ux, uy)
    b = O.Oracle(p)
    b.init_fields(*(np.roll(v, sh, axis=(0, 1)) for v in (phi, U, np.ones_like(phi), ux, uy)))
    a.step(20)
    b.step(20)
    fa, fb = a.fields(), b.fields()
    for k in ("phi", "U", "rho", "ux", "uy"):
        assert np.array_equal(np.roll(fa[k], sh, axis=(0, 1)), fb[k]), k


# ---------------------------------------------------------------------------
# P8: N of Eq. 21 equals (1/2)|grad phi|^2 d(a_s^2)/d(grad phi) (central
# differences), and a_s follows Eq. 3 at known normals.
@pytest.mark.parametrize("dim,fold", [(2, 4), (2, 5), (2, 6), (3, 0), (2, 0)])
def test_aniso_flux_identity(oracle_mod, dim, fold):
    p = Params(dim=dim, fold=fold, eps=0.04, theta0=0.3 if fold else 0.0)
    rng = np.random.default_rng(11)
    for _ in range(50):
        g = rng.normal(size=3) * rng.uniform(0.05, 2.0)
        if dim == 2:
            g[2] = 0.0
        a, N = O.aniso(p, g)
        fd = np.zeros(3)
        h = 1e-6
        for d in range(dim):
            e = np.zeros(3)
            e[d] = h
            ap, _ = O.aniso(p, g + e)
            am, _ = O.aniso(p, g - e)
            fd[d] = 0.5 * (g @ g) * (ap * ap - am * am) / (2 * h)
        np.testing.assert_allclose(N, fd, rtol=0, atol=1e-8 * max(1.0, np.abs(fd).max()))
    lit = Params(dim=dim, fold=fold, eps=0.04, aniso_literal=1)
    g = np.array([0.3, -0.2, 0.1 if dim == 3 else 0.0])
    _, N0 = O.aniso(Params(dim=dim, fold=fold, eps=0.04), g)
    _, N1 = O.aniso(lit, g)
    np.testing.assert_allclose(N1, 2 * N0, rtol=1e-15)


def test_aniso_known_values(oracle_mod):
    # normal n = -grad/|grad|: a gradient along -x is a normal along +x
    for k in (4, 5, 6):
        p = Params(fold=k, eps=0.05)
        assert abs(O.aniso(p, [-1, 0, 0])[0] - 1.05) < 1e-15
        assert abs(O.aniso(p, [1, 0, 0])[0] - (1 + 0.05 * math.cos(k * math.pi))) < 1e-15
        t = 2 * math.pi / (3 * k)
        g = -np.array([math.cos(t), math.sin(t), 0.0])
        assert abs(O.aniso(p, g)[0] - (1 + 0.05 * math.cos(k * t))) < 1e-14
    p = Params(fold=4, eps=0.05, theta0=math.pi / 4)
    assert abs(O.aniso(p, [-1, 0, 0])[0] - 0.95) < 1e-14
    # cubic 3D: a_s along <100> is 1 + eps, along <111> 1 - 5 eps / 3
    p = Params(dim=3, fold=0, eps=0.04)
    assert abs(O.aniso(p, [0, 0, -2])[0] - 1.04) < 1e-15
    assert abs(O.aniso(p, [1, 1, 1])[0] - (1 - 5 * 0.04 / 3)) < 1e-14
    assert O.aniso(p, [0, 0, 0])[0] == 1.0


def test_normal_points_out_of_the_crystal(oracle_mod):
    # on a seed, the node right of the centre has its normal along +x
    # (theta = 0) and the node left of it along -x (theta = pi); with k = 5
    # a_s differs between the two sides by 2 eps
    n = 64
    p = Params(nx=n, ny=n, fold=5, eps=0.05)
    o = O.Oracle(p)
    o.init_seed(32, 32, 0, 10.0, 0.3, 0.0, 1)
    a = o.aux()["a_s"]
    assert abs(a[32, 42] - 1.05) < 2e-3
    assert abs(a[32, 22] - 0.95) < 2e-3
    assert o.aux()["gx"][32, 42] < 0  # phi decreases outward


# The anisotropic flux N turns the stiffness a + a'' = 1 - 15 eps cos 4 theta
# to a minimum along the axes, so a 4-fold seed grows fastest along x and y
# (without N, or with N's sign flipped, the diagonals win).
def _crossing(vals):
    for d in range(1, len(vals)):
        if vals[d] < 0:
            return (d - 1) + vals[d - 1] / (vals[d - 1] - vals[d])
    return float("nan")


def test_fourfold_growth_habit(oracle_mod):
    # ratio of the axis to the diagonal interface distance: about 1.11 with N
    # as read, 0.99 with N dropped and 0.89 with N's sign flipped
    n = 96
    p = Params(nx=n, ny=n, fold=4, eps=0.05)
    o = O.Oracle(p)
    o.init_seed(n / 2, n / 2, 0, 6.0, 0.45, 0.0, 1)
    o.step(1500, threads=4)
    phi = o.fields()["phi"]
    c = n // 2
    axis = _crossing(phi[c, c:])
    diag = _crossing(np.array([phi[c + d, c + d] for d in range(c)])) * math.sqrt(2)
    assert axis > 1.05 * diag, (axis, diag)
