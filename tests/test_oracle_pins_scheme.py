"""Pins of the oracle's scheme as a whole, each against a result that the
phase-field model or the transport equations fix independently of the code:

- the relaxation rate of a perturbed planar front, which depends on the
  anisotropic flux N of Eq. 21 through the interface stiffness a_s + a_s''
  (the sharp-interface limit of the model);
- second-order self-convergence of the phi profile under refinement at fixed
  physical size (the paper's own validation, Sec. 3.1.1, error norm Eq. 25);
- a solute pulse carried out through the zero-gradient outlet: it follows the
  free-space advection-diffusion solution up to the last node and leaves no
  reflection.
"""
import os

import numpy as np
import pytest

import oracle as O
from oracle import INLET_OUTLET, PERIODIC, Params

THREADS = max(1, min(8, os.cpu_count() or 1))


# ---------------------------------------------------------------------------
# Anisotropic stiffness.  With U decoupled (lambda = 0) the model is the
# anisotropic Allen-Cahn equation tau0 a_s^2 d_t phi = W0^2 div(a_s^2 grad phi)
# + W0^2 div N + phi - phi^3.  Its sharp-interface limit (Karma & Rappel,
# Phys. Rev. E 57, 4323 (1998): capillary length d0 ~ W0 (a_s + a_s''),
# kinetic coefficient beta ~ tau0 a_s / W0) moves the front by curvature
# alone, V_n = -(d0 / beta) kappa = -(W0^2/tau0) (a_s + a_s'')/a_s kappa.  A
# front displaced by A cos(q s) along its tangent s therefore relaxes as
# A(t) = A0 exp(-sigma t) with
#   sigma = (W0^2 / tau0) (a_s(theta) + a_s''(theta)) / a_s(theta) q^2.
# The stiffness a_s + a_s'' exists only through N: for a_s = 1 + eps cos 4 theta
# it is 1 - 15 eps at theta = 0 and 1 + 15 eps at theta = pi/4, where a model
# without N, with the literal factor 2 of Eq. 21, or with N of the wrong sign
# or scale relaxes at another rate.
def _front_rate(theta_deg, eps, literal=0, n=128, w0=2.0, steps=3000):
    p = Params(nx=n, ny=n, fold=4, eps=eps, lambda_=0.0, w0=w0, aniso_literal=literal)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    a0 = 2.0
    if theta_deg == 0:
        # two fronts normal to x (at n/4 and 3n/4), displaced along y
        q = 2 * np.pi / n
        s, per, pert = x, float(n), a0 * np.cos(q * y)
    else:
        # two fronts normal to (1, 1): s = (x + y)/sqrt 2 is periodic with
        # period n/sqrt 2 on the torus; the displacement varies along y - x
        q = 2 * np.pi / (n / np.sqrt(2))
        per = n / np.sqrt(2)
        s, pert = np.mod((x + y) / np.sqrt(2), per), a0 * np.cos(2 * np.pi * (y - x) / n)
    d1, d2 = s - per / 4 - pert, s - 3 * per / 4 - pert
    phi = np.tanh(d1 / (np.sqrt(2) * w0)) - np.tanh(d2 / (np.sqrt(2) * w0)) - 1.0
    o = O.Oracle(p)
    o.init_fields(phi, np.zeros_like(phi))
    ts, amps = [], []
    every = 250
    for k in range(steps // every + 1):
        if k:
            o.step(every, THREADS)
        ts.append(k * every)
        amps.append(_front_amplitude(o.fields()["phi"], theta_deg))
    ts, amps = np.array(ts, float), np.abs(np.array(amps))
    # the rate from the last two thirds (the initial tanh profile adjusts first)
    k0 = len(ts) // 3
    rates = [-np.polyfit(ts[k0:], np.log(amps[k0:, j]), 1)[0] for j in range(2)]
    th = np.deg2rad(theta_deg)
    a_s = 1 + eps * np.cos(4 * th)
    a_s2 = -16 * eps * np.cos(4 * th)  # d^2 a_s / d theta^2
    sigma = w0 * w0 / O.tau0(p) * (a_s + a_s2) / a_s * q * q
    return np.array(rates), sigma


def _front_amplitude(phi, theta_deg):
    """Amplitude of the cos displacement mode of the rising and the falling
    front, from the phi = 0 crossing of every row (linear interpolation)."""
    n = phi.shape[0]
    out = []
    for rising in (True, False):
        pos, tang = [], []
        for yy in range(n):
            row = phi[yy]
            for xx in range(n):
                a, b = row[xx], row[(xx + 1) % n]
                if (a < 0) != (b < 0) and (a < 0) == rising:
                    xc = xx + a / (a - b)
                    break
            if theta_deg == 0:
                pos.append(xc)
                tang.append(2 * np.pi * yy / n)
            else:
                pos.append((xc + yy) / np.sqrt(2))
                tang.append(2 * np.pi * (yy - xc) / n)
        pos, c = np.array(pos), np.cos(np.array(tang))
        if theta_deg != 0:  # positions along the normal are periodic: unwrap
            per = n / np.sqrt(2)
            pos = pos - per * np.round((pos - np.median(pos)) / per)
        pos = pos - pos.mean()
        out.append(np.sum(pos * c) / np.sum(c * c))
    return out


@pytest.mark.parametrize("theta_deg", [0, 45])
def test_perturbed_front_relaxes_with_the_anisotropic_stiffness(oracle_mod, theta_deg):
    rates, sigma = _front_rate(theta_deg, eps=0.02)
    # measured 1.031 (theta = 0) and 1.004 (45 deg); the isotropic front (eps =
    # 0) is off by 2 % from lattice and finite-width effects.  The literal
    # factor 2 gives 0.59 / 1.24, N of the wrong sign 1.94 / 0.53, N three
    # times too large 1.33 / 0.85 (checked once each against a planted copy)
    np.testing.assert_allclose(rates / sigma, 1.0, atol=0.06)
    assert abs(rates[0] - rates[1]) <= 1e-9 * abs(rates[0])  # the two fronts alike


def test_literal_flux_factor_changes_the_relaxation(oracle_mod):
    # the same measurement discriminates: with the literal factor of Eq. 21 the
    # rate at theta = 0 is far below the variational model's closed form
    rates, sigma = _front_rate(0, eps=0.02, literal=1)
    assert rates[0] / sigma < 0.8, rates / sigma


# ---------------------------------------------------------------------------
# Self-convergence (Sec. 3.1.1, Eq. 25).  A hexagonal-anisotropy seed on grids
# of N, 2N, 4N nodes over the same physical domain: W0, the seed radius and
# the grid scale with the resolution, the time steps with its square
# (diffusive scaling keeps tau_phi0, tau_U and lambda in lattice units), and
# the phi profile along the centre line from the centre to the +x edge is
# compared at the coarse grid's node positions.  The l2 relative error of
# Eq. 25 between successive grids falls as the square of the spacing.
def test_self_convergence_is_second_order(oracle_mod):
    base, t0, w = 48, 160, 1.5
    prof = []
    for lev in range(3):
        n, s = base * 2 ** lev, 2 ** lev
        p = Params(nx=n, ny=n, fold=6, eps=0.02, w0=w * s, theta0=0.2)
        o = O.Oracle(p)
        o.init_seed(n / 2, n / 2, 0.0, base / 6 * s, 0.3, 0.0, 1)
        o.step(t0 * 4 ** lev, THREADS)
        phi = o.fields()["phi"]
        prof.append(phi[n // 2, n // 2: n // 2 + (base // 2) * s + 1: s])

    def e_l2(a, ref):  # Eq. 25
        return np.sqrt(np.sum((a - ref) ** 2) / np.sum(ref ** 2))

    e1, e2 = e_l2(prof[0], prof[1]), e_l2(prof[1], prof[2])
    order = np.log2(e1 / e2)
    # measured 1.94 (the paper reports slope -2); the interface crosses the line
    assert 1.7 <= order <= 2.3, (e1, e2, order)
    assert prof[2].max() > 0.9 and prof[2].min() < -0.9


# ---------------------------------------------------------------------------
# Zero-gradient outlet.  A solute pulse in a uniform liquid flow u along x
# (phi = -1, so u* = u and the flow is stationary) is carried to the outlet and
# out.  Inside the domain it is the free-space solution
#   U = U_inf + A (s0/s) exp(-(x - x0 - u t)^2 / (2 s^2)),  s^2 = s0^2 + 2 D t,
# D = cs^2 (tau_U - 1/2), also on the last nodes while it crosses the outlet
# (a zero-gradient outlet is transparent to an advection-dominated pulse), and
# nothing is reflected.  The outlet ghost copying node nx - 2 instead of nx - 1
# gives 3.1 % here, a bounce-back outlet reflects the pulse (> 50 %).
def test_pulse_leaves_through_the_outlet_without_reflection(oracle_mod):
    nx, ny = 256, 4
    u, u_inf, amp, x0, s0 = 0.08, 0.3, 0.1, 150.0, 8.0
    p = Params(nx=nx, ny=ny, flow=1, bc=(INLET_OUTLET, PERIODIC, PERIODIC), u_inlet=u,
               u0_inlet=u_inf, tau_u_liquid=0.55, eps=0.0)
    x = np.arange(nx, dtype=float)
    U0 = np.tile(u_inf + amp * np.exp(-(x - x0) ** 2 / (2 * s0 ** 2)), (ny, 1))
    o = O.Oracle(p)
    one = np.ones_like(U0)
    o.init_fields(-one, U0, one, u * one, 0 * one)
    D = (p.tau_u_liquid - 0.5) / 3.0
    for t in (800, 1325, 1450, 1600, 1750, 2400):
        o.step(t - o.step_count, THREADS)
        s2 = s0 ** 2 + 2 * D * t
        peak = amp * s0 / np.sqrt(s2)
        exact = u_inf + peak * np.exp(-(x - x0 - u * t) ** 2 / (2 * s2))
        U = o.fields()["U"]
        assert np.abs(U - U[0]).max() < 1e-14  # uniform across y
        err = np.abs(U[0] - exact).max() / peak
        # measured <= 0.92 % (largest when the peak has just left, t = 1450)
        assert err < 0.015, (t, err)
    # the pulse is gone: no reflected remainder
    assert np.abs(U - u_inf).max() < 1e-6 * amp
