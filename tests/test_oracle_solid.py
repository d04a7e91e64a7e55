"""Pins of the oracle's solid nodes (walls and obstacles; the paper's reactor
walls and baffles, Sec. 3.1.2 and Sec. 3.2): half-way bounce-back for f, g
and h, frozen solid nodes, zero normal phi-derivative in the gradient.

Pinned against: the closed-form Poiseuille profile in a channel cut out of a
periodic domain by solid rows; the domain walls (rows of solid nodes inside
the grid reproduce the wall boundary condition, whose own pin is the
Poiseuille profile of test_oracle_pins); conservation of mass and of the
solute invariant around obstacles; mirror symmetry; fixed points.  The same
in 3D (D3Q19 flow, D3Q7 solute and phase field): planes of solid nodes
against the domain walls normal to y and to z, Poiseuille flow between solid
planes, conservation, mirror symmetry and rest around 3D obstacles.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import Params, PERIODIC, WALL, INLET_OUTLET


@pytest.fixture(scope="module")
def orc(oracle_mod):
    return oracle_mod


def test_poiseuille_in_a_masked_channel(orc):
    # walls at rows 3 and 20 of a periodic 24-row domain: the fluid rows 4..19
    # see half-way walls at y = 3.5 and 19.5, exactly as the domain walls
    tau, H, b = 0.5 + math.sqrt(3.0 / 16.0), 16, 1e-6
    ny = 24
    p = Params(nx=4, ny=ny, flow=1, tau_f=tau, eps=0.0, lambda_=0.0,
               bc=(PERIODIC, PERIODIC, PERIODIC), body=(b, 0.0, 0.0))
    o = O.Oracle(p)
    mask = np.zeros((ny, 4), np.uint8)
    mask[3, :] = mask[20, :] = 1
    o.set_solid(mask)
    n = p.nodes
    o.init_fields(-np.ones(n), np.zeros(n), np.ones(n), np.zeros(n), np.zeros(n))
    f0 = o.pops("f")
    o.step(25000)
    nu = (tau - 0.5) / 3.0
    y = np.arange(H) + 0.5
    exact = b / (2 * nu) * y * (H - y)
    got = o.fields()["ux"][4:20, 0]
    assert np.abs(got / exact - 1).max() < 1e-6, np.abs(got / exact - 1).max()
    # the solid rows kept their initial state
    assert np.array_equal(o.pops("f")[:, [3, 20]], f0[:, [3, 20]])


@pytest.mark.parametrize("flow,collision", [(0, 0), (1, 0), (1, 1)])
def test_solid_rows_reproduce_the_domain_walls(orc, flow, collision):
    # A: periodic x, walls in y, ny = 30.  B: periodic x and y, ny = 32, rows
    # 0 and 31 solid.  Same fields on the fluid rows (a seed touching the
    # lower wall, so that the gradient next to the wall is exercised).
    nx, ny = 40, 30
    kw = dict(nx=nx, flow=flow, eps=0.04, fold=4, theta0=0.3, collision=collision,
              body=(2e-6, 0.0, 0.0) if flow else (0.0, 0.0, 0.0))
    pa = Params(ny=ny, bc=(PERIODIC, WALL, PERIODIC), **kw)
    pb = Params(ny=ny + 2, bc=(PERIODIC, PERIODIC, PERIODIC), **kw)
    rng = np.random.default_rng(3)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    phi = np.tanh((7.0 - np.hypot(x - 17.3, y - 3.2)) / (math.sqrt(2) * 2.0))
    phi += 0.01 * rng.uniform(-1, 1, phi.shape)
    U = 0.35 + 0.01 * rng.uniform(-1, 1, phi.shape)
    ux = 0.01 * np.sin(2 * np.pi * y / ny) if flow else np.zeros_like(phi)
    a = O.Oracle(pa)
    a.init_fields(phi, U, None, ux, None)
    pad = lambda f, v: np.concatenate([np.full((1, nx), v), f, np.full((1, nx), v)])
    b = O.Oracle(pb)
    b.init_fields(pad(phi, -1.0), pad(U, 0.35), None, pad(ux, 0.0), None)
    mask = np.zeros((ny + 2, nx), np.uint8)
    mask[0, :] = mask[-1, :] = 1
    b.set_solid(mask)
    a.step(200)
    b.step(200)
    fa, fb = a.fields(), b.fields()
    for k in ("phi", "U", "rho", "ux", "uy"):
        assert np.abs(fa[k] - fb[k][1:-1]).max() < 1e-13, k
    for k in "fgh":
        if k == "f" and not flow:
            continue
        assert np.abs(a.pops(k) - b.pops(k)[:, 1:-1]).max() < 1e-13, k
    a.close()
    b.close()


def baffle_mask(nx, ny, x0, y0, y1, w=2):
    m = np.zeros((ny, nx), np.uint8)
    m[y0:y1, x0:x0 + w] = 1
    return m


@pytest.mark.parametrize("collision", [0, 1])
def test_conservation_around_obstacles(orc, collision):
    nx, ny = 56, 44
    p = Params(nx=nx, ny=ny, flow=1, eps=0.05, fold=6, body=(3e-6, 1e-6, 0.0),
               collision=collision)
    o = O.Oracle(p)
    mask = baffle_mask(nx, ny, 8, 10, 30) | baffle_mask(nx, ny, 40, 25, 41, 3)
    mask[2:5, 20:24] = 1
    o.init_seed(25.0, 20.0, 0.0, 6.0, 0.4, 0.01, 7)
    o.set_solid(mask)
    d0 = o.diag(25, 20)
    o.step(200)
    d1 = o.diag(25, 20)
    assert d1["solid_volume"] > d0["solid_volume"] * 1.02  # the crystal grew
    assert abs(d1["solute_total"] / d0["solute_total"] - 1) < 1e-12
    assert abs(d1["mass_total"] / d0["mass_total"] - 1) < 1e-12
    f = o.fields()
    assert np.abs(f["ux"]).max() > 1e-5  # the flow went round the obstacles


def test_mirror_symmetry_with_an_obstacle(orc):
    # obstacle and seed symmetric about y = (ny - 1)/2, flow along x
    nx, ny = 48, 40
    p = Params(nx=nx, ny=ny, flow=1, eps=0.03, fold=4, bc=(INLET_OUTLET, PERIODIC, PERIODIC),
               u_inlet=0.01, u0_inlet=0.3)
    o = O.Oracle(p)
    mask = np.zeros((ny, nx), np.uint8)
    mask[12:28, 10:12] = 1
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    phi = np.tanh((6.0 - np.hypot(x - 30.0, y - (ny - 1) / 2)) / (math.sqrt(2) * 2.0))
    o.init_fields(phi, np.full_like(phi, 0.3), None, np.full_like(phi, 0.01), None)
    o.set_solid(mask)
    o.step(150)
    f = o.fields()
    for k in ("phi", "U", "rho", "ux"):
        assert np.abs(f[k] - f[k][::-1]).max() < 1e-12, k
    assert np.abs(f["uy"] + f["uy"][::-1]).max() < 1e-12
    assert np.abs(f["uy"]).max() > 1e-5  # the flow was deflected


def test_liquid_at_rest_is_a_fixed_point_with_obstacles(orc):
    p = Params(nx=32, ny=24, flow=1, eps=0.05, fold=4)
    o = O.Oracle(p)
    n = p.nodes
    o.init_fields(-np.ones(n), np.full(n, 0.2))
    o.set_solid(baffle_mask(32, 24, 12, 5, 19))
    s0 = o.fields()
    o.step(50)
    s1 = o.fields()
    for k in ("phi", "U", "rho", "ux", "uy"):
        assert np.abs(s1[k] - s0[k]).max() < 1e-14, k


def test_mask_rejections(orc):
    p = Params(nx=16, ny=12, flow=1, bc=(INLET_OUTLET, PERIODIC, PERIODIC), u_inlet=0.01)
    o = O.Oracle(p)
    m = np.zeros((12, 16), np.uint8)
    m[3, 0] = 1
    with pytest.raises(ValueError):
        o.set_solid(m)
    m[3, 0] = 0
    m[3, 15] = 1
    with pytest.raises(ValueError):
        o.set_solid(m)
    m[3, 15] = 0
    m[3, 7] = 1
    o.set_solid(m)


# ---- 3D ---------------------------------------------------------------------------
def test_3d_poiseuille_between_solid_planes(orc):
    tau, H, b = 0.5 + math.sqrt(3.0 / 16.0), 16, 1e-6
    nz = 24
    p = Params(dim=3, nx=4, ny=4, nz=nz, fold=0, flow=1, tau_f=tau, eps=0.0, lambda_=0.0,
               bc=(PERIODIC, PERIODIC, PERIODIC), body=(b, 0.0, 0.0))
    o = O.Oracle(p)
    mask = np.zeros((nz, 4, 4), np.uint8)
    mask[3] = mask[20] = 1
    o.set_solid(mask)
    n = p.nodes
    o.init_fields(-np.ones(n), np.zeros(n), np.ones(n), np.zeros(n), np.zeros(n), np.zeros(n))
    f0 = o.pops("f")
    o.step(25000, 4)
    nu = (tau - 0.5) / 3.0
    z = np.arange(H) + 0.5
    exact = b / (2 * nu) * z * (H - z)
    got = o.fields()["ux"][4:20, 0, 0]
    assert np.abs(got / exact - 1).max() < 1e-6, np.abs(got / exact - 1).max()
    assert np.array_equal(o.pops("f")[:, [3, 20]], f0[:, [3, 20]])


@pytest.mark.parametrize("flow,collision", [(0, 0), (1, 0), (1, 1)])
@pytest.mark.parametrize("axis", [1, 2])
def test_3d_solid_planes_reproduce_the_domain_walls(orc, flow, collision, axis):
    # A: walls normal to `axis` (1: y, 2: z), periodic otherwise.  B: periodic,
    # two more nodes along `axis`, the first and last planes solid.  A seed
    # touching the lower wall, so that the gradient next to it is exercised.
    dims = [14, 12, 10]
    kw = dict(dim=3, fold=0, flow=flow, eps=0.04, collision=collision,
              body=(2e-6, 0.0, 0.0) if flow else (0, 0, 0))
    bc_a = [PERIODIC, PERIODIC, PERIODIC]
    bc_a[axis] = WALL
    pa = Params(nx=dims[0], ny=dims[1], nz=dims[2], bc=tuple(bc_a), **kw)
    db = list(dims)
    db[axis] += 2
    pb = Params(nx=db[0], ny=db[1], nz=db[2], bc=(PERIODIC,) * 3, **kw)
    rng = np.random.default_rng(4)
    zz, yy, xx = np.mgrid[0:dims[2], 0:dims[1], 0:dims[0]].astype(float)
    centre = [6.3, 5.2, 4.1]
    centre[axis] = 2.2
    r = np.sqrt((xx - centre[0]) ** 2 + (yy - centre[1]) ** 2 + (zz - centre[2]) ** 2)
    phi = np.tanh((4.5 - r) / (math.sqrt(2) * 2.0)) + 0.01 * rng.uniform(-1, 1, r.shape)
    U = 0.35 + 0.01 * rng.uniform(-1, 1, r.shape)
    ux = 0.01 * np.sin(2 * np.pi * (yy if axis == 2 else zz) / 8.0) if flow else np.zeros_like(r)
    ax = 2 - axis  # the array axis of `axis` ([z, y, x] order)

    def pad(f, v):
        w = [(0, 0)] * 3
        w[ax] = (1, 1)
        return np.pad(f, w, constant_values=v)
    a = O.Oracle(pa)
    a.init_fields(phi, U, None, ux, None, None)
    b = O.Oracle(pb)
    b.init_fields(pad(phi, -1.0), pad(U, 0.35), None, pad(ux, 0.0), None, None)
    mask = np.zeros(pb.shape, np.uint8)
    sl = [slice(None)] * 3
    sl[ax] = 0
    mask[tuple(sl)] = 1
    sl[ax] = -1
    mask[tuple(sl)] = 1
    b.set_solid(mask)
    a.step(100, 4)
    b.step(100, 4)
    inner = [slice(None)] * 3
    inner[ax] = slice(1, -1)
    fa, fb = a.fields(), b.fields()
    for k in ("phi", "U", "rho", "ux", "uy", "uz"):
        assert np.abs(fa[k] - fb[k][tuple(inner)]).max() < 1e-13, k
    for k in "fgh":
        if k == "f" and not flow:
            continue
        assert np.abs(a.pops(k) - b.pops(k)[(slice(None),) + tuple(inner)]).max() < 1e-13, k


@pytest.mark.parametrize("collision", [0, 1])
def test_3d_conservation_around_obstacles(orc, collision):
    p = Params(dim=3, nx=24, ny=20, nz=16, fold=0, flow=1, eps=0.05, body=(3e-6, 1e-6, -1e-6),
               collision=collision)
    o = O.Oracle(p)
    mask = np.zeros(p.shape, np.uint8)
    mask[2:14, 4:16, 3:5] = 1     # a baffle
    mask[6:9, 1:3, 17:21] = 1     # a block touching nothing else
    o.init_seed(13.0, 10.0, 8.0, 6.0, 0.4, 0.01, 7)
    o.set_solid(mask)
    d0 = o.diag(13, 10, 8)
    o.step(120, 4)
    d1 = o.diag(13, 10, 8)
    assert d1["solid_volume"] > d0["solid_volume"] * 1.02
    assert abs(d1["solute_total"] / d0["solute_total"] - 1) < 1e-12
    assert abs(d1["mass_total"] / d0["mass_total"] - 1) < 1e-12
    assert np.abs(o.fields()["ux"]).max() > 1e-5


def test_3d_mirror_symmetry_and_rest_with_an_obstacle(orc):
    # obstacle and seed symmetric about y = (ny - 1)/2 and z = (nz - 1)/2,
    # flow along x from the inlet
    nx, ny, nz = 24, 14, 12
    p = Params(dim=3, nx=nx, ny=ny, nz=nz, fold=0, flow=1, eps=0.03,
               bc=(INLET_OUTLET, PERIODIC, PERIODIC), u_inlet=0.005, u0_inlet=0.3)
    o = O.Oracle(p)
    mask = np.zeros(p.shape, np.uint8)
    mask[3:9, 4:10, 6:8] = 1
    zz, yy, xx = np.mgrid[0:nz, 0:ny, 0:nx].astype(float)
    r = np.sqrt((xx - 15.0) ** 2 + (yy - (ny - 1) / 2) ** 2 + (zz - (nz - 1) / 2) ** 2)
    phi = np.tanh((3.5 - r) / (math.sqrt(2) * 2.0))
    o.init_fields(phi, np.full_like(phi, 0.3), None, np.full_like(phi, 0.005), None, None)
    o.set_solid(mask)
    o.step(80, 4)
    f = o.fields()
    for k in ("phi", "U", "rho", "ux"):
        assert np.abs(f[k] - f[k][:, ::-1, :]).max() < 1e-12, k
        assert np.abs(f[k] - f[k][::-1, :, :]).max() < 1e-12, k
    assert np.abs(f["uy"] + f["uy"][:, ::-1, :]).max() < 1e-12
    assert np.abs(f["uz"] + f["uz"][::-1, :, :]).max() < 1e-12
    assert np.abs(f["uy"]).max() > 1e-6  # the flow was deflected
    # liquid at rest around the obstacle is a fixed point
    q = Params(dim=3, nx=16, ny=12, nz=10, fold=0, flow=1, eps=0.05)
    r0 = O.Oracle(q)
    r0.init_fields(-np.ones(q.nodes), np.full(q.nodes, 0.2))
    m = np.zeros(q.shape, np.uint8)
    m[2:8, 3:9, 7:9] = 1
    r0.set_solid(m)
    s0 = r0.fields()
    r0.step(30, 4)
    s1 = r0.fields()
    for k in ("phi", "U", "rho", "ux", "uy", "uz"):
        assert np.abs(s1[k] - s0[k]).max() < 1e-14, k
    # the inlet and outlet columns must be fluid
    bad = np.zeros(p.shape, np.uint8)
    bad[5, 7, nx - 1] = 1
    with pytest.raises(ValueError):
        O.Oracle(p).set_solid(bad)
