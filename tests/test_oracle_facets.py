"""Pins of the oracle's crystal-shape measurements and polygon seed.

The expected values come from plane geometry, not from the oracle: the
polygon's sides, vertices and side midpoints are constructed here from its
facet lines, the fit from textbook identities of least squares.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import facets as F

W0 = 2.0


def normals(k, theta):
    a = theta + 2.0 * math.pi * np.arange(k) / k
    return np.stack([np.cos(a), np.sin(a)], axis=1)


def rhombus_normals(theta, acute=math.pi / 3):
    # long diagonal along theta: the sides make acute/2 with it, so their
    # normals sit at +-(pi/2 - acute/2) and pi -+ (pi/2 - acute/2)
    b = math.pi / 2 - acute / 2
    a = np.array([b, math.pi - b, math.pi + b, -b]) + theta
    return np.stack([np.cos(a), np.sin(a)], axis=1)


def polygon_phi(nx, ny, c, n, d):
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    s = np.full((ny, nx), -np.inf)
    for (ux, uy), di in zip(n, d):
        s = np.maximum(s, (x - c[0]) * ux + (y - c[1]) * uy - di)
    return np.tanh(-s / (math.sqrt(2.0) * W0))


def vertices(c, n, d):
    """Vertex between facets i and i+1 (facets in order around the polygon)."""
    k = len(d)
    out = []
    for i in range(k):
        j = (i + 1) % k
        A = np.array([n[i], n[j]])
        r = np.array([d[i] + n[i] @ c, d[j] + n[j] @ c])
        out.append(np.linalg.solve(A, r))
    return np.array(out)


def test_regular_hexagon():
    c = np.array([64.37, 60.81])
    n = normals(6, 0.13)
    d = np.full(6, 20.3)
    r = F.facets(polygon_phi(128, 128, c, n, d), n)
    assert np.abs(r["L"] - 20.3).max() < 0.02, r["L"]
    assert np.abs(r["centre"] - c).max() < 0.02
    assert abs(r["Q"] - 1.0) < 2e-3
    assert abs(r["L_avg"] - 20.3) < 0.02


def test_rhombus_aspect_and_sizes():
    c = np.array([70.5, 55.25])
    n = rhombus_normals(0.0)
    d = np.full(4, 15.0)
    r = F.facets(polygon_phi(160, 120, c, n, d), n)
    v = vertices(c, n, d)
    width = v[:, 0].max() - v[:, 0].min()
    height = v[:, 1].max() - v[:, 1].min()
    assert abs(width / height - math.sqrt(3.0)) < 1e-9  # the 60-degree rhombus itself
    assert abs(r["aspect"] - math.sqrt(3.0)) < 0.03, r["aspect"]
    # the 60-degree tips fall between grid lines: the last crossing can stop
    # 0.5 / tan(30 deg) = 0.87 lu short of a tip
    assert abs(r["width"] - width) < 0.9 and abs(r["height"] - height) < 0.9
    assert np.abs(r["L"] - 15.0).max() < 0.02
    assert np.abs(r["centre"] - c).max() < 0.02


def test_irregular_hexagon_centre_joins_opposite_side_midpoints():
    c0 = np.array([90.2, 84.7])
    n = normals(6, 0.21)
    d = np.array([20.0, 26.0, 18.0, 24.0, 22.0, 30.0])
    r = F.facets(polygon_phi(180, 170, c0, n, d), n)
    v = vertices(c0, n, d)
    mid = np.array([(v[i - 1] + v[i]) / 2.0 for i in range(6)])  # side i: vertices i-1, i
    # the three lines joining opposite midpoints, least-squares intersection
    A = np.zeros((2, 2))
    rhs = np.zeros(2)
    for i in range(3):
        u = mid[i + 3] - mid[i]
        u /= np.linalg.norm(u)
        M = np.eye(2) - np.outer(u, u)
        A += M
        rhs += M @ mid[i]
    centre = np.linalg.solve(A, rhs)
    assert np.abs(r["side_centre"] - mid).max() < 0.1, r["side_centre"] - mid
    assert np.abs(r["centre"] - centre).max() < 0.1
    L = d + n @ c0 - n @ centre
    assert np.abs(r["L"] - L).max() < 0.1
    # the construction matters: the plain centroid of the contour is elsewhere
    pts = F.contour_points(polygon_phi(180, 170, c0, n, d))
    assert np.abs(pts.mean(axis=0) - centre).max() > 0.5


def test_translation_moves_the_centre_only():
    n = normals(6, 0.3)
    d = np.array([14.0, 17.0, 15.0, 16.0, 13.0, 18.0])
    phi = polygon_phi(100, 90, np.array([45.3, 40.6]), n, d)
    big = np.full((110, 120), -1.0)
    big[7:97, 11:111] = phi
    a = F.facets(phi, n)
    b = F.facets(big, n)
    assert np.abs(b["centre"] - a["centre"] - np.array([11.0, 7.0])).max() < 1e-9
    assert np.abs(b["L"] - a["L"]).max() < 1e-9
    assert a["points"] == b["points"]


def test_contour_points_lie_on_straight_sides():
    # a half-plane phi = tanh((x0 - x) / (sqrt 2 W0)): the crossings of every
    # row sit at x0 up to the linear-interpolation error of tanh across one
    # lattice spacing, third order near its zero (3.5e-3 lu at W0 = 2)
    y, x = np.mgrid[0:20, 0:40].astype(np.float64)
    phi = np.tanh((17.3 - x) / (math.sqrt(2.0) * W0))
    p = F.contour_points(phi)
    assert p.shape[0] == 20
    assert np.abs(p[:, 0] - 17.3).max() < 5e-3
    assert np.array_equal(p[:, 1], np.arange(20.0))


def test_no_crystal():
    r = F.facets(np.full((30, 30), -1.0), normals(6, 0.0))
    assert r["points"] == 0 and np.isnan(r["L_avg"]) and np.isnan(r["Q"])


def test_growth_fit_of_a_line_is_exact():
    t = np.arange(12.0) * 3.0
    b, a, r2 = F.growth_fit(t, 2.5 + 0.07 * t)
    assert abs(b - 0.07) < 1e-14 and abs(a - 2.5) < 1e-13 and abs(r2 - 1.0) < 1e-14


def test_growth_fit_textbook_identities():
    rng = np.random.default_rng(7)
    t = np.sort(rng.uniform(0, 12, 13))
    L = 1.0 + 0.08 * t + rng.normal(0, 0.05, t.size)
    b, a, r2 = F.growth_fit(t, L)
    pb, pa = np.polyfit(t, L, 1)
    assert abs(b - pb) < 1e-12 and abs(a - pa) < 1e-12
    # simple regression with intercept: R^2 is the squared correlation
    assert abs(r2 - np.corrcoef(t, L)[0, 1] ** 2) < 1e-12
    # no trend: R^2 near 0 (the paper's slow sides show 0.1-0.2)
    L0 = 3.0 + rng.normal(0, 0.05, t.size)
    assert F.growth_fit(t, L0)[2] < 0.5
    assert np.isnan(F.growth_fit(t, np.full(t.size, 2.0))[2])


@pytest.fixture(scope="module")
def orc():
    oracle.build()
    return oracle


def test_oracle_polygon_seed_has_the_polygon_shape(orc):
    p = orc.Params(nx=128, ny=112, w0=W0)
    o = orc.Oracle(p)
    c = (63.6, 55.2)
    n = normals(6, 0.4)
    d = np.array([19.0, 22.0, 17.0, 21.0, 20.0, 23.0])
    o.init_polygon(c[0], c[1], n, d, 0.3, 0.0, 1)
    f = o.fields()
    assert np.abs(f["U"] - 0.3).max() < 1e-14 and np.abs(f["rho"] - 1.0).max() < 1e-14
    want = polygon_phi(128, 112, np.array(c), n, d)
    assert np.abs(f["phi"] - want).max() < 1e-13
    r = F.facets(f["phi"], n)
    v = vertices(np.array(c), n, d)
    assert np.abs(r["support"] - (d + n @ np.array(c))).max() < 0.02
    assert r["points"] > 0 and np.all(r["side_centre"][:, 0] > v[:, 0].min() - 1)
    o.close()


def test_oracle_polygon_seed_noise_is_the_round_seeds(orc):
    p = orc.Params(nx=40, ny=36, w0=W0)
    n = normals(4, 0.0)
    d = np.full(4, 9.0)
    out = {}
    for name, amp in (("a", 0.0), ("b", 0.01)):
        o = orc.Oracle(p)
        o.init_polygon(20.0, 18.0, n, d, 0.2, amp, 42)
        out["poly" + name] = o.fields()["phi"]
        o.init_seed(20.0, 18.0, 0.0, 9.0, 0.2, amp, 42)
        out["round" + name] = o.fields()["phi"]
        o.close()
    dp = out["polyb"] - out["polya"]
    dr = out["roundb"] - out["rounda"]
    assert np.abs(dp).max() > 5e-3
    assert np.abs(dp - dr).max() < 1e-15
