"""Crystal-shape measurements of the paper's result sections, in FP64.

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module; the product package
never does.

What is measured (the paper's words restated):
  * Sec. 3.1.2 -- the crystal's average size: join the centres of opposite
    sides, take the crystal centre where those lines meet, number the sides,
    and measure each side's normal distance L_i from that centre;
    L_avg = mean of the L_i.
  * Eqs. 26-28 -- the growth rate is the slope of a straight-line fit of
    L(t), its reliability the coefficient of determination
    R^2 = 1 - A_res / A_tot with A_res = sum (L - L')^2 about the fitted line
    L' and A_tot = sum (L - mean L)^2.
  * Sec. 3.2 -- the quality parameter Q = max L_i / min L_i and the aspect
    ratio, the crystal's horizontal size over its vertical size.

Readings where the paper leaves the procedure to a figure:
  * the crystal boundary is the phi = 0 contour, located on every x- and
    y-edge of the grid whose end values change sign (phi > 0 at one end,
    not at the other) by linear interpolation; edges across a periodic
    wrap are not used;
  * side i lies on its supporting line, the line with normal n_i through
    the contour point farthest along n_i (support value h_i = max p . n_i);
    its ends are where that line meets the supporting lines of sides i - 1
    and i + 1 (the sides of the smallest polygon with these normals that
    holds the crystal), its centre the midpoint of the two ends;
  * sides i and i + k/2 are the opposite pairs (normals given in order
    around the crystal, n_{i+k/2} = -n_i); when the joining lines do not
    meet in one point the centre is their least-squares intersection;
  * L_i = h_i - c . n_i;
  * the horizontal (vertical) size is the extent of the contour points
    along x (y).
"""
from __future__ import annotations

import numpy as np


def contour_points(phi):
    """phi = 0 crossings of a 2D field phi[y, x]: an (N, 2) array of (x, y),
    first those on x-edges (row by row), then those on y-edges."""
    phi = np.asarray(phi, dtype=np.float64)
    pos = phi > 0.0
    # x-edges (x, y) - (x + 1, y)
    a, b = phi[:, :-1], phi[:, 1:]
    yy, xx = np.nonzero(pos[:, :-1] != pos[:, 1:])
    fa, fb = a[yy, xx], b[yy, xx]
    px = np.stack([xx + fa / (fa - fb), yy.astype(np.float64)], axis=1)
    # y-edges (x, y) - (x, y + 1)
    a, b = phi[:-1, :], phi[1:, :]
    yy, xx = np.nonzero(pos[:-1, :] != pos[1:, :])
    fa, fb = a[yy, xx], b[yy, xx]
    py = np.stack([xx.astype(np.float64), yy + fa / (fa - fb)], axis=1)
    return np.concatenate([px, py], axis=0)


def _least_squares_point(points, dirs):
    """The point closest, in the sum of squared distances, to the lines
    through points[p] along unit directions dirs[p]."""
    A = np.zeros((2, 2))
    r = np.zeros(2)
    for a, u in zip(points, dirs):
        M = np.eye(2) - np.outer(u, u)
        A += M
        r += M @ a
    return np.linalg.solve(A, r)


def _meet(n1, h1, n2, h2):
    """Intersection of the lines p . n1 = h1 and p . n2 = h2."""
    return np.linalg.solve(np.array([n1, n2]), np.array([h1, h2]))


def facets(phi, normals):
    """Shape of the crystal phi > 0 with k facets of outward unit normals
    normals[k, 2] (k even, in order around the crystal, opposite facets k/2
    apart).  Returns a dict:
    points (contour point count), support [k], side_centre [k, 2],
    centre [2], L [k], L_avg, Q, width, height, aspect.  With no contour,
    every value but points is NaN."""
    n = np.asarray(normals, dtype=np.float64).reshape(-1, 2)
    k = n.shape[0]
    assert k % 2 == 0 and np.allclose(n[k // 2:], -n[:k // 2], atol=1e-9)
    nan = float("nan")
    pts = contour_points(phi)
    out = dict(points=int(pts.shape[0]))
    if pts.shape[0] == 0:
        out.update(support=np.full(k, nan), side_centre=np.full((k, 2), nan),
                   centre=np.full(2, nan), L=np.full(k, nan), L_avg=nan, Q=nan,
                   width=nan, height=nan, aspect=nan)
        return out
    # the supporting line of every side, its two ends and its centre
    support = (pts @ n.T).max(axis=0)
    ends = [_meet(n[i], support[i], n[(i + 1) % k], support[(i + 1) % k]) for i in range(k)]
    side_centre = np.array([0.5 * (ends[i - 1] + ends[i]) for i in range(k)])
    # lines joining the centres of opposite sides; the crystal centre
    anchors, dirs = [], []
    for i in range(k // 2):
        d = side_centre[i + k // 2] - side_centre[i]
        ln = np.hypot(d[0], d[1])
        if ln > 0.0:
            anchors.append(side_centre[i])
            dirs.append(d / ln)
    if len(dirs) >= 2 and abs(np.linalg.det(sum(np.eye(2) - np.outer(u, u) for u in dirs))) > 1e-12:
        centre = _least_squares_point(anchors, dirs)
    else:
        centre = side_centre.mean(axis=0)
    # normal distance of every side from the centre
    L = support - n @ centre
    width = pts[:, 0].max() - pts[:, 0].min()
    height = pts[:, 1].max() - pts[:, 1].min()
    out.update(support=support, side_centre=side_centre, centre=centre, L=L,
               L_avg=float(L.mean()), Q=float(L.max() / L.min()), width=float(width),
               height=float(height), aspect=float(width / height) if height > 0 else nan)
    return out


def growth_fit(t, L):
    """Straight-line fit L'(t) = a + b t of a size history (Eqs. 26-28):
    returns (b, a, R^2).  R^2 is NaN when every L is the same (A_tot = 0)."""
    t = np.asarray(t, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)
    assert t.size == L.size and t.size >= 2
    tm, Lm = t.mean(), L.mean()
    stt = ((t - tm) ** 2).sum()
    assert stt > 0.0
    b = ((t - tm) * (L - Lm)).sum() / stt
    a = Lm - b * tm
    fit = a + b * t
    A_res = ((L - fit) ** 2).sum()  # Eq. 27
    A_tot = ((L - Lm) ** 2).sum()  # Eq. 28
    r2 = 1.0 - A_res / A_tot if A_tot > 0.0 else float("nan")  # Eq. 26
    return float(b), float(a), float(r2)
