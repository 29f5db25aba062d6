"""Pins that tie the CPU oracle to facts outside itself.

Each check takes an oracle module (the real one, or a copy with a planted
mistake) and raises AssertionError when the oracle disagrees with:
  * exact rational arithmetic for Q (Python `fractions`),
  * the textbook even-odd test evaluated at a rational perturbation
    p' = p + (1/(4W), 1/(16 W^2)) of every lattice point (no vertex lies on
    the ray from p', and no edge passes between p and p'),
  * closed forms: an axis-aligned rectangle owns exactly [x0,x1) x [y0,y1),
    a grid of unit squares owns each lattice point of its extent once,
  * the half-plane form of a convex polygon at p',
  * brute force (O0) against the hierarchical join (O1).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from synth.partition import PolygonSet


def poly_set(rings_per_poly, parents=None):
    """PolygonSet from python lists: rings_per_poly[p] = [ring, ...], ring =
    [(x, y), ...]."""
    vx, vy, ring_off, pro = [], [], [0], [0]
    for rings in rings_per_poly:
        for ring in rings:
            for x, y in ring:
                vx.append(x)
                vy.append(y)
            ring_off.append(len(vx))
        pro.append(len(ring_off) - 1)
    return PolygonSet(np.array(vx, np.int32), np.array(vy, np.int32),
                      np.array(ring_off, np.int64), np.array(pro, np.int64),
                      parents=parents or [])


# ---------------------------------------------------------------- Q pins
def exact_q(v: float):
    """Nearest integer to v*10^7 (ties to even) with exact rationals."""
    if not math.isfinite(v):
        return None
    q = round(Fraction(v) * 10**7)  # Fraction rounding is half-to-even
    return q if abs(q) <= 2**31 - 1 else None


def q_cases(rng):
    ks = np.concatenate([
        rng.integers(-1_800_000_000, 1_800_000_001, 20000),
        [0, 1, -1, 2**31 - 1, -(2**31 - 1), 1_800_000_000, -1_800_000_000, 900_000_000],
    ])
    vals = [float(k) / 1e7 for k in ks] + [float(k) * 1e-7 for k in ks[:5000]]
    # ties: v = odd / 256 has v * 1e7 = odd * 39062.5 exactly
    vals += [o / 256.0 for o in range(-4001, 4002, 2)]
    # neighbours of ties and of the range limits
    for base in [0.00390625, 0.01171875, (2**31 - 1) / 1e7, 2**31 / 1e7, -(2**31) / 1e7,
                 214.74836475, -214.74836475, 214.74836465]:
        vals += [base, np.nextafter(base, np.inf), np.nextafter(base, -np.inf)]
    vals += [0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 1e-300, 4.9e-8, 5e-8,
             5.000000000000001e-8, 1.5e-7, 2.5e-7, 1e300, -1e300, float("inf"),
             float("-inf"), float("nan"), 2.0**52, 2.0**53, 180.0, -180.0, 90.0, -90.0]
    # random doubles across magnitudes
    vals += list(rng.uniform(-200, 200, 20000))
    vals += list(rng.uniform(-1, 1, 5000) * 10.0 ** rng.integers(-12, 3, 5000))
    return np.array(vals, np.float64)


def check_quantize(orc, rng):
    v = q_cases(rng)
    q, ok = orc.quantize(v)
    for i, x in enumerate(v):
        e = exact_q(float(x))
        if e is None:
            assert not ok[i], (x, q[i])
        else:
            assert ok[i] and int(q[i]) == e, (repr(float(x)), int(q[i]), e)


# ------------------------------------------------- crossing-rule pins
def textbook_even_odd(rings, px, py, W):
    """Classic crossing count at p' = (px + d, py + e), d = 1/(4W),
    e = 1/(16 W^2), in exact rationals."""
    X = Fraction(px) + Fraction(1, 4 * W)
    Y = Fraction(py) + Fraction(1, 16 * W * W)
    c = 0
    for ring in rings:
        m = len(ring)
        for i in range(m):
            ax, ay = ring[i]
            bx, by = ring[(i + 1) % m]
            if (ay > Y) != (by > Y):
                xi = ax + (bx - ax) * (Y - ay) / (by - ay)
                if xi > X:
                    c ^= 1
    return c


def random_rings(rng, span, max_vert=8, second_ring_p=0.4):
    rings = []
    nr = 2 if rng.random() < second_ring_p else 1
    for _ in range(nr):
        m = int(rng.integers(3, max_vert + 1))
        ring = [(int(rng.integers(0, span + 1)), int(rng.integers(0, span + 1))) for _ in range(m)]
        if rng.random() < 0.3:  # collinear run / horizontal edge
            x, y = ring[0]
            ring.insert(1, (min(span, x + 1), y))
            ring.insert(2, (min(span, x + 2), y))
        rings.append(ring)
    return rings


def check_perturbation(orc, rng, n_poly=150, span=6):
    W = 4 * (span + 4)
    for _ in range(n_poly):
        rings = random_rings(rng, span)
        ps = poly_set([rings])
        for px in range(-1, span + 2):
            for py in range(-1, span + 2):
                want = textbook_even_odd(rings, px, py, W)
                got = orc.inside(ps, 0, px, py)
                assert got == want, (rings, px, py, got, want)


def check_fans(orc):
    """Polygons meeting at one vertex and along shared edges: every lattice
    point of the covered square has exactly one owner."""
    c = (5, 5)
    ring_pts = [(0, 0), (5, 0), (10, 0), (10, 5), (10, 10), (5, 10), (0, 10), (0, 5)]
    polys = []
    for i in range(len(ring_pts)):
        a, b = ring_pts[i], ring_pts[(i + 1) % len(ring_pts)]
        polys.append([[c, a, b]])
    ps = poly_set(polys)
    qx, qy = np.meshgrid(np.arange(-2, 13), np.arange(-2, 13), indexing="ij")
    qx, qy = qx.ravel(), qy.ravel()
    cnt = orc.count_owners_q(ps, qx, qy)
    inner = (qx >= 0) & (qx < 10) & (qy >= 0) & (qy < 10)
    assert (cnt[inner] == 1).all() and (cnt[~inner] == 0).all()


def check_rectangles(orc, rng, n=40):
    for _ in range(n):
        x0, x1 = sorted(rng.choice(np.arange(-20, 21), 2, replace=False))
        y0, y1 = sorted(rng.choice(np.arange(-20, 21), 2, replace=False))
        ring = [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]
        if rng.random() < 0.5 and x1 - x0 > 1:  # extra collinear vertex on the bottom edge
            ring.insert(1, (int(rng.integers(x0 + 1, x1)), y0))
        if rng.random() < 0.5:
            ring = ring[::-1]
        k = int(rng.integers(0, len(ring)))
        ring = ring[k:] + ring[:k]
        ps = poly_set([[ring]])
        X, Y = np.meshgrid(np.arange(-22, 23), np.arange(-22, 23), indexing="ij")
        X, Y = X.ravel(), Y.ravel()
        got = orc.count_owners_q(ps, X, Y)
        want = ((X >= x0) & (X < x1) & (Y >= y0) & (Y < y1)).astype(np.int32)
        assert (got == want).all(), (ring,)


def check_unit_grid(orc, g=5):
    polys = [[[(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]] for i in range(g) for j in range(g)]
    ps = poly_set(polys)
    X, Y = np.meshgrid(np.arange(-1, g + 2), np.arange(-1, g + 2), indexing="ij")
    X, Y = X.ravel(), Y.ravel()
    got = orc.join_bruteforce_q(ps, X, Y)
    inside = (X >= 0) & (X < g) & (Y >= 0) & (Y < g)
    want = np.where(inside, X * g + Y, -1)
    assert (got == want).all()


def check_convex(orc, rng, n=60):
    """Convex polygon: inside(p) iff p' lies strictly left of every CCW edge."""
    for _ in range(n):
        pts = rng.integers(0, 12, (12, 2))
        hull = convex_hull([tuple(map(int, p)) for p in pts])
        if len(hull) < 3:
            continue
        ps = poly_set([[hull]])
        W = 4 * 16
        d, e = Fraction(1, 4 * W), Fraction(1, 16 * W * W)
        for px in range(-1, 13):
            for py in range(-1, 13):
                X, Y = px + d, py + e
                inside = all(
                    (bx - ax) * (Y - ay) - (by - ay) * (X - ax) > 0
                    for (ax, ay), (bx, by) in zip(hull, hull[1:] + hull[:1]))
                assert orc.inside(ps, 0, px, py) == int(inside), (hull, px, py)


def convex_hull(points):
    pts = sorted(set(points))
    if len(pts) <= 2:
        return pts

    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])

    lower, upper = [], []
    for p in pts:
        while len(lower) >= 2 and cross(lower[-2], lower[-1], p) <= 0:
            lower.pop()
        lower.append(p)
    for p in reversed(pts):
        while len(upper) >= 2 and cross(upper[-2], upper[-1], p) <= 0:
            upper.pop()
        upper.append(p)
    return lower[:-1] + upper[:-1]


def check_o0_o1(orc, pset, lon, lat):
    a = orc.join_bruteforce(pset, lon, lat)
    b = orc.join_hier(pset, lon, lat)
    c = orc.join_hier(pset, lon, lat, flat=True)
    assert (a == b).all(), int((a != b).sum())
    assert (a == c).all(), int((a != c).sum())


def check_partition(orc, pset, n, rng):
    """Every lattice point of the tiled box has one owner; points on the
    right/top border and outside have none."""
    X0, Y0, X1, Y1 = pset.box
    qx = rng.integers(X0, X1, n)
    qy = rng.integers(Y0, Y1, n)
    cnt = orc.count_owners_q(pset, qx, qy)
    assert (cnt == 1).all(), np.bincount(cnt)
    # vertices themselves (on shared edges and corners) also have one owner
    inner = (pset.vx < X1) & (pset.vy < Y1)
    vi = rng.choice(np.nonzero(inner)[0], min(n, int(inner.sum())), replace=False)
    cnt = orc.count_owners_q(pset, pset.vx[vi], pset.vy[vi])
    assert (cnt == 1).all(), np.bincount(cnt)
    bx = np.concatenate([np.full(200, X1), rng.integers(X0, X1 + 1, 200), np.full(50, X0 - 1)])
    by = np.concatenate([rng.integers(Y0, Y1 + 1, 200), np.full(200, Y1), rng.integers(Y0, Y1, 50)])
    cnt = orc.count_owners_q(pset, bx, by)
    assert (cnt == 0).all()
