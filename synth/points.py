"""Seeded synthetic query points (stand-ins for the paper's mobile-device
locations, Sec. V), as float64 longitude/latitude in degrees.

Nothing here classifies a point: these are plain random draws.
"""
from __future__ import annotations

import numpy as np

from .partition import UNITS_PER_DEG


def lattice_to_degrees(q) -> np.ndarray:
    """The double nearest q * 1e-7 for integer lattice coordinates q."""
    return np.asarray(q, np.int64).astype(np.float64) / UNITS_PER_DEG


def uniform_lattice(box, n, rng, outside_frac=0.01, margin=500_000):
    """n lattice points: uniform in [X0,X1) x [Y0,Y1), plus `outside_frac`
    of them uniform in the surrounding margin ring (outside the box)."""
    X0, Y0, X1, Y1 = box
    n_out = int(round(n * outside_frac))
    n_in = n - n_out
    qx = rng.integers(X0, X1, n_in, dtype=np.int64)
    qy = rng.integers(Y0, Y1, n_in, dtype=np.int64)
    ox = np.empty(0, np.int64)
    oy = np.empty(0, np.int64)
    while len(ox) < n_out:
        m = 2 * (n_out - len(ox)) + 16
        cx = rng.integers(X0 - margin, X1 + margin, m, dtype=np.int64)
        cy = rng.integers(Y0 - margin, Y1 + margin, m, dtype=np.int64)
        out = (cx < X0) | (cx >= X1) | (cy < Y0) | (cy >= Y1)
        ox = np.concatenate([ox, cx[out]])
        oy = np.concatenate([oy, cy[out]])
    qx = np.concatenate([qx, ox[:n_out]])
    qy = np.concatenate([qy, oy[:n_out]])
    perm = rng.permutation(n)
    return qx[perm], qy[perm]


def degenerate_lattice(pset, n, rng):
    """Lattice points placed on polygon vertices, on lattice points of edges
    and one unit around vertices: the cases the tie rule has to settle."""
    V = pset.n_vert
    k = n // 3
    vi = rng.integers(0, V, k)
    px = [pset.vx[vi].astype(np.int64)]
    py = [pset.vy[vi].astype(np.int64)]
    # lattice points on edges a -> b (next vertex of the same ring)
    r_of = np.searchsorted(pset.ring_off, np.arange(V), side="right") - 1
    nxt = np.arange(V) + 1
    last = pset.ring_off[1:] - 1
    nxt[last] = pset.ring_off[:-1]
    ei = rng.integers(0, V, k)
    ax, ay = pset.vx[ei].astype(np.int64), pset.vy[ei].astype(np.int64)
    bx, by = pset.vx[nxt[ei]].astype(np.int64), pset.vy[nxt[ei]].astype(np.int64)
    g = np.gcd(np.abs(bx - ax), np.abs(by - ay))
    g = np.maximum(g, 1)
    t = (rng.random(k) * (g + 1)).astype(np.int64)
    t = np.minimum(t, g)
    px.append(ax + (bx - ax) // g * t)
    py.append(ay + (by - ay) // g * t)
    # one unit around vertices
    m = n - 2 * k
    wi = rng.integers(0, V, m)
    px.append(pset.vx[wi].astype(np.int64) + rng.integers(-1, 2, m))
    py.append(pset.vy[wi].astype(np.int64) + rng.integers(-1, 2, m))
    del r_of
    return np.concatenate(px), np.concatenate(py)


class Mixture:
    """64 Gaussian components (centres uniform in the box, sigma log-uniform
    in [0.02, 0.3] degrees, weights Dirichlet(1)) plus a uniform share."""

    def __init__(self, box, rng, n_comp=64, sigma_deg=(0.02, 0.3), uniform_frac=0.10):
        X0, Y0, X1, Y1 = box
        self.box = box
        self.centres = np.c_[rng.uniform(X0, X1, n_comp), rng.uniform(Y0, Y1, n_comp)]
        lo, hi = np.log(sigma_deg[0]), np.log(sigma_deg[1])
        self.sigma = np.exp(rng.uniform(lo, hi, n_comp)) * UNITS_PER_DEG
        self.weights = rng.dirichlet(np.ones(n_comp))
        self.uniform_frac = uniform_frac

    def sample_units(self, n, rng, inside_only=False):
        """n points in lattice units (float64, not rounded)."""
        X0, Y0, X1, Y1 = self.box
        n_uni = int(round(n * self.uniform_frac))
        n_mix = n - n_uni
        comp = rng.choice(len(self.weights), n_mix, p=self.weights)
        xy = rng.standard_normal((n_mix, 2))
        xy *= self.sigma[comp, None]
        xy += self.centres[comp]
        uni = np.c_[rng.uniform(X0, X1, n_uni), rng.uniform(Y0, Y1, n_uni)]
        pts = np.concatenate([xy, uni])
        if inside_only:
            def inner(p):
                return p[(p[:, 0] > X0 + 1) & (p[:, 0] < X1 - 1)
                         & (p[:, 1] > Y0 + 1) & (p[:, 1] < Y1 - 1)]
            pts = inner(pts)
            while len(pts) < n:
                extra = inner(self.sample_units(2 * (n - len(pts)) + 1024, rng))
                pts = np.concatenate([pts, extra])
            pts = pts[:n]
        return pts[rng.permutation(len(pts))]

    def sample_units_iid(self, n, rng):
        """n points in lattice units, each independently from the mixture
        (component 64 = the uniform share), so their order needs no shuffle."""
        X0, Y0, X1, Y1 = self.box
        k = len(self.weights)
        p = np.concatenate([self.weights * (1.0 - self.uniform_frac), [self.uniform_frac]])
        cdf = np.cumsum(p)
        cdf[-1] = 1.0
        comp = np.minimum(np.searchsorted(cdf, rng.random(n), side="right"), k)
        sig = np.concatenate([self.sigma, [0.0]])[comp]
        cx = np.concatenate([self.centres[:, 0], [0.0]])[comp]
        cy = np.concatenate([self.centres[:, 1], [0.0]])[comp]
        uni = comp == k
        x = np.where(uni, rng.uniform(X0, X1, n), rng.standard_normal(n) * sig + cx)
        y = np.where(uni, rng.uniform(Y0, Y1, n), rng.standard_normal(n) * sig + cy)
        return np.c_[x, y]

    def sample_degrees(self, n, rng, chunk=1 << 24):
        """n points as float64 lon/lat degrees, generated in chunks."""
        lon = np.empty(n, np.float64)
        lat = np.empty(n, np.float64)
        for a in range(0, n, chunk):
            b = min(n, a + chunk)
            p = self.sample_units(b - a, rng)
            lon[a:b] = p[:, 0] / UNITS_PER_DEG
            lat[a:b] = p[:, 1] / UNITS_PER_DEG
        return lon, lat
