"""The workloads: seeded polygon sets and point streams for each configuration.

tiny      1,000 Voronoi blocks of jittered-lattice seeds in [0,1]^2 degrees,
          median 20 vertices, 1e6 uniform lattice points + 1% outside.
state     200,000 blocks over a 5x5 degree box (lon -75..-70, lat 40..45),
          seeds from the 64-Gaussian point mixture plus 10% uniform, 3-level
          hierarchy (40 counties, ~5,000 tracts), lognormal vertex counts
          (median 12, sigma 1.1, clamp [4, 2000], three forced 2,000-vertex
          blocks), 2% of blocks with a hole filled by an island block;
          1e8 mixture points.
national  800,000 blocks in 50 disjoint regions of 3-10 degrees inside lon
          [-125,-65] x lat [24,50]; each region a state-style hierarchy.
batched   8 sets of 10k-200k blocks (log-spaced), vertex medians 6..40, and
          4,096 queries with lognormal sizes in [100, 1e6] (mean ~5e4).
"""
from __future__ import annotations

import numpy as np

from .partition import (UNITS_PER_DEG, attach_hierarchy, lognormal_targets, merge_sets,
                        voronoi_partition)
from .points import Mixture, lattice_to_degrees, uniform_lattice

SEEDS = {"tiny": 1, "state": 2, "national": 3, "batched": 4, "serve": 5}


def _rng(seed, stream):
    return np.random.Generator(np.random.PCG64([seed, stream]))


def tiny_set(seed=SEEDS["tiny"], n_blocks=1000, deg=1.0, origin=(0.0, 0.0),
             vert_median=20, holes=0.0, hierarchy=True):
    """Voronoi partition of jittered-lattice seeds in a deg x deg box."""
    rng = _rng(seed, 0)
    X0 = int(round(origin[0] * UNITS_PER_DEG))
    Y0 = int(round(origin[1] * UNITS_PER_DEG))
    side = int(round(deg * UNITS_PER_DEG))
    box = (X0, Y0, X0 + side, Y0 + side)
    g = int(np.ceil(np.sqrt(n_blocks)))
    cell = side / g
    ii, jj = np.meshgrid(np.arange(g), np.arange(g), indexing="ij")
    sx = X0 + (ii.ravel() + 0.5 + rng.uniform(-0.4, 0.4, g * g)) * cell
    sy = Y0 + (jj.ravel() + 0.5 + rng.uniform(-0.4, 0.4, g * g)) * cell
    pick = np.sort(rng.choice(g * g, n_blocks, replace=False))
    seeds = np.c_[sx[pick], sy[pick]]
    targets = lognormal_targets(rng, n_blocks, vert_median, 0.5, 4, 400)
    hole_mask = rng.random(n_blocks) < holes if holes > 0 else None
    pset, hosts = voronoi_partition(seeds, box, rng, targets, hole_mask=hole_mask)
    if hierarchy:
        attach_hierarchy(pset, seeds, hosts, rng, n_tracts=max(1, n_blocks // 20),
                         n_counties=max(1, n_blocks // 200))
    pset.meta["config"] = "tiny"
    return pset


def tiny_points(pset, n=1_000_000, seed=SEEDS["tiny"], outside_frac=0.01):
    rng = _rng(seed, 1)
    qx, qy = uniform_lattice(pset.box, n, rng, outside_frac=outside_frac)
    return lattice_to_degrees(qx), lattice_to_degrees(qy)


def _state_like(rng, box, n_blocks, mixture, vert_median=12, vert_sigma=1.1,
                vert_max=2000, n_forced=3, hole_frac=0.02, n_tracts=5000, n_counties=40):
    n_seeds = int(round(n_blocks / (1.0 + hole_frac)))
    seeds = mixture.sample_units(n_seeds, rng, inside_only=True)
    targets = lognormal_targets(rng, n_seeds, vert_median, vert_sigma, 4, vert_max)
    forced = rng.choice(n_seeds, n_forced, replace=False) if n_forced else None
    if forced is not None:
        targets[forced] = vert_max
    hole_mask = rng.random(n_seeds) < hole_frac
    pset, hosts = voronoi_partition(seeds, box, rng, targets, hole_mask=hole_mask,
                                    forced=forced)
    attach_hierarchy(pset, seeds, hosts, rng, n_tracts=n_tracts, n_counties=n_counties)
    return pset


STATE_BOX_DEG = (-75.0, 40.0, -70.0, 45.0)


def _box_units(b):
    return tuple(int(round(v * UNITS_PER_DEG)) for v in b)


def state_mixture(seed=SEEDS["state"], box_deg=STATE_BOX_DEG):
    return Mixture(_box_units(box_deg), _rng(seed, 10))


def state_set(seed=SEEDS["state"], n_blocks=200_000, box_deg=STATE_BOX_DEG, **kw):
    box = _box_units(box_deg)
    mix = state_mixture(seed, box_deg)
    pset = _state_like(_rng(seed, 0), box, n_blocks, mix, **kw)
    pset.meta["config"] = "state"
    return pset


def state_points(n=100_000_000, seed=SEEDS["state"], box_deg=STATE_BOX_DEG, stream=1):
    mix = state_mixture(seed, box_deg)
    return mix.sample_degrees(n, _rng(seed, stream))


def national_regions(seed=SEEDS["national"], n_regions=50):
    """50 disjoint boxes with sides in 3-10 degrees inside lon [-125,-65] x
    lat [24,50]: sides drawn skewed towards 3 degrees (the window holds only
    ~1,560 square degrees); a box that cannot be placed shrinks (not below
    3 degrees) until it fits."""
    rng = _rng(seed, 20)
    boxes = []

    def free(b):
        return all(b[2] <= c[0] or c[2] <= b[0] or b[3] <= c[1] or c[3] <= b[1] for c in boxes)

    while len(boxes) < n_regions:
        w = 3.0 + 7.0 * rng.random() ** 3
        h = 3.0 + 7.0 * rng.random() ** 3
        placed = False
        while not placed:
            for _ in range(400):
                x0 = rng.uniform(-125, -65 - w)
                y0 = rng.uniform(24, 50 - h)
                b = (x0, y0, x0 + w, y0 + h)
                if free(b):
                    boxes.append(b)
                    placed = True
                    break
            if not placed:
                if w <= 3.0 and h <= 3.0:
                    boxes = []  # start over with the rng's next values
                    break
                w, h = max(3.0, 0.9 * w), max(3.0, 0.9 * h)
    return [tuple(round(v, 4) for v in b) for b in boxes]


def _region_share(boxes, total):
    area = np.array([(b[2] - b[0]) * (b[3] - b[1]) for b in boxes])
    share = np.floor(total * area / area.sum()).astype(np.int64)
    share[np.argmax(area)] += total - share.sum()
    return share


def national_set(seed=SEEDS["national"], n_blocks=800_000, n_regions=50):
    boxes = national_regions(seed, n_regions)
    share = _region_share(boxes, n_blocks)
    parts = []
    for r, b in enumerate(boxes):
        mix = Mixture(_box_units(b), _rng(seed, 100 + r))
        nb = int(share[r])
        parts.append(_state_like(_rng(seed, 1000 + r), _box_units(b), nb, mix,
                                 n_tracts=max(4, nb // 40), n_counties=max(2, nb // 5000),
                                 n_forced=1))
    box = (min(p.box[0] for p in parts), min(p.box[1] for p in parts),
           max(p.box[2] for p in parts), max(p.box[3] for p in parts))
    pset = merge_sets(parts, box)
    pset.meta["config"] = "national"
    return pset


class NationalPoints:
    """Mixture points over the 50 regions, drawn chunk by chunk (regions are
    picked in proportion to their block counts)."""

    def __init__(self, seed=SEEDS["national"], n_regions=50):
        boxes = national_regions(seed, n_regions)
        self.mixes = [Mixture(_box_units(b), _rng(seed, 100 + r)) for r, b in enumerate(boxes)]
        area = np.array([(b[2] - b[0]) * (b[3] - b[1]) for b in boxes])
        self.p = area / area.sum()
        self.seed = seed

    def chunk(self, i, n):
        """Chunk i of n points: an i.i.d. region label per point; each
        region's points are drawn i.i.d. from its mixture and placed at that
        region's positions (so the stream is in random spatial order)."""
        rng = _rng(self.seed, 5000 + i)
        cdf = np.cumsum(self.p)
        cdf[-1] = 1.0
        reg = np.minimum(np.searchsorted(cdf, rng.random(n), side="right"),
                         len(self.mixes) - 1).astype(np.uint8)
        order = np.argsort(reg, kind="stable")
        counts = np.bincount(reg, minlength=len(self.mixes))
        lon = np.empty(n, np.float64)
        lat = np.empty(n, np.float64)
        at = 0
        for r, c in enumerate(counts):
            if not c:
                continue
            pts = self.mixes[r].sample_units_iid(int(c), rng)
            pos = order[at:at + c]
            lon[pos] = pts[:, 0] / UNITS_PER_DEG
            lat[pos] = pts[:, 1] / UNITS_PER_DEG
            at += c
        return lon, lat


def batched_set(s, seed=SEEDS["batched"], n_sets=8, lo=10_000, hi=200_000, scale=1.0):
    """Set s of the batched workload: log-spaced block counts and vertex
    medians 6..40 over the n_sets sets."""
    sizes = np.rint(np.geomspace(lo, hi, n_sets) * scale).astype(np.int64)
    medians = np.rint(np.geomspace(6, 40, n_sets)).astype(np.int64)
    deg = float(np.sqrt(sizes[s] / 8000.0))  # ~8,000 blocks per square degree
    box_deg = (-100.0 + 12 * s, 30.0, -100.0 + 12 * s + deg, 30.0 + deg)
    mix = Mixture(_box_units(box_deg), _rng(seed, 300 + s))
    pset = _state_like(_rng(seed, 400 + s), _box_units(box_deg), int(sizes[s]), mix,
                       vert_median=int(medians[s]), n_tracts=max(4, int(sizes[s]) // 40),
                       n_counties=max(2, int(sizes[s]) // 5000), n_forced=1)
    pset.meta.update(config="batched", set=s, mixture=mix)
    return pset


def batched_sets(seed=SEEDS["batched"], n_sets=8, lo=10_000, hi=200_000, scale=1.0):
    """8 sets with log-spaced block counts and vertex medians 6..40."""
    return [batched_set(s, seed, n_sets, lo, hi, scale) for s in range(n_sets)]


def batched_query_sizes(seed=SEEDS["batched"], n_queries=4096, lo=100, hi=1_000_000,
                        median=10_000, mean=50_000):
    """Lognormal sizes truncated to [lo, hi]; sigma solved for the mean."""
    rng = _rng(seed, 500)
    z = rng.standard_normal(n_queries * 4)

    def trunc_mean(sig):
        s = np.exp(np.log(median) + sig * z)
        s = s[(s >= lo) & (s <= hi)]
        return s.mean()

    a, b = 0.1, 4.0
    for _ in range(60):
        m = 0.5 * (a + b)
        if trunc_mean(m) < mean:
            a = m
        else:
            b = m
    sig = 0.5 * (a + b)
    s = np.exp(np.log(median) + sig * rng.standard_normal(n_queries * 4))
    s = s[(s >= lo) & (s <= hi)][:n_queries]
    return np.rint(s).astype(np.int64), sig


def national_points_chunk(i, n, seed=SEEDS["national"]):
    """Chunk i (lon, lat) of the national point stream (picklable helper for
    process pools)."""
    return NationalPoints(seed).chunk(i, n)
