"""Seeded synthetic polygon partitions shaped like census block groups.

These stand in for the TIGER state/county/block-group shapefiles the paper
reads (Sec. II), which are not available here. Everything is deterministic
from a seed. The module contains no point-in-polygon arithmetic: it only
builds vertex rings and the region -> county -> tract -> block parent arrays.

Construction (all coordinates are int on the 1e-7 degree lattice):
  1. Voronoi diagram of the block seeds, clipped to the box by mirroring the
     seeds across the four box sides (the mirror bisectors are the box edges).
  2. Voronoi vertices are snapped once to the lattice and shared by index, so
     neighbouring blocks use identical coordinates.
  3. Every shared edge is subdivided once; the interior points are jittered
     perpendicular to the edge inside a thin double cone around it (half
     angle below 0.45 x the smallest adjacent vertex angle, amplitude below a
     fifth of the seed-to-edge distance), and both neighbours reuse the same
     points in opposite order. Box-boundary edges are subdivided without
     jitter so the blocks tile the box exactly.
  4. Optional holes: a star-shaped ring around a block's seed, well inside
     the block, becomes an inner ring of the host and the outer ring of a new
     island block, so the blocks still partition the box.
  5. Tracts and counties are unions of blocks by nearest tract / county seed,
     so parent boxes are unions of child boxes and no parent polygon exists.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

UNITS_PER_DEG = 10_000_000


@dataclass
class PolygonSet:
    vx: np.ndarray             # int32 [V]
    vy: np.ndarray             # int32 [V]
    ring_off: np.ndarray       # int64 [R+1]: ring r = vertices [ring_off[r], ring_off[r+1])
    poly_ring_off: np.ndarray  # int64 [P+1]: polygon p = rings [poly_ring_off[p], ...[p+1])
    parents: list = field(default_factory=list)  # parents[l][i] = level-(l+1) node of level-l node i
    box: tuple = (0, 0, 0, 0)  # (X0, Y0, X1, Y1): the blocks tile [X0,X1] x [Y0,Y1]
    meta: dict = field(default_factory=dict)

    @property
    def n_poly(self) -> int:
        return len(self.poly_ring_off) - 1

    @property
    def n_vert(self) -> int:
        return len(self.vx)

    def vertex_counts(self) -> np.ndarray:
        v = self.ring_off[self.poly_ring_off]
        return np.diff(v)


def _ring_next(ring_start: np.ndarray, ring_len: np.ndarray) -> np.ndarray:
    """Index of the cyclic successor of every flat ring element."""
    total = int(ring_len.sum())
    idx = np.arange(total, dtype=np.int64)
    rid = np.repeat(np.arange(len(ring_len)), ring_len)
    nxt = idx + 1
    last = ring_start + ring_len - 1
    nxt[last[ring_len > 0]] = ring_start[ring_len > 0]
    return nxt, rid


def _compact_rings(ids: np.ndarray, ring_len: np.ndarray):
    """Drop cyclically repeated consecutive vertex ids inside each ring."""
    start = np.concatenate([[0], np.cumsum(ring_len)[:-1]]).astype(np.int64)
    nxt, rid = _ring_next(start, ring_len)
    keep = ids != ids[nxt]
    # a ring whose vertices are all equal keeps nothing
    new_len = np.bincount(rid[keep], minlength=len(ring_len)).astype(np.int64)
    return ids[keep], new_len


def _orient_ccw(ids, ring_len, cx, cy):
    """Reverse rings with negative signed area (orientation is cosmetic)."""
    start = np.concatenate([[0], np.cumsum(ring_len)[:-1]]).astype(np.int64)
    nxt, rid = _ring_next(start, ring_len)
    x = cx[ids].astype(np.float64)
    y = cy[ids].astype(np.float64)
    cross = x * y[nxt] - x[nxt] * y
    area2 = np.bincount(rid, weights=cross, minlength=len(ring_len))
    flip = area2 < 0
    if flip.any():
        pos = np.arange(len(ids), dtype=np.int64) - start[rid]
        src = np.where(flip[rid], start[rid] + ring_len[rid] - 1 - pos, np.arange(len(ids)))
        ids = ids[src]
    return ids


def voronoi_partition(seeds, box, rng, targets, hole_mask=None, forced=None,
                      max_cone_deg=8.0):
    """Partition `box` into the Voronoi cells of `seeds` (float units).

    targets[i] is the wished vertex count of block i (reached by edge
    subdivision; the realized counts are reported in meta). hole_mask[i]
    gives block i a hole filled by a new island block (appended at the end).
    Returns (PolygonSet without parents, island_host array).
    """
    from scipy.spatial import Voronoi

    X0, Y0, X1, Y1 = (int(b) for b in box)
    seeds = np.asarray(seeds, np.float64)
    n = len(seeds)
    sx, sy = seeds[:, 0], seeds[:, 1]
    assert (sx > X0).all() and (sx < X1).all() and (sy > Y0).all() and (sy < Y1).all()
    mir = np.concatenate([
        seeds,
        np.c_[2 * X0 - sx, sy], np.c_[2 * X1 - sx, sy],
        np.c_[sx, 2 * Y0 - sy], np.c_[sx, 2 * Y1 - sy],
    ])
    c = np.array([(X0 + X1) / 2, (Y0 + Y1) / 2])
    scale = float(max(X1 - X0, Y1 - Y0))
    vor = Voronoi((mir - c) / scale)
    verts = vor.vertices * scale + c

    # region vertex lists of the original seeds, flattened
    regs = [vor.regions[vor.point_region[i]] for i in range(n)]
    ring_len = np.array([len(r) for r in regs], np.int64)
    flat = np.fromiter((v for r in regs for v in r), np.int64, count=int(ring_len.sum()))
    assert (flat >= 0).all(), "unbounded Voronoi region despite mirroring"

    # snap used vertices once to the lattice, onto the box edges when close
    used, inv = np.unique(flat, return_inverse=True)
    ux = np.rint(verts[used, 0])
    uy = np.rint(verts[used, 1])
    tol = 2.0
    ux[np.abs(verts[used, 0] - X0) <= tol] = X0
    ux[np.abs(verts[used, 0] - X1) <= tol] = X1
    uy[np.abs(verts[used, 1] - Y0) <= tol] = Y0
    uy[np.abs(verts[used, 1] - Y1) <= tol] = Y1
    ux = np.clip(ux, X0, X1).astype(np.int64)
    uy = np.clip(uy, Y0, Y1).astype(np.int64)
    # canonical vertex ids by snapped coordinate (merges vertices that snap together)
    key = (ux - X0) * (1 << 32) + (uy - Y0)
    ukey, canon = np.unique(key, return_inverse=True)
    cx = (ukey >> 32) + X0
    cy = (ukey & ((1 << 32) - 1)) + Y0
    ids = canon[inv]
    ids, ring_len = _compact_rings(ids, ring_len)
    ids = _orient_ccw(ids, ring_len, cx, cy)
    start = np.concatenate([[0], np.cumsum(ring_len)[:-1]]).astype(np.int64)
    nxt, rid = _ring_next(start, ring_len)

    # vertex angles (radians, in (0, pi)) at every ring position
    prv = np.empty_like(nxt)
    prv[nxt] = np.arange(len(nxt))
    wx, wy = cx[ids].astype(np.float64), cy[ids].astype(np.float64)
    ax_, ay_ = cx[ids[prv]] - wx, cy[ids[prv]] - wy
    bx_, by_ = cx[ids[nxt]] - wx, cy[ids[nxt]] - wy
    ang = np.arctan2(np.abs(ax_ * by_ - ay_ * bx_), ax_ * bx_ + ay_ * by_)

    # undirected edges
    u, v = ids, ids[nxt]
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    ekey = lo * (len(cx) + 1) + hi
    ekeys, einv = np.unique(ekey, return_inverse=True)
    n_edge = len(ekeys)
    ea = ekeys // (len(cx) + 1)
    eb = ekeys % (len(cx) + 1)
    owners = np.bincount(einv, minlength=n_edge)
    assert owners.max() <= 2, "an edge is shared by more than two blocks"
    fwd = u < v  # occurrence runs a->b along the canonical edge direction
    # owner seeds of each edge (second = -1 for box-boundary edges)
    own0 = np.full(n_edge, -1, np.int64)
    own1 = np.full(n_edge, -1, np.int64)
    _, first_occ = np.unique(einv, return_index=True)
    own0[:] = rid[first_occ]
    second = np.ones(len(einv), bool)
    second[first_occ] = False
    own1[einv[second]] = rid[second]
    boundary = owners == 1
    on_side = (((cx[ea] == X0) & (cx[eb] == X0)) | ((cx[ea] == X1) & (cx[eb] == X1))
               | ((cy[ea] == Y0) & (cy[eb] == Y0)) | ((cy[ea] == Y1) & (cy[eb] == Y1)))
    open_edges = int((boundary & ~on_side).sum())

    # cone half-angle at each edge end: 0.45 x smallest adjacent vertex angle
    ang_a = np.full(n_edge, np.pi)
    ang_b = np.full(n_edge, np.pi)
    at_u = ang           # angle at the occurrence's start vertex
    at_v = ang[nxt]      # angle at its end vertex
    np.minimum.at(ang_a, einv[fwd], at_u[fwd])
    np.minimum.at(ang_b, einv[fwd], at_v[fwd])
    np.minimum.at(ang_b, einv[~fwd], at_u[~fwd])
    np.minimum.at(ang_a, einv[~fwd], at_v[~fwd])
    tan_cone_a = np.tan(np.minimum(0.45 * ang_a, np.radians(max_cone_deg)))
    tan_cone_b = np.tan(np.minimum(0.45 * ang_b, np.radians(max_cone_deg)))

    # subdivision counts from the owners' wished vertex counts
    targets = np.asarray(targets, np.float64)
    deg = ring_len.astype(np.float64)
    wish = np.maximum(0.0, targets - deg) / np.maximum(deg, 1.0)
    w0 = wish[own0]
    w1 = np.where(own1 >= 0, wish[np.maximum(own1, 0)], w0)
    ew = 1.15 * np.sqrt(w0 * w1)
    if forced is not None and len(forced):
        fmask = np.zeros(n, bool)
        fmask[np.asarray(forced)] = True
        touch = fmask[own0] | np.where(own1 >= 0, fmask[np.maximum(own1, 0)], False)
        ew = np.where(touch, np.maximum(w0, w1), ew)
    k = np.floor(ew + rng.random(n_edge)).astype(np.int64)
    dxe = (cx[eb] - cx[ea]).astype(np.float64)
    dye = (cy[eb] - cy[ea]).astype(np.float64)
    elen = np.hypot(dxe, dye)
    k = np.clip(k, 0, np.minimum(1000, (elen // 16).astype(np.int64)))

    # seed-to-edge distance (half the seed separation) caps the jitter
    s0 = seeds[own0]
    s1 = np.where((own1 >= 0)[:, None], seeds[np.maximum(own1, 0)], s0)
    dseed = 0.5 * np.hypot(*(s1 - s0).T)

    sub_off = np.concatenate([[0], np.cumsum(k)]).astype(np.int64)
    tot = int(sub_off[-1])
    e_of = np.repeat(np.arange(n_edge), k)
    j = np.arange(tot, dtype=np.int64) - sub_off[e_of] + 1
    t = j / (k[e_of] + 1.0)
    L = elen[e_of]
    amp = np.minimum.reduce([
        0.2 * dseed[e_of],
        tan_cone_a[e_of] * t * L,
        tan_cone_b[e_of] * (1.0 - t) * L,
    ])
    amp = np.where(boundary[e_of], 0.0, amp)
    off = amp * rng.uniform(-1.0, 1.0, tot)
    nx_ = -dye[e_of] / np.maximum(L, 1.0)
    ny_ = dxe[e_of] / np.maximum(L, 1.0)
    px = np.rint(cx[ea][e_of] + t * dxe[e_of] + off * nx_).astype(np.int64)
    py = np.rint(cy[ea][e_of] + t * dye[e_of] + off * ny_).astype(np.int64)
    # boundary edges stay exactly on their box side
    bx_side = boundary[e_of] & (cx[ea][e_of] == cx[eb][e_of])
    by_side = boundary[e_of] & (cy[ea][e_of] == cy[eb][e_of])
    px = np.where(bx_side, cx[ea][e_of], px)
    py = np.where(by_side, cy[ea][e_of], py)

    # assemble output rings: each occurrence emits its start vertex followed by
    # its edge's subdivision points in the occurrence's direction
    occ_len = 1 + k[einv]
    occ_off = np.concatenate([[0], np.cumsum(occ_len)]).astype(np.int64)
    out_n = int(occ_off[-1])
    ox = np.empty(out_n, np.int64)
    oy = np.empty(out_n, np.int64)
    ox[occ_off[:-1]] = cx[u]
    oy[occ_off[:-1]] = cy[u]
    occ_of = np.repeat(np.arange(len(u)), k[einv])
    jj = np.arange(len(occ_of), dtype=np.int64) - np.repeat(
        np.concatenate([[0], np.cumsum(k[einv])[:-1]]), k[einv])
    kk = k[einv][occ_of]
    src = sub_off[einv[occ_of]] + np.where(fwd[occ_of], jj, kk - 1 - jj)
    dst = occ_off[occ_of] + 1 + jj
    ox[dst] = px[src]
    oy[dst] = py[src]
    out_ring_len = np.bincount(rid, weights=occ_len, minlength=n).astype(np.int64)
    # drop consecutive duplicates created by rounding
    okey = (ox - X0) * (1 << 32) + (oy - Y0)
    okey2, out_ring_len = _compact_rings(okey, out_ring_len)
    ox = (okey2 >> 32) + X0
    oy = (okey2 & ((1 << 32) - 1)) + Y0

    rings_x = [ox]
    rings_y = [oy]
    ring_lens = [out_ring_len]
    # polygon p owns ring p, plus a hole ring for hosts
    n_rings_of = np.ones(n, np.int64)
    island_host = np.zeros(0, np.int64)
    hole_x, hole_y, hole_len = [], [], []
    if hole_mask is not None and np.any(hole_mask):
        # distance from each seed to its nearest neighbour bisector or box side
        dmin = np.minimum.reduce([sx - X0, X1 - sx, sy - Y0, Y1 - sy])
        rp = vor.ridge_points
        m = (rp[:, 0] < n) & (rp[:, 1] < n)
        dd = 0.5 * np.hypot(*(seeds[rp[m, 0]] - seeds[rp[m, 1]]).T)
        np.minimum.at(dmin, rp[m, 0], dd)
        np.minimum.at(dmin, rp[m, 1], dd)
        hosts = np.nonzero(np.asarray(hole_mask) & (0.35 * dmin >= 100.0))[0]
        island_host = hosts
        for h in hosts:
            mv = int(rng.integers(5, 10))
            a = 2 * np.pi * (np.arange(mv) + rng.uniform(-0.3, 0.3, mv)) / mv
            r = 0.35 * dmin[h] * rng.uniform(0.5, 1.0, mv)
            hx = np.rint(sx[h] + r * np.cos(a)).astype(np.int64)
            hy = np.rint(sy[h] + r * np.sin(a)).astype(np.int64)
            hole_x.append(hx)
            hole_y.append(hy)
            hole_len.append(mv)
        n_rings_of[hosts] += 1

    # final ring order: polygon 0..n-1 (outer, then hole), then islands
    outer_start = np.concatenate([[0], np.cumsum(out_ring_len)[:-1]]).astype(np.int64)
    vx_parts, vy_parts, rl = [], [], []
    hole_of = {int(h): i for i, h in enumerate(island_host)}
    if hole_of:
        for p in range(n):
            s = outer_start[p]
            vx_parts.append(ox[s:s + out_ring_len[p]])
            vy_parts.append(oy[s:s + out_ring_len[p]])
            rl.append(out_ring_len[p])
            hi = hole_of.get(p)
            if hi is not None:
                vx_parts.append(hole_x[hi])
                vy_parts.append(hole_y[hi])
                rl.append(hole_len[hi])
        for hi in range(len(island_host)):
            vx_parts.append(hole_x[hi])
            vy_parts.append(hole_y[hi])
            rl.append(hole_len[hi])
        vx = np.concatenate(vx_parts)
        vy = np.concatenate(vy_parts)
        rl = np.asarray(rl, np.int64)
        rings_per_poly = np.concatenate([n_rings_of, np.ones(len(island_host), np.int64)])
    else:
        vx, vy, rl = ox, oy, out_ring_len
        rings_per_poly = n_rings_of
    ring_off = np.concatenate([[0], np.cumsum(rl)]).astype(np.int64)
    poly_ring_off = np.concatenate([[0], np.cumsum(rings_per_poly)]).astype(np.int64)
    pset = PolygonSet(vx.astype(np.int32), vy.astype(np.int32), ring_off, poly_ring_off,
                      parents=[], box=(X0, Y0, X1, Y1))
    pset.meta.update(open_edges=open_edges, n_seeds=n, n_islands=len(island_host))
    return pset, island_host


def nearest_assign(points, centres):
    """Index of the nearest centre for every point (ties: lowest index)."""
    from scipy.spatial import cKDTree

    _, idx = cKDTree(centres).query(points, k=1)
    return idx.astype(np.int64)


def attach_hierarchy(pset, seeds, island_host, rng, n_tracts, n_counties, region_of_county=None):
    """Tracts/counties as unions of blocks by nearest seed (parents only)."""
    n = len(seeds)
    n_tracts = max(1, min(n_tracts, n))
    n_counties = max(1, min(n_counties, n_tracts))
    tseed_idx = rng.choice(n, n_tracts, replace=False)
    tract = nearest_assign(seeds, seeds[tseed_idx])
    cseed_idx = rng.choice(n_tracts, n_counties, replace=False)
    county = nearest_assign(seeds[tseed_idx], seeds[tseed_idx][cseed_idx])
    block_tract = np.concatenate([tract, tract[island_host]]).astype(np.int32)
    if region_of_county is None:
        region_of_county = np.zeros(n_counties, np.int32)
    pset.parents = [block_tract, county.astype(np.int32),
                    np.asarray(region_of_county, np.int32)]
    return pset


def lognormal_targets(rng, n, median, sigma, lo, hi):
    t = np.exp(np.log(median) + sigma * rng.standard_normal(n))
    return np.clip(np.rint(t), lo, hi).astype(np.int64)


def merge_sets(parts, box):
    """Concatenate polygon sets (regions) into one set with a region level."""
    vx = np.concatenate([p.vx for p in parts])
    vy = np.concatenate([p.vy for p in parts])
    ring_off = [np.zeros(1, np.int64)]
    pro = [np.zeros(1, np.int64)]
    vbase = rbase = 0
    par = [[], [], []]
    tbase = cbase = 0
    for ri, p in enumerate(parts):
        ring_off.append(p.ring_off[1:] + vbase)
        pro.append(p.poly_ring_off[1:] + rbase)
        vbase += p.n_vert
        rbase += len(p.ring_off) - 1
        par[0].append(p.parents[0] + tbase)
        par[1].append(p.parents[1] + cbase)
        n_counties = int(p.parents[1].max()) + 1
        par[2].append(np.full(n_counties, ri, np.int32))
        tbase += len(p.parents[1])
        cbase += n_counties
    out = PolygonSet(vx, vy, np.concatenate(ring_off), np.concatenate(pro),
                     parents=[np.concatenate(a).astype(np.int32) for a in par], box=box)
    out.meta["regions"] = [p.box for p in parts]
    return out
