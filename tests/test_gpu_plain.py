"""GPU parity of the plain projection path against the CPU oracle.

Ids are integers, so the bar is bit-exact equality with the oracle (O1,
itself pinned to O0 and to the paper in test_oracle_pins.py) on every case.
All calls go through the C ABI (libpip.so via the Python binding).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from synth import configs, degenerate_lattice, lattice_to_degrees
from tests import oracle_pins as pins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pipm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_03156_gb300 as pipm
    from paper_2005_03156_gb300 import build
    build.build()
    pipm.lib()
    return pipm


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def project(pipm, s, lon, lat):
    out = pipm.pip_project(s, dev(lon), dev(lat))
    pipm.pip_set_check(s)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_device_quantizer_matches_oracle(pipm):
    v = pins.q_cases(np.random.default_rng(7))
    q, ok = pipm.pip_quantize(dev(v))
    torch.cuda.synchronize()
    oq, ook = oracle.quantize(v)
    ok = ok.cpu().numpy().astype(bool)
    q = q.cpu().numpy()
    assert (ok == ook).all()
    assert (q[ok] == oq[ok]).all()


def test_tiny_full_config(pipm, tiny_set):
    s = pipm.load_polygon_set(tiny_set)
    lon, lat = configs.tiny_points(tiny_set)
    got = project(pipm, s, lon, lat)
    want = oracle.join_hier(tiny_set, lon, lat)
    assert (got == want).all(), int((got != want).sum())
    info = s.info()
    assert info["leaves"] > 0 and info["interior_cells"] > 0


def test_degenerate_points(pipm, tiny_set):
    s = pipm.load_polygon_set(tiny_set)
    qx, qy = degenerate_lattice(tiny_set, 200_000, np.random.default_rng(21))
    lon, lat = lattice_to_degrees(qx), lattice_to_degrees(qy)
    got = project(pipm, s, lon, lat)
    want = oracle.join_hier(tiny_set, lon, lat)
    assert (got == want).all(), int((got != want).sum())


def test_holes_and_islands(pipm, tiny_set_holes):
    ps = tiny_set_holes
    s = pipm.load_polygon_set(ps)
    qx, qy = degenerate_lattice(ps, 100_000, np.random.default_rng(22))
    lon, lat = lattice_to_degrees(qx), lattice_to_degrees(qy)
    lon2, lat2 = configs.tiny_points(ps, n=200_000, seed=23)
    lon, lat = np.concatenate([lon, lon2]), np.concatenate([lat, lat2])
    got = project(pipm, s, lon, lat)
    want = oracle.join_hier(ps, lon, lat)
    assert (got == want).all(), int((got != want).sum())


OPTION_CASES = [
    dict(max_depth=-1),                                  # uniform grid
    dict(max_depth=-1, cell_log2=14),                    # fine uniform grid
    dict(max_depth=-1, cell_log2=22),                    # one coarse cell
    dict(leaf_edges=2, size_ratio=64),                   # deep trie, many palette overflows
    dict(cell_log2=21, leaf_edges=4, max_depth=8),       # coarse top grid, deep trie
    dict(stage_depth=1, pts_per_cta=7),                  # single stage, tiny items
    dict(stage_depth=2, pts_per_cta=1000),               # items larger than the CTA
    dict(stage_depth=-1, pts_per_cta=300),               # no staging
    dict(cand_mode=2),                                   # box rasterization
    dict(cand_mode=1, size_ratio=-1, leaf_edges=1000, compact_edges=-1),  # long lists (warp ballots)
    dict(compact_edges=-1),                              # no compact leaves: every leaf is residual
    dict(leaf_edges=2, size_ratio=64, compact_edges=-1),  # deep trie, palette overflows become leaves
    dict(compact_edges=1),                               # one-slot records only
    dict(compact_edges=7),                               # records of up to four slots
    dict(compact_edges=2, max_depth=1),                  # compact records beside residual leaves
    dict(compact_edges=7, cell_log2=21, max_depth=8),    # coarse top grid, compact deep down
    dict(compact_edges=3, max_depth=-1, cell_log2=15),   # uniform grid of compact cells
    dict(compact_edges=1, compact_early=1),              # compact cells stop splitting (one edge)
    dict(compact_edges=3, compact_early=1, size_ratio=16),  # ... and up to three edges, shallow
    dict(bin_residual=1),                                # residual binned by superbin
    dict(bin_residual=-1, leaf_edges=2, size_ratio=8),   # residual tested in arrival order (holes skipped)
]


def test_binned_and_arrival_order_crossing_tests_agree(pipm, tiny_set_holes):
    """The crossing kernel over the binned residual (bin_residual = 1) and over
    the queue in arrival order (the default) give the oracle's ids, at a
    residual density of many points per superbin."""
    ps = tiny_set_holes
    lon, lat = configs.tiny_points(ps, n=200_000, seed=27)
    want = oracle.join_hier(ps, lon, lat)
    for b in (1, 0):
        s = pipm.load_polygon_set(ps, opts=dict(leaf_edges=1000, size_ratio=-1, max_depth=-1, cell_log2=16,
                                                bin_residual=b))
        got, stats = pipm.pip_project_ex(s, torch.from_numpy(lon).cuda(), torch.from_numpy(lat).cuda())
        assert (got.cpu().numpy() == want).all(), b
        assert stats["residual"] >= 8 * s.info()["superbins"]


@pytest.mark.parametrize("opts", OPTION_CASES, ids=[str(o) for o in OPTION_CASES])
def test_build_options(pipm, tiny_set_holes, opts):
    ps = tiny_set_holes
    s = pipm.load_polygon_set(ps, opts=opts)
    qx, qy = degenerate_lattice(ps, 60_000, np.random.default_rng(24))
    lon, lat = lattice_to_degrees(qx), lattice_to_degrees(qy)
    lon2, lat2 = configs.tiny_points(ps, n=100_000, seed=25)
    lon, lat = np.concatenate([lon, lon2]), np.concatenate([lat, lat2])
    got = project(pipm, s, lon, lat)
    want = oracle.join_hier(ps, lon, lat)
    assert (got == want).all(), (opts, int((got != want).sum()))


def test_compact_leaves_answer_in_the_classify_kernel(pipm, tiny_set_holes):
    """Compact leaves (boundary cells with few distinct edges, answered by the
    exact crossing test inside K1): results equal the oracle and the index
    without compact leaves, and almost no point is left for the residual
    crossing kernel."""
    ps = tiny_set_holes
    qx, qy = degenerate_lattice(ps, 60_000, np.random.default_rng(26))
    lon, lat = lattice_to_degrees(qx), lattice_to_degrees(qy)
    lon2, lat2 = configs.tiny_points(ps, n=200_000, seed=27)
    lon, lat = np.concatenate([lon, lon2]), np.concatenate([lat, lat2])
    want = oracle.join_hier(ps, lon, lat)
    res = {}
    for ce in (3, -1):
        s = pipm.load_polygon_set(ps, opts={"compact_edges": ce})
        out, stats = pipm.pip_project_ex(s, dev(lon), dev(lat))
        pipm.pip_set_check(s)
        got = out.cpu().numpy()
        assert (got == want).all(), (ce, int((got != want).sum()))
        res[ce] = (s.info(), stats["residual"])
    info_on, residual_on = res[3]
    info_off, residual_off = res[-1]
    assert info_on["compact_leaves"] > 0 and sum(info_on["compact_by_edges"]) == info_on["compact_leaves"]
    assert info_on["compact_by_edges"][4:] == [0, 0, 0, 0]  # at most 3 edges
    assert info_off["compact_leaves"] == 0
    assert residual_on * 10 < residual_off


def test_hierarchy_descent_equals_rasterization(pipm, tiny_set):
    s = pipm.load_polygon_set(tiny_set)
    o1, i1 = pipm.pip_set_top_candidates(s, 1)
    o2, i2 = pipm.pip_set_top_candidates(s, 2)
    assert (o1 == o2).all() and (i1 == i2).all()
    # brute force: polygons whose closed box meets each cell's closed rect
    info = s.info()
    sh, x0, y0, nx = info["cell_log2"], info["grid_x0"], info["grid_y0"], info["grid_nx"]
    v = tiny_set.ring_off[tiny_set.poly_ring_off]
    for p in np.random.default_rng(3).choice(tiny_set.n_poly, 50, replace=False):
        xs, ys = tiny_set.vx[v[p]:v[p + 1]], tiny_set.vy[v[p]:v[p + 1]]
        cx0, cx1 = (xs.min() - x0) >> sh, (xs.max() - x0) >> sh
        cy0, cy1 = (ys.min() - y0) >> sh, (ys.max() - y0) >> sh
        for cy in range(cy0, cy1 + 1):
            for cx in range(cx0, cx1 + 1):
                c = cy * nx + cx
                assert p in i1[o1[c]:o1[c + 1]]


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 31, 33, 1023, 1025, 4097])
def test_ragged_sizes(pipm, tiny_set, n):
    s = pipm.load_polygon_set(tiny_set)
    lon, lat = configs.tiny_points(tiny_set, n=max(n, 1), seed=30 + n)
    lon, lat = lon[:n], lat[:n]
    got = project(pipm, s, lon, lat) if n else np.zeros(0, np.int32)
    want = oracle.join_hier(tiny_set, lon, lat)
    assert (got == want).all()


def test_unaligned_pointers_take_scalar_path(pipm, tiny_set):
    s = pipm.load_polygon_set(tiny_set)
    lon, lat = configs.tiny_points(tiny_set, n=10_001, seed=40)
    dl, da = dev(lon), dev(lat)
    out = torch.empty(10_001, dtype=torch.int32, device="cuda")
    got = pipm.pip_project(s, dl[1:], da[1:], out[1:])
    torch.cuda.synchronize()
    want = oracle.join_hier(tiny_set, lon[1:], lat[1:])
    assert (out[1:].cpu().numpy() == want).all()
    del got


def test_host_pointer_streaming(pipm, tiny_set):
    s = pipm.load_polygon_set(tiny_set)
    lon, lat = configs.tiny_points(tiny_set, n=300_000, seed=41)
    got = pipm.pip_project(s, lon, lat)              # numpy in/out -> chunked pipeline
    want = oracle.join_hier(tiny_set, lon, lat)
    assert (got == want).all()
    lon_p = torch.from_numpy(lon).pin_memory()
    lat_p = torch.from_numpy(lat).pin_memory()
    out_p = torch.empty(len(lon), dtype=torch.int32).pin_memory()
    pipm.pip_project(s, lon_p, lat_p, out_p)
    assert (out_p.numpy() == want).all()


def test_invalid_coordinates(pipm, tiny_set):
    s = pipm.load_polygon_set(tiny_set)
    bad = np.array([np.nan, np.inf, -np.inf, 1e300, 215.0, -215.0, 0.5, 0.5], np.float64)
    ok = np.array([0.5, 0.5, 0.5, 0.5, 0.5, 0.5, np.nan, 214.7483648], np.float64)
    got = project(pipm, s, bad, ok)
    assert (got == -1).all()
    got = project(pipm, s, ok[:6], bad[:6])
    assert (got == -1).all()


def test_overlapping_polygons_lowest_id(pipm):
    a = [[(0, 0), (600, 0), (600, 600), (0, 600)]]
    b = [[(300, 300), (900, 300), (900, 900), (300, 900)]]
    c = [[(100, 100), (200, 100), (200, 200), (100, 200)]]
    ps = pins.poly_set([b, a, c])
    s = pipm.pip_set_load_i32(ps.vx, ps.vy, ps.ring_off, ps.poly_ring_off, opts=dict(cell_log2=6))
    X, Y = np.meshgrid(np.arange(-5, 910, 3), np.arange(-5, 910, 3), indexing="ij")
    lon, lat = lattice_to_degrees(X.ravel()), lattice_to_degrees(Y.ravel())
    got = project(pipm, s, lon, lat)
    want = oracle.join_hier(ps, lon, lat)
    assert (got == want).all()


def test_f64_vertex_load(pipm, tiny_set):
    s = pipm.pip_set_load_f64(lattice_to_degrees(tiny_set.vx), lattice_to_degrees(tiny_set.vy),
                              tiny_set.ring_off, tiny_set.poly_ring_off, parents=tiny_set.parents)
    lon, lat = configs.tiny_points(tiny_set, n=100_000, seed=42)
    assert (project(pipm, s, lon, lat) == oracle.join_hier(tiny_set, lon, lat)).all()


def test_load_errors(pipm):
    PipError = pipm.PipError
    ps = pins.poly_set([[[(0, 0), (10, 0), (10, 10)]]])
    with pytest.raises(PipError) as e:
        pipm.pip_set_load_i32(ps.vx, ps.vy, np.array([0, 2], np.int64), ps.poly_ring_off)
    assert e.value.status == 1
    big = pins.poly_set([[[(-2**31 + 5, 0), (2**31 - 5, 0), (0, 10)]]])
    with pytest.raises(PipError) as e:
        pipm.pip_set_load_i32(big.vx, big.vy, big.ring_off, big.poly_ring_off)
    assert e.value.status == 4
    with pytest.raises(PipError) as e:
        pipm.pip_set_load_i32(ps.vx, ps.vy, ps.ring_off, ps.poly_ring_off,
                              parents=[np.array([-1], np.int32)])
    assert e.value.status == 1


def test_rebuild_keeps_results(pipm, tiny_set):
    s = pipm.load_polygon_set(tiny_set)
    lon, lat = configs.tiny_points(tiny_set, n=100_000, seed=43)
    a = project(pipm, s, lon, lat)
    pipm.pip_set_rebuild(s, dict(cell_log2=15, max_depth=1))
    b = project(pipm, s, lon, lat)
    assert (a == b).all()


@pytest.mark.slow
def test_state_scale_sampled(pipm):
    """Full state-scale set and 1e8 points in the bench's launch shape;
    a random sample of outputs is checked against the oracle point by point,
    and every output is a valid id."""
    ps = configs.state_set()
    s = pipm.load_polygon_set(ps)
    assert s.info()["size_ratio"] == 128  # the automatic split ratio
    lon, lat = configs.state_points()
    dlon, dlat = dev(lon), dev(lat)
    out = pipm.pip_project(s, dlon, dlat)
    pipm.pip_set_check(s)
    got = out.cpu().numpy()
    assert got.min() >= -1 and got.max() < ps.n_poly
    idx = np.random.default_rng(44).choice(len(lon), 200_000, replace=False)
    want = oracle.join_hier(ps, lon[idx], lat[idx])
    assert (got[idx] == want).all(), int((got[idx] != want).sum())


def kd_rectangles(rng, box, n):
    """Axis-aligned partition of box by random kd splits (T-junctions,
    many horizontal edges)."""
    rects = [box]
    while len(rects) < n:
        i = int(np.argmax([(r[2] - r[0]) * (r[3] - r[1]) for r in rects]))
        x0, y0, x1, y1 = rects.pop(i)
        if (x1 - x0 >= y1 - y0 and x1 - x0 > 2) or y1 - y0 <= 2:
            m = int(rng.integers(x0 + 1, x1))
            rects += [(x0, y0, m, y1), (m, y0, x1, y1)]
        else:
            m = int(rng.integers(y0 + 1, y1))
            rects += [(x0, y0, x1, m), (x0, m, x1, y1)]
    return [[[(a, b), (c, b), (c, d), (a, d)]] for a, b, c, d in rects]


@pytest.mark.parametrize("opts", [None, dict(leaf_edges=1, size_ratio=64, compact_edges=-1),
                                  dict(max_depth=-1), dict(cell_log2=12, max_depth=5),
                                  dict(compact_edges=7, cell_log2=12, max_depth=5)])
def test_axis_aligned_partition(pipm, opts):
    rng = np.random.default_rng(50)
    box = (1000, 2000, 1000 + 40_000, 2000 + 30_000)
    ps = pins.poly_set(kd_rectangles(rng, box, 400))
    s = pipm.pip_set_load_i32(ps.vx, ps.vy, ps.ring_off, ps.poly_ring_off, opts=opts)
    # every vertex, points one unit around vertices, and uniform lattice points
    qx = np.concatenate([ps.vx, ps.vx + 1, ps.vx - 1, ps.vx, rng.integers(box[0] - 5, box[2] + 5, 100_000)])
    qy = np.concatenate([ps.vy, ps.vy, ps.vy + 1, ps.vy - 1, rng.integers(box[1] - 5, box[3] + 5, 100_000)])
    lon, lat = lattice_to_degrees(qx), lattice_to_degrees(qy)
    got = project(pipm, s, lon, lat)
    want = oracle.join_hier(ps, lon, lat)
    assert (got == want).all(), int((got != want).sum())
    inside = (qx >= box[0]) & (qx < box[2]) & (qy >= box[1]) & (qy < box[3])
    assert (got[inside] >= 0).all() and (got[~inside] == -1).all()


def test_parent_ids_follow_the_hierarchy(pipm, tiny_set):
    s = pipm.load_polygon_set(tiny_set)
    lon, lat = configs.tiny_points(tiny_set, n=50_000, seed=55)
    ids = pipm.pip_project(s, dev(lon), dev(lat))
    want = oracle.join_hier(tiny_set, lon, lat)  # expected ancestors come from the oracle's ids
    assert (ids.cpu().numpy() == want).all()
    for level, par in enumerate(tiny_set.parents, start=1):
        got = pipm.pip_parent_ids(s, ids, level).cpu().numpy()
        want = np.where(want >= 0, par[np.maximum(want, 0)], -1)
        assert (got == want).all(), level
    with pytest.raises(pipm.PipError):
        pipm.pip_parent_ids(s, ids, len(tiny_set.parents) + 1)


@pytest.mark.parametrize("case", ["tiny_4096", "small_64"])
def test_approximate_mode_error_bound(pipm, tiny_set, case):
    """Approximate mode (Sec. IV, the error-bounded variant of true-hit
    filtering): no crossing test runs at query time; a point in a boundary
    leaf (side 2^k <= approx_units, aligned to the top grid) gets the exact
    id (oracle) of the leaf's centre lattice point, which lies at Chebyshev
    distance <= approx_units / 2; every other point gets its exact id. The
    check: each returned id equals the oracle's id at the point or at the
    centre of one of the aligned power-of-two cells of side <= approx_units
    around it."""
    if case == "tiny_4096":
        ps, approx = tiny_set, 4096
    else:
        ps, approx = configs.tiny_set(n_blocks=200, deg=0.1, origin=(0.3, 0.4)), 64
    s = pipm.load_polygon_set(ps, opts={"approx_units": approx})
    lon, lat = configs.tiny_points(ps, n=200_000, seed=11)
    out, stats = pipm.pip_project_ex(s, dev(lon), dev(lat))
    pipm.pip_set_check(s)
    got = out.cpu().numpy()
    assert stats["residual"] == 0  # every leaf answers from its table entry
    want = oracle.join_hier(ps, lon, lat)
    qx, ok_x = oracle.quantize(lon)
    qy, ok_y = oracle.quantize(lat)
    ok = ok_x & ok_y
    assert (got[~ok] == -1).all()
    info = s.info()
    gx0, gy0 = int(info["grid_x0"]), int(info["grid_y0"])
    allowed = got == want
    k = 0
    while (1 << k) <= approx:
        side = 1 << k
        cx = gx0 + ((qx.astype(np.int64) - gx0) // side) * side + side // 2
        cy = gy0 + ((qy.astype(np.int64) - gy0) // side) * side + side // 2
        assert (np.abs(cx - qx) <= approx // 2).all() and (np.abs(cy - qy) <= approx // 2).all()
        at_centre = oracle.join_hier(ps, lattice_to_degrees(cx), lattice_to_degrees(cy))
        allowed |= got == at_centre
        k += 1
    bad = np.nonzero(ok & ~allowed)[0]
    assert len(bad) == 0, (len(bad), bad[:5].tolist())
    mism = int((got != want).sum())
    assert mism < 0.05 * len(got), mism
    # the same set built exact still answers exactly
    e = pipm.load_polygon_set(ps)
    assert (project(pipm, e, lon, lat) == want).all()


def test_bounded_wait_runs_out_and_context_survives(pipm, tiny_set):
    """Failure detection without a fault: a device wait on an mbarrier that
    nothing completes gives up after its limit, the kernel reports it
    (PIP_ETIMEOUT) and returns, and the context keeps working."""
    import time
    t0 = time.perf_counter()
    assert pipm.pip_selftest_bounded_wait(20_000_000) == 5  # 20 ms limit -> PIP_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    with pytest.raises(pipm.PipError):
        pipm._native.check(pipm.pip_selftest_bounded_wait(0))
    s = pipm.load_polygon_set(tiny_set)
    lon, lat = configs.tiny_points(tiny_set, n=50_000)
    assert (project(pipm, s, lon, lat) == oracle.join_hier(tiny_set, lon, lat)).all()


def _torch_allocator(fail_after=None):
    """An allocator hook on torch's caching allocator that records live
    blocks; with fail_after=k the (k+1)-th allocation returns NULL."""
    from paper_2005_03156_gb300 import _native
    state = {"live": {}, "allocs": 0, "frees": 0}

    @_native.ALLOC_FN
    def alloc(nbytes, stream, ctx):
        if fail_after is not None and state["allocs"] >= fail_after:
            return None
        state["allocs"] += 1
        p = torch.cuda.caching_allocator_alloc(max(int(nbytes), 1))
        state["live"][p] = int(nbytes)
        return p

    @_native.FREE_FN
    def free(ptr, stream, ctx):
        state["frees"] += 1
        state["live"].pop(ptr)
        torch.cuda.caching_allocator_delete(ptr)

    return _native.Allocator(alloc, free, None), state


def test_allocator_hook_and_injected_failures(pipm, tiny_set):
    """Every device allocation of a set goes through the caller's hook; an
    allocation that fails part-way through a load gives PIP_ENOMEM and every
    block taken so far is given back; the context keeps working."""
    lon, lat = configs.tiny_points(tiny_set, n=30_000)
    want = oracle.join_hier(tiny_set, lon, lat)
    A, st = _torch_allocator()
    s = pipm.load_polygon_set(tiny_set, allocator=A)
    assert (project(pipm, s, lon, lat) == want).all()
    assert st["allocs"] > 0
    s.free()
    torch.cuda.synchronize()
    assert not st["live"] and st["frees"] == st["allocs"]
    for k in (0, 1, 5, 20):
        B, sb = _torch_allocator(fail_after=k)
        with pytest.raises(pipm.PipError) as e:
            pipm.load_polygon_set(tiny_set, allocator=B)
        assert e.value.status == 2, (k, e.value)
        torch.cuda.synchronize()
        assert not sb["live"], (k, len(sb["live"]))
    s2 = pipm.load_polygon_set(tiny_set)
    assert (project(pipm, s2, lon, lat) == want).all()


def test_too_many_points_for_one_device_call_is_refused(pipm, tiny_set):
    """The residual queue is indexed with 32 bits: a device-resident call of
    2^32 points is refused with PIP_EINVAL before any memory is touched."""
    import ctypes
    s = pipm.load_polygon_set(tiny_set)
    lon, lat = dev(np.zeros(4)), dev(np.zeros(4))
    out = torch.empty(4, dtype=torch.int32, device="cuda")
    lib = pipm._native.load()
    st = lib.pip_project(s.handle, ctypes.c_void_p(lon.data_ptr()), ctypes.c_void_p(lat.data_ptr()),
                         1 << 32, ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1  # PIP_EINVAL
    assert (project(pipm, s, np.zeros(4), np.zeros(4)) == oracle.join_hier(tiny_set, np.zeros(4), np.zeros(4))).all()
