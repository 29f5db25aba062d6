"""Batched form (one persistent work-stealing launch in a CUDA graph) and the
autotuners: every query's ids must equal the CPU oracle's, and separate
plain projections of the same queries, bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from synth import configs, degenerate_lattice, lattice_to_degrees

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


@pytest.fixture(scope="module")
def sets(pipm):
    a = configs.tiny_set()
    b = configs.tiny_set(seed=11, n_blocks=400, holes=0.1)
    c = configs.tiny_set(seed=12, n_blocks=2000, deg=0.5, origin=(-70.0, 40.0), hierarchy=False)
    return [(a, pipm.load_polygon_set(a)), (b, pipm.load_polygon_set(b)),
            (c, pipm.load_polygon_set(c, opts=dict(stage_depth=2)))]


def make_queries(sets, rng, sizes):
    qs = []
    for n in sizes:
        k = int(rng.integers(0, len(sets)))
        ps, s = sets[k]
        if n == 0:
            lon = lat = np.zeros(0)
        else:
            qx, qy = degenerate_lattice(ps, max(3, n // 4), rng)
            lon1, lat1 = lattice_to_degrees(qx), lattice_to_degrees(qy)
            lon2, lat2 = configs.tiny_points(ps, n=n, seed=int(rng.integers(1 << 30)))
            lon = np.concatenate([lon1, lon2])[:n]
            lat = np.concatenate([lat1, lat2])[:n]
        dl = torch.from_numpy(np.ascontiguousarray(lon)).cuda()
        da = torch.from_numpy(np.ascontiguousarray(lat)).cuda()
        out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        qs.append((k, s, dl, da, out))
    return qs


def plain_results(pipm, qs):
    res = []
    for k, s, dl, da, out in qs:
        res.append(pipm.pip_project(s, dl, da).cpu().numpy() if len(dl) else np.zeros(0, np.int32))
    torch.cuda.synchronize()
    return res


def oracle_results(sets, qs):
    return [oracle.join_hier(sets[k][0], dl.cpu().numpy(), da.cpu().numpy()) if len(dl)
            else np.zeros(0, np.int32) for k, s, dl, da, out in qs]


def test_batched_equals_plain(pipm, sets):
    rng = np.random.default_rng(60)
    sizes = [0, 1, 2, 3, 5, 100, 4095, 4096, 4097, 20000, 1] + list(rng.integers(1, 30000, 40))
    qs = make_queries(sets, rng, sizes)
    want = oracle_results(sets, qs)
    for i, p in enumerate(plain_results(pipm, qs)):
        assert (p == want[i]).all(), i
    plan = pipm.Plan(max_points=sum(sizes) + 10, max_queries=len(qs))
    plan.run([(s, dl, da, out) for k, s, dl, da, out in qs])
    plan.check()
    for i, ((k, s, dl, da, out), w) in enumerate(zip(qs, want)):
        assert (out.cpu().numpy() == w).all(), i


def test_plan_reuse_and_double_buffering(pipm, sets):
    rng = np.random.default_rng(61)
    plan = pipm.Plan(max_points=400_000, max_queries=64)
    rounds = []
    for r in range(4):  # back-to-back runs with different query lists
        sizes = list(rng.integers(0, 20000, int(rng.integers(1, 40))))
        qs = make_queries(sets, rng, sizes)
        plan.run([(s, dl, da, out) for k, s, dl, da, out in qs])
        rounds.append(qs)
    plan.check()
    for qs in rounds:
        want = oracle_results(sets, qs)
        for (k, s, dl, da, out), w in zip(qs, want):
            assert (out.cpu().numpy() == w).all()


def test_plan_tune_all_knobs_exact(pipm, sets):
    rng = np.random.default_rng(62)
    sizes = list(rng.integers(1, 50000, 30))
    qs = make_queries(sets, rng, sizes)
    want = oracle_results(sets, qs)
    plan = pipm.Plan(max_points=sum(sizes), max_queries=len(qs))
    knobs = plan.tune([(s, dl, da, out) for k, s, dl, da, out in qs])  # runs every knob setting
    assert knobs["pts_per_cta"] in (128, 256, 512, 1024) and knobs["staged"] in (0, 1)
    for q in qs:
        q[4].fill_(-7)
    plan.run([(s, dl, da, out) for k, s, dl, da, out in qs])
    plan.check()
    for (k, s, dl, da, out), w in zip(qs, want):
        assert (out.cpu().numpy() == w).all()


def test_project_batch_one_shot(pipm, sets):
    rng = np.random.default_rng(63)
    qs = make_queries(sets, rng, [10, 3000, 0, 7777])
    want = oracle_results(sets, qs)
    pipm.pip_project_batch([(s, dl, da, out) for k, s, dl, da, out in qs])
    for (k, s, dl, da, out), w in zip(qs, want):
        assert (out.cpu().numpy() == w).all()


def test_plan_limits(pipm, sets):
    rng = np.random.default_rng(64)
    qs = make_queries(sets, rng, [100, 200])
    plan = pipm.Plan(max_points=250, max_queries=2)
    with pytest.raises(pipm.PipError) as e:
        plan.run([(s, dl, da, out) for k, s, dl, da, out in qs])
    assert e.value.status == 1
    with pytest.raises(pipm.PipError):
        pipm.Plan(max_points=0, max_queries=1)


def test_set_tune_keeps_results(pipm):
    ps = configs.tiny_set(seed=13, n_blocks=800, holes=0.05)
    s = pipm.load_polygon_set(ps)
    lon, lat = configs.tiny_points(ps, n=200_000, seed=65)
    dl, da = torch.from_numpy(lon).cuda(), torch.from_numpy(lat).cuda()
    chosen = pipm.pip_set_tune(s, dl, da)
    assert chosen["pts_per_cta"] in (128, 256, 512, 1024)
    assert chosen["stage_depth"] in (-1, 1, 2)
    got = pipm.pip_project(s, dl, da).cpu().numpy()
    assert (got == oracle.join_hier(ps, lon, lat)).all()
    assert s.info()["cell_log2"] == chosen["cell_log2"]


def test_prepared_query_list_runs_repeatedly(pipm, sets):
    """A query list marshalled once (Queries) and run several times gives the
    oracle's ids each time (outputs reset between runs)."""
    rng = np.random.default_rng(66)
    sizes = [0, 1, 4097, 5000, 123] + list(rng.integers(1, 20000, 20))
    qs = make_queries(sets, rng, sizes)
    want = oracle_results(sets, qs)
    prepared = pipm.Queries([(s, dl, da, out) for k, s, dl, da, out in qs])
    plan = pipm.Plan(max_points=sum(sizes), max_queries=len(qs))
    for _ in range(3):
        for q in qs:
            q[4].fill_(-7)
        plan.run(prepared)
        plan.check()
        for i, ((k, s, dl, da, out), w) in enumerate(zip(qs, want)):
            assert (out.cpu().numpy() == w).all(), i
