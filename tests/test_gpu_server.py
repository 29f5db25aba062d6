"""Served form: continuous batching over resident sets. Every request's ids
must equal the CPU oracle's, served alone, served in a concurrent mix and
projected by the plain path (tolerance 0: ids are integers)."""
import threading
import time

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
def resident(pipm):
    ps = [configs.tiny_set(), configs.tiny_set(seed=11, n_blocks=400, holes=0.1),
          configs.tiny_set(seed=12, n_blocks=1500, deg=0.5, origin=(-70.0, 40.0))]
    return ps, [pipm.load_polygon_set(p) for p in ps]


def requests(ps_list, rng, sizes):
    reqs = []
    for n in sizes:
        k = int(rng.integers(0, len(ps_list)))
        ps = ps_list[k]
        qx, qy = degenerate_lattice(ps, max(3, n // 3), rng)
        lon2, lat2 = configs.tiny_points(ps, n=max(n, 1), seed=int(rng.integers(1 << 30)))
        lon = np.concatenate([lattice_to_degrees(qx), lon2])[:n]
        lat = np.concatenate([lattice_to_degrees(qy), lat2])[:n]
        lon_p = torch.from_numpy(np.ascontiguousarray(lon)).pin_memory()
        lat_p = torch.from_numpy(np.ascontiguousarray(lat)).pin_memory()
        out = torch.full((n,), -7, dtype=torch.int32).pin_memory()
        reqs.append((k, lon_p, lat_p, out))
    return reqs


def oracle_ids(ps_list, reqs):
    return [oracle.join_hier(ps_list[k], lon.numpy(), lat.numpy()) if len(lon) else np.zeros(0, np.int32)
            for k, lon, lat, _ in reqs]


def plain(pipm, sets, reqs):
    res = []
    for k, lon, lat, out in reqs:
        if len(lon) == 0:
            res.append(np.zeros(0, np.int32))
            continue
        res.append(pipm.pip_project(sets[k], lon.cuda(), lat.cuda()).cpu().numpy())
    torch.cuda.synchronize()
    return res


def test_alone_equals_mix_equals_plain(pipm, resident):
    ps_list, sets = resident
    rng = np.random.default_rng(70)
    sizes = [0, 1, 2, 31, 1000, 40000, 100_000] + list((10 ** rng.uniform(0, 5, 120)).astype(int))
    reqs = requests(ps_list, rng, sizes)
    want = oracle_ids(ps_list, reqs)
    for i, got in enumerate(plain(pipm, sets, reqs)):
        assert (got == want[i]).all(), i
    srv = pipm.Server(sets, dict(n_streams=2, max_batch_queries=64))
    # alone: one request at a time
    alone = []
    for k, lon, lat, out in reqs[:40]:
        t = srv.submit(k, lon, lat, out)
        srv.wait(t)
        alone.append(out.numpy().copy())
        out.fill_(-7)
    # mix: all requests from 4 threads with random gaps
    tickets = [None] * len(reqs)

    def producer(idx):
        r = np.random.default_rng(int(idx[0]) + 100)
        for i in idx:
            k, lon, lat, out = reqs[i]
            tickets[i] = srv.submit(k, lon, lat, out)
            time.sleep(float(r.uniform(0, 0.0005)))

    parts = np.array_split(np.arange(len(reqs)), 4)
    ths = [threading.Thread(target=producer, args=(p,)) for p in parts]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    for t in tickets:
        srv.wait(t, timeout_us=60_000_000)
    st = srv.stats()
    srv.close()
    for i, (k, lon, lat, out) in enumerate(reqs):
        assert (out.numpy() == want[i]).all(), i
    for i, a in enumerate(alone):
        assert (a == want[i]).all(), i
    assert st["completed"] == 40 + len(reqs)
    assert st["p99_us"] >= st["p50_us"] > 0
    assert st["mean_batch_queries"] >= 1.0


def test_server_limits(pipm, resident):
    ps_list, sets = resident
    srv = pipm.Server(sets, dict(n_streams=1, max_batch_points=1000, max_batch_queries=8))
    big = np.zeros(1001)
    out = np.zeros(1001, np.int32)
    st, _ = srv.try_submit(5, big[:10], big[:10], out[:10])
    assert st == 1  # no such set
    t = srv.submit(0, big[:0], big[:0], out[:0])  # empty request completes
    srv.wait(t, timeout_us=10_000_000)
    srv.close()


def test_request_larger_than_a_launch_is_split(pipm, resident):
    """A request of about three launches (cap 1000 points) plus a ragged tail
    is served in parts and its ticket completes once; small requests submitted
    meanwhile from another thread are served alongside. Every id equals the
    oracle's."""
    ps_list, sets = resident
    rng = np.random.default_rng(73)
    big = requests(ps_list, rng, [3 * 1000 + 17, 2000, 1000])
    small = requests(ps_list, rng, list((10 ** rng.uniform(0, 3, 40)).astype(int)))
    want_big, want_small = oracle_ids(ps_list, big), oracle_ids(ps_list, small)
    srv = pipm.Server(sets, dict(n_streams=2, max_batch_points=1000, max_batch_queries=8))
    tickets = [None] * len(small)

    def producer():
        for i, (k, lon, lat, out) in enumerate(small):
            tickets[i] = srv.submit(k, lon, lat, out)

    th = threading.Thread(target=producer)
    th.start()
    big_t = [srv.submit(k, lon, lat, out) for k, lon, lat, out in big]
    th.join()
    for t in big_t + tickets:
        srv.wait(t, timeout_us=60_000_000)
    st = srv.stats()
    srv.close()
    for i, (k, lon, lat, out) in enumerate(big):
        assert (out.numpy() == want_big[i]).all(), i
    for i, (k, lon, lat, out) in enumerate(small):
        assert (out.numpy() == want_small[i]).all(), i
    assert st["completed"] == len(big) + len(small)  # one completion per ticket, not per part
    assert st["launches"] >= 6


def test_pageable_host_buffers(pipm, resident):
    ps_list, sets = resident
    rng = np.random.default_rng(71)
    reqs = requests(ps_list, rng, [5000, 70_000])
    want = oracle_ids(ps_list, reqs)
    srv = pipm.Server(sets, dict(n_streams=2))
    outs = []
    for k, lon, lat, out in reqs:
        o = np.full(len(lon), -7, np.int32)
        hl, ha = lon.numpy().copy(), lat.numpy().copy()  # pageable, alive until done
        t = srv.submit(k, hl, ha, o)
        srv.wait(t)
        outs.append(o)
    srv.close()
    for o, w in zip(outs, want):
        assert (o == w).all()
