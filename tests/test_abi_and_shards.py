"""CPU-only checks: the C-ABI library builds for sm_103a, loads and exports
every function include/pip.h declares (no GPU calls); host sharding and the
max-over-ranks timing reduction across two gloo ranks."""
import os
import re
import socket

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "include", "pip.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\**\s+(pip_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("pip_set_load_i32", "pip_set_load_f64", "pip_project", "pip_project_batch",
                 "pip_plan_create", "pip_plan_run", "pip_set_tune", "pip_server_create",
                 "pip_server_submit", "pip_server_wait", "pip_server_destroy", "pip_set_free",
                 "pip_last_error", "pip_project_noalloc"):
        assert must in names, must


def test_library_builds_loads_and_exports_every_symbol():
    if not (os.environ.get("NVCC") or __import__("shutil").which("nvcc")
            or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    import ctypes
    from paper_2005_03156_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.pip_version.restype = ctypes.c_int32
    assert lib.pip_version() >= 10000
    from paper_2005_03156_gb300 import _native
    assert set(_native.SIGNATURES) >= set(declared_functions())  # the binding covers the header


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2005_03156_gb300 import _native
    monkeypatch.setattr(_native, "_lib", None)
    monkeypatch.setattr(_native, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        _native.load()


def test_shard_bounds_partition():
    from paper_2005_03156_gb300.shard import shard_bounds
    for n in (0, 1, 7, 100, 1_000_003):
        for w in (1, 2, 3, 8):
            b = [shard_bounds(n, r, w) for r in range(w)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[i][1] == b[i + 1][0] for i in range(w - 1))
            assert max(e - s for s, e in b) - min(e - s for s, e in b) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    from paper_2005_03156_gb300.shard import max_over_ranks, shard_bounds
    from synth import configs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ps = configs.tiny_set(n_blocks=200)
        lon, lat = configs.tiny_points(ps, n=20_001)
        a, b = shard_bounds(len(lon), rank, world)
        ids = oracle.join_hier(ps, lon[a:b], lat[a:b], threads=1)
        import torch
        parts = [None] * world
        dist.all_gather_object(parts, (a, b, ids.tolist()))
        t = max_over_ranks(float(rank + 1))
        q.put((rank, parts, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import multiprocessing as mp

    import oracle
    from synth import configs
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ps = configs.tiny_set(n_blocks=200)
    lon, lat = configs.tiny_points(ps, n=20_001)
    want = oracle.join_hier(ps, lon, lat)
    for rank, parts, t in res:
        assert t == 2.0  # max over ranks of rank + 1
        got = np.full(len(lon), -9, np.int32)
        for a, b, ids in parts:
            got[a:b] = ids
        assert (got == want).all()


def _struct_fields(name):
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r";", text)
    assert m, name
    return re.findall(r"\b(?:int32_t|int64_t|double|void\s*\*|pip_set|const double\s*\*|int32_t\s*\*)\s+([a-z_0-9]+)\s*;", m.group(1))


def test_binding_structs_match_the_header():
    from paper_2005_03156_gb300 import _native
    for cname, pycls in (("pip_build_opts", _native.BuildOpts), ("pip_project_stats", _native.ProjectStats)):
        assert _struct_fields(cname) == [f for f, _ in pycls._fields_], cname


def _failing_rank_main(rank, world, port, q):
    import datetime

    import torch.distributed as dist

    from paper_2005_03156_gb300.shard import max_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)  # this rank dies between steps, before the step's timing reduction
    try:
        max_over_ranks(1.0)
        q.put((rank, "no error"))
    except Exception as e:  # the survivor's collective must fail, not hang
        q.put((rank, type(e).__name__))


def test_dead_rank_fails_the_timing_reduction_instead_of_hanging():
    import multiprocessing as mp
    import queue
    import time

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_rank_main, args=(r, 2, port, q)) for r in range(2)]
    t0 = time.time()
    for p in procs:
        p.start()
    try:
        rank, what = q.get(timeout=120)
    except queue.Empty:
        rank, what = None, "hung"
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
            p.join()
    assert rank == 0 and what not in ("no error", "hung"), (rank, what)
    assert procs[1].exitcode == 3
    assert time.time() - t0 < 150
