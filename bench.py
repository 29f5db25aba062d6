#!/usr/bin/env python
"""Point -> census-block projections/s on GB300 (Kepner et al., "Fast Mapping
onto Census Blocks"), measured on the state-scale workload by default:
200,000 synthetic block polygons (3-level hierarchy, lognormal vertex
counts, 2% holes) over 5x5 degrees and 1e8 float64 mixture points.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config state|tiny] [--points N] [--no-e2e] [--no-cpu-baseline]

One step = one pip_project call over the whole batch (K1 classify, K2 bin
when binning is on, K3 cross), inputs resident in HBM. Under torchrun (N > 1) every rank
projects its own 1e8 points against a replica of the set (weak scaling, no
collective on the data path); value = all ranks' points / max rank time.
At N = 1 the same line also carries the metric's two other parts, measured
after the plain join: "batched" (the 4,096-query batched workload over 8
resident sets in one graph launch, against the same queries as separate
plain launches) and "serve" (one offered load of the serving workload over
3 resident state-scale sets: p50/p99 latency of the continuous-batching
server against per-request plain launches); --no-batched / --no-serve skip
them. The polygon sets are built in spawned worker processes meanwhile.
--impl reference times the CPU oracle (hierarchical box filter + exact
crossing test, all host cores) on bounded samples of the same workload.
Other modes: --mode batched | serve | national (one workload each).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "point→block projections/s"
UNIT = "projections/s"
BYTES_PER_POINT = 20  # 16 B of float64 lon/lat read + 4 B of int32 id written


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="state", choices=["state", "tiny"])
    ap.add_argument("--points", type=int, default=0, help="override the point count")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--opts", default="", help="build options, e.g. cell_log2=15,max_depth=3")
    ap.add_argument("--mode", default="plain", choices=["plain", "batched", "serve", "national"],
                    help="plain: state-scale join (default); batched: 4096 queries over 8 sets in one "
                         "graph launch vs per-query launches; serve: Poisson arrivals over 3 resident "
                         "sets, p50/p99 vs per-request launches; national: 1e9 points streamed from "
                         "pinned host memory")
    ap.add_argument("--tune", action="store_true", help="run the autotuner on a sample first")
    ap.add_argument("--requests", type=int, default=20000, help="serve: requests per offered load")
    ap.add_argument("--queries", type=int, default=0, help="batched: use only the first N queries")
    ap.add_argument("--loads", default="1e8,2e8,5e8,1e9", help="serve: offered loads in points/s")
    ap.add_argument("--no-batched", action="store_true", help="plain mode: skip the batched leg")
    ap.add_argument("--no-serve", action="store_true", help="plain mode: skip the serving leg")
    ap.add_argument("--serve-load", type=float, default=5e8, help="plain mode: the serving leg's offered load")
    ap.add_argument("--serve-requests", type=int, default=3000, help="plain mode: the serving leg's requests")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(cfg, rank, n_override, ps=None):
    from synth import configs
    if cfg == "tiny":
        ps = configs.tiny_set()
        n = n_override or 1_000_000
        lon, lat = configs.tiny_points(ps, n=n, seed=configs.SEEDS["tiny"] + rank)
        desc = f"tiny plain join: {ps.n_poly} Voronoi blocks over 1x1 deg, {n:.0e} uniform lattice points (+1% outside)"
    else:
        ps = ps if ps is not None else configs.state_set()
        n = n_override or 100_000_000
        lon, lat = configs.state_points(n=n, stream=1 + rank)
        desc = (f"state-scale plain join: {ps.n_poly} blocks (40 counties, ~5,000 tracts) over 5x5 deg, "
                f"{n:.0e} float64 points from a 64-Gaussian mixture + 10% uniform")
    return ps, lon, lat, n, desc


class ClockSampler:
    """nvidia-smi samples every 200 ms while running (clocks and throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


_ALL_CPUS = None  # the process's CPUs before bind_host_to_gpu


def bind_host_to_gpu(device: int):
    """Run this process on the CPUs next to the GPU (its PCI device's
    local_cpulist), so pinned host buffers are first touched in the GPU's
    NUMA node and host-to-device copies do not cross sockets. Returns the
    CPU list used, or None when it cannot be determined."""
    try:
        import torch
        p = torch.cuda.get_device_properties(device)
        bus = getattr(p, "pci_bus_id", None)
        dom = getattr(p, "pci_domain_id", 0) or 0
        dev = getattr(p, "pci_device_id", 0) or 0
        if bus is None:
            return None
        path = f"/sys/bus/pci/devices/{dom:04x}:{bus:02x}:{dev:02x}.0/local_cpulist"
        spec = open(path).read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        global _ALL_CPUS
        _ALL_CPUS = os.sched_getaffinity(0)
        cpus &= _ALL_CPUS
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return spec
    except Exception:
        return None


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2005_03156_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f in ("kernels.cuh", "pip_internal.cuh", "project.cu", "index.cu"):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


TRAFFIC_JSON = os.path.join(ROOT, "profiles", "k1_classify_state.json")


def recorded_traffic(points):
    """DRAM bytes (read + write) per K1 launch from the committed summary of
    one ncu capture of K1 on the state workload, scaled to `points` (the
    bytes per point do not depend on the point count: one pass over the
    points against the same index), when the capture was taken on the
    current kernel sources; else None."""
    try:
        with open(TRAFFIC_JSON) as f:
            rec = json.load(f)
        if rec.get("source_hash") != kernel_source_hash():
            return None
        return float(rec["dram_bytes_per_point"]) * points
    except (OSError, KeyError, ValueError):
        return None


def cpu_baseline(ps, lon, lat, budget_s=12.0):
    """The oracle's hierarchical join on this host's cores, on a bounded
    sample of the same points (sized for ~budget_s seconds)."""
    import numpy as np
    import oracle
    if _ALL_CPUS:
        os.sched_setaffinity(0, _ALL_CPUS)  # the oracle gets every host core
    cores = os.cpu_count() or 1
    H = oracle.Hier(ps, threads=cores)  # hierarchy prepared once, outside the timing
    t = time.perf_counter()
    H.join(lon[:200_000], lat[:200_000])
    rate = 200_000 / (time.perf_counter() - t)
    m = int(min(len(lon), max(200_000, rate * budget_s)))
    t = time.perf_counter()
    H.join(lon[:m], lat[:m])
    dt = time.perf_counter() - t
    t = time.perf_counter()
    m1 = 100_000
    H.join(lon[:m1], lat[:m1], threads=1)
    dt1 = time.perf_counter() - t
    del np
    return {"value": m / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {m} of the {len(lon)} workload points, all {cores} host threads; "
                      f"single-thread rate {m1 / dt1:.4g}/s on {m1} points",
            "single_thread": m1 / dt1}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    ps, lon, lat, n, desc = workload(args.config, 0, args.points)
    cores = os.cpu_count() or 1
    sample = min(4_000_000, n)  # points per step: a bounded sample of the workload
    H = oracle.Hier(ps, threads=cores)  # the oracle's box hierarchy, prepared once
    for i in range(args.warmup):
        a = (i * sample) % max(1, n - sample + 1)
        H.join(lon[a:a + sample], lat[a:a + sample])
    times = []
    for i in range(args.steps):
        a = ((args.warmup + i) * sample) % max(1, n - sample + 1)
        t = time.perf_counter()
        H.join(lon[a:a + sample], lat[a:a + sample])
        times.append(time.perf_counter() - t)
    tot = sum(times)
    value = sample * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": desc, "step": f"{sample} points per step (bounded sample)",
                   "oracle": "hierarchical closed-box filter + exact crossing test (C++)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} points per step x {args.steps} steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    # the batched and serving legs run at N=1 on the default workload; their
    # polygon sets are built in worker processes while this one works
    legs = ws == 1 and args.config == "state" and not args.points
    do_batched, do_serve = legs and not args.no_batched, legs and not args.no_serve
    jobs = [("state", SERVE_SEEDS[0])] if ws == 1 and args.config == "state" else []
    jobs += [("state", sd) for sd in SERVE_SEEDS[1:]] if do_serve else []
    jobs += BATCHED_JOBS if do_batched else []
    ex, futs = start_generation(jobs) if jobs else (None, {})
    torch.cuda.set_device(local)
    host_cpus = bind_host_to_gpu(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2005_03156_gb300 import build as pbuild
    pbuild.build()
    import paper_2005_03156_gb300 as pipm

    pre = futs[("state", SERVE_SEEDS[0])].result() if ("state", SERVE_SEEDS[0]) in futs else None
    ps, lon, lat, n, desc = workload(args.config, rank, args.points, ps=pre)
    opts = {}
    for kv in filter(None, args.opts.split(",")):
        k, v = kv.split("=")
        opts[k] = int(v)
    s = pipm.load_polygon_set(ps, opts=opts or None)
    info = s.info()
    dlon = torch.from_numpy(lon).cuda()
    dlat = torch.from_numpy(lat).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        pipm.pip_project(s, dlon, dlat, out)
    pipm.pip_set_check(s)
    _, pstats = pipm.pip_project_ex(s, dlon, dlat, out)
    torch.cuda.synchronize()

    pipm.pip_profile_enable(s, args.steps)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    l0 = pipm.pip_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        pipm.pip_project(s, dlon, dlat, out)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = pipm.pip_kernel_launches() - l0
    clk = clocks.stop()
    barrier()
    from paper_2005_03156_gb300.shard import max_over_ranks
    ms = max_over_ranks(ev0.elapsed_time(ev1), device="cuda")
    prof = pipm.pip_profile_read(s, args.steps)
    pipm.pip_profile_enable(s, 0)
    pipm.pip_set_check(s)
    ms_step = ms / args.steps
    value = n * ws * args.steps / (ms / 1e3)
    k1 = float(np.mean(prof["k1_ms"])) if len(prof["k1_ms"]) else float("nan")
    bn = float(np.mean(prof["bin_ms"])) if len(prof["bin_ms"]) else float("nan")
    k3 = float(np.mean(prof["k3_ms"])) if len(prof["k3_ms"]) else float("nan")
    peak, peak_kind = measured_peak()
    achieved = BYTES_PER_POINT * n / (k1 / 1e3) / 1e9
    # the recorded traffic is for the default index of the state workload
    traffic = recorded_traffic(n) if (not opts and args.config == "state") else None

    e2e = None
    if not args.no_e2e:
        hl = torch.from_numpy(lon).pin_memory()
        ha = torch.from_numpy(lat).pin_memory()
        ho = torch.empty(n, dtype=torch.int32).pin_memory()
        k_e2e = max(2, min(args.steps, 5))
        pipm.pip_project(s, hl, ha, ho)  # warm
        barrier()
        t = time.perf_counter()
        for _ in range(k_e2e):
            pipm.pip_project(s, hl, ha, ho)
        dt = max_over_ranks(time.perf_counter() - t, device="cuda")
        e2e = {"value": n * ws * k_e2e / dt, "unit": UNIT, "h2d_bytes_per_step": 16 * n,
               "d2h_bytes_per_step": 4 * n, "steps": k_e2e,
               "path": "pip_project with pinned host lon/lat/out: chunked H2D / compute / D2H on 2 streams"}
        del hl, ha, ho

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(ps, lon, lat)

    # the batched and serving legs (the metric's other two parts), on the
    # same GPU after the plain join's buffers are released
    batched = serve = None
    if do_batched or do_serve:
        del dlon, dlat, out
        s.free()
        torch.cuda.empty_cache()
    if do_batched:
        bsets = [futs[j].result() for j in BATCHED_JOBS]
        batched = batched_leg(pipm, bsets, steps=5, warmup=2)
        del bsets
    if do_serve:
        ssets = [ps] + [futs[("state", sd)].result() for sd in SERVE_SEEDS[1:]]
        serve = serve_leg(pipm, ssets, [args.serve_load], args.serve_requests)
    if ex is not None:
        ex.shutdown()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"host_cpus": host_cpus, "workload": desc, "points_per_gpu": n, "polygons": ps.n_poly,
                       "vertices": ps.n_vert, "l2": "inputs larger than L2 (1.6 GB of points per step vs 129 MB L2)",
                       "parallelism": f"replicas x{ws} (points sharded, set replicated)",
                       "index": {k: info[k] for k in ("cell_log2", "fanout_log2", "depth", "leaves",
                                                      "interior_cells", "superbins", "index_bytes",
                                                      "build_ms", "table_entries")},
                       "residual_fraction": pstats["residual"] / n, "build_opts": opts or "default"},
            "roofline": {"bound": "hbm", "kernel": "k_classify_dq (K1)", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json copy bandwidth)",
                         "bytes_per_launch": BYTES_PER_POINT * n,
                         "step": {"achieved": BYTES_PER_POINT * n / (ms_step / 1e3) / 1e9,
                                  "frac": BYTES_PER_POINT * n / (ms_step / 1e3) / 1e9 / peak,
                                  "note": "the whole projection (K1, K3 and, when binning is on, K2) against the same 20 B/point"}},
            "stages_ms": {"k1_classify": k1, "k2_bin": bn, "k3_cross": k3},
            "e2e": e2e, "gpu_launches": launches, "clocks": clk, "cpu_baseline": cpu,
        }
        if batched is not None:
            line["batched"] = batched
            line["config"]["batched"] = batched["workload"] + ", 5 timed graph launches after 2 warm-up"
        if serve is not None:
            r = serve["loads"][0]
            line["serve"] = {"offered_pts_s": r["served"]["offered_pts_s"], "requests": args.serve_requests,
                             "served": r["served"], "plain_per_request": r["plain_per_request"],
                             "served_equals_plain": r["served_equals_plain"], "clocks": serve["clocks"]}
            line["config"]["serve"] = serve["workload"]
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _opts_arg(args):
    opts = {}
    for kv in filter(None, args.opts.split(",")):
        k, v = kv.split("=")
        opts[k] = int(v)
    return opts or None


def _gen_set(kind, arg):
    """One polygon set, built in a worker process (picklable result)."""
    from synth import configs
    if kind == "state":
        return configs.state_set(seed=arg)
    return configs.batched_set(arg)


def start_generation(jobs):
    """Build polygon sets in spawned worker processes, started before any
    CUDA call (spawn, not fork: the workers hold no CUDA state)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    ex = cf.ProcessPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1)),
                                mp_context=mp.get_context("spawn"))
    return ex, {job: ex.submit(_gen_set, *job) for job in jobs}


BATCHED_JOBS = [("batched", k) for k in range(8)]
SERVE_SEEDS = (2, 6, 7)  # the state seed and two more: 3 resident state-scale sets


def batched_leg(pipm, psets, steps, warmup, opts=None, n_queries=0, tune=False):
    """4096 lognormal queries (100..1e6 points, mean ~5e4) over the 8
    resident sets: one persistent graph launch per step against the same
    queries as separate plain launches (3 rounds)."""
    import numpy as np
    import torch
    from synth import configs
    t0 = time.perf_counter()
    sizes, sigma = configs.batched_query_sizes()
    rng = np.random.Generator(np.random.PCG64([configs.SEEDS["batched"], 600]))
    set_of = rng.integers(0, len(psets), len(sizes))
    if n_queries:  # the first queries only (small cases for profiling)
        sizes, set_of = sizes[:n_queries], set_of[:n_queries]
    n_total = int(sizes.sum())
    sets = [pipm.load_polygon_set(p, opts=opts) for p in psets]
    # points: each set's mixture, one block of points per set, queries slice it
    per_set = [int(sizes[set_of == k].sum()) + 2 * int((set_of == k).sum()) for k in range(len(psets))]
    pts = []
    for k, p in enumerate(psets):
        lon, lat = p.meta["mixture"].sample_degrees(max(1, per_set[k]),
                                                    np.random.Generator(np.random.PCG64([configs.SEEDS["batched"], 700 + k])))
        pts.append((torch.from_numpy(lon).cuda(), torch.from_numpy(lat).cuda()))
    gen_s = time.perf_counter() - t0
    if tune:
        for k, s in enumerate(sets):
            m = min(5_000_000, per_set[k])
            if m > 0:
                pipm.pip_set_tune(s, pts[k][0][:m], pts[k][1][:m])
    used = [0] * len(psets)
    qs, outs = [], []
    for i, n in enumerate(sizes):
        k = int(set_of[i])
        a = used[k]
        used[k] += int(n)
        used[k] = min(per_set[k], (used[k] + 1) // 2 * 2)  # queries start 16-byte aligned
        out = torch.empty(int(n), dtype=torch.int32, device="cuda")
        qs.append((sets[k], pts[k][0][a:a + n], pts[k][1][a:a + n], out))
        outs.append(out)
    # the query list marshalled once (as a C caller keeps its pip_query array):
    # rebuilding it in Python costs ~8 ms a run for 4,096 queries, more than
    # the launch itself
    prepared = pipm.Queries(qs)
    plan = pipm.Plan(max_points=n_total, max_queries=len(qs))
    knobs = plan.tune(prepared)
    for _ in range(warmup):
        plan.run(prepared)
    plan.check()
    stream = torch.cuda.current_stream()
    l0 = pipm.pip_kernel_launches()
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.run(prepared)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    batched_ms = e0.elapsed_time(e1) / steps
    batched_launches = (pipm.pip_kernel_launches() - l0) / steps
    plan.check()
    got = [o.clone() for o in outs]
    # the same queries as separate plain launches
    for q in qs[:64]:
        pipm.pip_project(q[0], q[1], q[2], q[3])
    torch.cuda.synchronize()
    plain_steps = max(1, min(3, steps))
    l0 = pipm.pip_kernel_launches()
    e0.record(stream)
    for _ in range(plain_steps):
        for q in qs:
            pipm.pip_project(q[0], q[1], q[2], q[3])
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / plain_steps
    plain_launches = (pipm.pip_kernel_launches() - l0) / plain_steps
    equal = all(torch.equal(a, b) for a, b in zip(got, outs))
    for s in sets:
        s.free()
    del pts, qs, outs, got
    torch.cuda.empty_cache()
    return {
        "value": n_total / (batched_ms / 1e3), "unit": UNIT, "ms_per_step": batched_ms, "steps": steps,
        "warmup": warmup, "gpu_launches": batched_launches,
        "workload": f"batched: {len(sizes)} queries (lognormal, sigma {sigma:.2f}, 100..1e6, mean "
                    f"{sizes.mean():.0f}) over 8 sets of {min(p.n_poly for p in psets)}.."
                    f"{max(p.n_poly for p in psets)} blocks, {n_total} points",
        "points": n_total, "plan": knobs, "generation_s": gen_s, "tuned_sets": bool(tune),
        "plain_per_query": {"value": n_total / (plain_ms / 1e3), "ms_per_step": plain_ms,
                            "gpu_launches": plain_launches, "rounds": plain_steps},
        "speedup_vs_plain": plain_ms / batched_ms, "batched_equals_plain": equal, "clocks": clk,
    }


def run_batched(args):
    """The batched workload alone (see batched_leg)."""
    import torch
    ex, futs = start_generation(BATCHED_JOBS)
    from paper_2005_03156_gb300 import build as pbuild
    pbuild.build()
    import paper_2005_03156_gb300 as pipm
    torch.cuda.set_device(0)
    host_cpus = bind_host_to_gpu(0)
    psets = [futs[j].result() for j in BATCHED_JOBS]
    ex.shutdown()
    leg = batched_leg(pipm, psets, args.steps, args.warmup, opts=_opts_arg(args), n_queries=args.queries,
                      tune=args.tune)
    line = {
        "metric": METRIC + " (batched)", "value": leg["value"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": leg["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"host_cpus": host_cpus, "workload": leg["workload"], "plan": leg["plan"],
                   "generation_s": leg["generation_s"], "tuned_sets": leg["tuned_sets"]},
        "plain_per_query": leg["plain_per_query"], "speedup_vs_plain": leg["speedup_vs_plain"],
        "batched_equals_plain": leg["batched_equals_plain"], "gpu_launches": leg["gpu_launches"],
        "clocks": leg["clocks"],
    }
    print(json.dumps(line))


def serve_leg(pipm, psets, loads, nreq):
    """Poisson arrivals at each offered load, request sizes log-uniform in
    [1, 1e6], uniform over the resident state-scale sets: the continuous-
    batching server against per-request plain launches (pinned host buffers)."""
    import numpy as np
    import torch
    from synth import configs
    sets = [pipm.load_polygon_set(p) for p in psets]
    pool_n = 20_000_000
    pools = []
    for sd in SERVE_SEEDS[:len(psets)]:
        lon, lat = configs.state_points(n=pool_n, seed=sd, stream=9)
        pools.append((torch.from_numpy(lon).pin_memory(), torch.from_numpy(lat).pin_memory()))
    results = []
    clocks = ClockSampler(0)
    clocks.start()
    for load in loads:
        rng = np.random.Generator(np.random.PCG64([configs.SEEDS["serve"], int(load) % 100003]))
        sizes = np.exp(rng.uniform(0, np.log(1e6), nreq)).astype(np.int64)
        sizes = np.maximum(1, sizes)
        mean = sizes.mean()
        gaps = rng.exponential(mean / load, nreq)
        arrive = np.cumsum(gaps)
        which = rng.integers(0, len(sets), nreq)
        offs = rng.integers(0, pool_n - 1_000_000, nreq)
        outs = [torch.empty(int(n), dtype=torch.int32).pin_memory() for n in sizes]

        def req(i):
            k, a, n = int(which[i]), int(offs[i]), int(sizes[i])
            return k, pools[k][0][a:a + n], pools[k][1][a:a + n], outs[i]

        # served: submit on schedule, collect completions
        srv = pipm.Server(sets, dict(n_streams=3, max_batch_points=1 << 23, max_batch_queries=1024))
        for w in range(4):  # warm-up: 12 requests at once, so every slot runs
            tw = [srv.submit(*req(j)) for j in range(12)]
            for t in tw:
                srv.wait(t)
        srv.stats(reset=True)
        tickets = [0] * nreq
        t0 = time.perf_counter()
        for i in range(nreq):
            while time.perf_counter() - t0 < arrive[i]:
                pass
            k, lon, lat, out = req(i)
            tickets[i] = srv.submit(k, lon, lat, out)
        for t in tickets:
            srv.wait(t)
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        served_ids = [o.clone() for o in outs]
        served = {"offered_pts_s": load, "p50_us": st["p50_us"], "p99_us": st["p99_us"],
                  "sustained_pts_s": float(sizes.sum()) / wall, "launches": st["launches"],
                  "mean_batch_queries": st["mean_batch_queries"], "requests": nreq,
                  "points": int(sizes.sum())}
        # per-request plain launches, in arrival order (a request starts when
        # it has arrived and the previous one is done)
        lat_us = np.zeros(nreq)
        t0 = time.perf_counter()
        for i in range(nreq):
            while time.perf_counter() - t0 < arrive[i]:
                pass
            k, lon, lat, out = req(i)
            pipm.pip_project(sets[k], lon, lat, out)
            lat_us[i] = (time.perf_counter() - t0 - arrive[i]) * 1e6
        wall_p = time.perf_counter() - t0
        plain = {"p50_us": float(np.percentile(lat_us, 50)), "p99_us": float(np.percentile(lat_us, 99)),
                 "sustained_pts_s": float(sizes.sum()) / wall_p}
        equal = all(torch.equal(a, b) for a, b in zip(served_ids, outs))
        results.append({"served": served, "plain_per_request": plain, "served_equals_plain": equal})
        print(json.dumps({"load": load, **results[-1]}), file=sys.stderr, flush=True)
    clk = clocks.stop()
    for s in sets:
        s.free()
    return {"loads": results, "clocks": clk,
            "workload": f"serving: Poisson arrivals, sizes log-uniform [1, 1e6], {len(sets)} resident "
                        f"state-scale sets (seeds {', '.join(str(x) for x in SERVE_SEEDS[:len(sets)])}), "
                        f"pinned host buffers, {nreq} requests per offered load"}


def run_serve(args):
    """The serving workload alone (see serve_leg)."""
    import torch
    jobs = [("state", sd) for sd in SERVE_SEEDS]
    ex, futs = start_generation(jobs)
    from paper_2005_03156_gb300 import build as pbuild
    pbuild.build()
    import paper_2005_03156_gb300 as pipm
    torch.cuda.set_device(0)
    host_cpus = bind_host_to_gpu(0)
    psets = [futs[j].result() for j in jobs]
    ex.shutdown()
    loads = [float(x) for x in args.loads.split(",")]
    leg = serve_leg(pipm, psets, loads, args.requests)
    best = max(leg["loads"], key=lambda r: r["served"]["sustained_pts_s"])
    line = {
        "metric": "p50/p99 serve latency and sustained " + METRIC, "value": best["served"]["sustained_pts_s"],
        "unit": UNIT, "n_gpus": 1, "steps": len(loads), "warmup": 0, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"host_cpus": host_cpus, "workload": leg["workload"], "requests_per_load": args.requests},
        "loads": leg["loads"], "clocks": leg["clocks"],
    }
    print(json.dumps(line))


def _national_chunk(a):
    from synth import configs
    return configs.national_points_chunk(*a)


def run_national(args):
    """1e9 mixture points over 50 regions (800,000 blocks) streamed from
    pinned host memory in 1e8-point chunks through pip_project."""
    import numpy as np
    import torch
    from synth import configs
    from paper_2005_03156_gb300 import build as pbuild
    pbuild.build()
    import paper_2005_03156_gb300 as pipm
    torch.cuda.set_device(0)
    host_cpus = bind_host_to_gpu(0)
    t0 = time.perf_counter()
    ps = configs.national_set()
    s = pipm.load_polygon_set(ps, opts=_opts_arg(args))
    gen_set = time.perf_counter() - t0
    chunk = 100_000_000
    n_chunks = max(1, (args.points or 1_000_000_000) // chunk)
    npts = configs.NationalPoints()
    lon_h = torch.empty(n_chunks * chunk, dtype=torch.float64).pin_memory()
    lat_h = torch.empty(n_chunks * chunk, dtype=torch.float64).pin_memory()
    out_h = torch.empty(n_chunks * chunk, dtype=torch.int32).pin_memory()
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(n_chunks, max(1, (os.cpu_count() or 2) // 2))) as pool:
        for c, (lon, lat) in enumerate(pool.imap(_national_chunk, [(c, chunk) for c in range(n_chunks)])):
            lon_h[c * chunk:(c + 1) * chunk] = torch.from_numpy(lon)
            lat_h[c * chunk:(c + 1) * chunk] = torch.from_numpy(lat)
    del npts
    gen_pts = time.perf_counter() - t0 - gen_set
    # pinned H2D bandwidth probe (after a warm copy: first touches of pinned
    # pages are slower), best of 5
    dbuf = torch.empty(chunk, dtype=torch.float64, device="cuda")
    dbuf.copy_(lon_h[:chunk], non_blocking=True)
    torch.cuda.synchronize()
    best = 1e9
    for _ in range(5):
        t = time.perf_counter()
        dbuf.copy_(lon_h[:chunk], non_blocking=True)
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t)
    h2d_gbs = chunk * 8 / best / 1e9
    del dbuf
    for _ in range(max(1, args.warmup)):  # warm: touches every pinned page; early host-to-device
        pipm.pip_project(s, lon_h, lat_h, out_h)  # copies after a large index build ran slower
    clocks = ClockSampler(0)
    clocks.start()
    t = time.perf_counter()
    steps = max(1, args.steps)
    step_ms = []
    for _ in range(steps):
        t1 = time.perf_counter()
        pipm.pip_project(s, lon_h, lat_h, out_h)
        step_ms.append((time.perf_counter() - t1) * 1e3)
    dt = (time.perf_counter() - t) / steps
    clk = clocks.stop()
    # device-resident time of one chunk, by stage (what the stream hides behind the copies)
    dl = lon_h[:chunk].cuda()
    da = lat_h[:chunk].cuda()
    do = torch.empty(chunk, dtype=torch.int32, device="cuda")
    pipm.pip_project(s, dl, da, do)
    pipm.pip_profile_enable(s, 3)
    for _ in range(3):
        pipm.pip_project(s, dl, da, do)
    torch.cuda.synchronize()
    prof = pipm.pip_profile_read(s, 3)
    pipm.pip_profile_enable(s, 0)
    chunk_stages = {"k1_classify": float(np.mean(prof["k1_ms"])), "k2_bin": float(np.mean(prof["bin_ms"])),
                    "k3_cross": float(np.mean(prof["k3_ms"]))}
    del dl, da, do
    n = n_chunks * chunk
    idx = np.random.default_rng(5).choice(n, 100_000, replace=False)
    import oracle
    want = oracle.join_hier(ps, lon_h.numpy()[idx], lat_h.numpy()[idx])
    ok = bool((out_h.numpy()[idx] == want).all())
    bound = min(6773.2, h2d_gbs) * 1e9 / 16
    line = {
        "metric": METRIC + " (national, streamed from pinned host)", "value": n / dt, "unit": UNIT,
        "n_gpus": 1, "steps": steps, "warmup": max(1, args.warmup), "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"host_cpus": host_cpus, "workload": f"national: {ps.n_poly} blocks in 50 regions, {n:.0e} points in "
                               f"{n_chunks} chunks of 1e8 from pinned host memory",
                   "index": {k: s.info()[k] for k in ("cell_log2", "depth", "leaves", "index_bytes", "build_ms")},
                   "generation_s": {"set": gen_set, "points": gen_pts}},
        "h2d_gbs": h2d_gbs, "bound_pts_s": bound, "frac_of_bound": (n / dt) / bound,
        "sampled_parity_100k": ok, "clocks": clk, "device_chunk_stages_ms": chunk_stages,
        "step_ms": {"min": min(step_ms), "median": float(np.median(step_ms)), "max": max(step_ms)},
        "median_step_pts_s": n / (float(np.median(step_ms)) / 1e3),
    }
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "batched":
        run_batched(args)
    elif args.mode == "serve":
        run_serve(args)
    elif args.mode == "national":
        run_national(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
