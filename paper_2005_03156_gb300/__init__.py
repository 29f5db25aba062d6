"""GB300 census-block point-in-polygon join (Kepner et al., "Fast Mapping onto
Census Blocks"): Python binding of libpip.so.

The functions below carry the C ABI's names (include/pip.h) and only
marshal arguments: tensors become device pointers, the current torch stream
becomes the cudaStream_t. Every step of the join runs in the library's CUDA
kernels; there is no CPU path.

  pip_set_load_i32 / pip_set_load_f64   load a polygon set, build its index
  pip_project / pip_project_ex          points -> int32 block ids (-1 outside)
  pip_project_batch, pip_plan_*         many queries in one graph launch
  pip_set_tune                          autotuner (cell size, points/CTA, stages)
  pip_server_*                          continuous-batching serving loop
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import BuildOpts, PipError, ProjectStats, Query, ServerOpts, ServerStats, SetInfo

__all__ = [
    "PipError", "BuildOpts", "PolygonSet", "pip_set_load_i32", "pip_set_load_f64", "pip_project",
    "pip_project_ex", "pip_quantize", "pip_set_info", "pip_set_rebuild", "pip_set_free",
    "pip_set_check", "pip_set_top_candidates", "pip_project_batch", "Plan", "pip_set_tune",
    "Server", "lib", "pip_locate", "Queries",
]


def lib():
    return _native.load()


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(x):
    """Device or host pointer of a tensor / numpy array (kept alive by caller)."""
    if x is None:
        return ctypes.c_void_p(0)
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())


def _opts(opts):
    if opts is None:
        return None
    if isinstance(opts, BuildOpts):
        return opts
    o = BuildOpts()
    for k, v in dict(opts).items():
        setattr(o, k, int(v))
    return o


class PolygonSet:
    """Handle of a loaded set (owns the library's device memory)."""

    def __init__(self, handle):
        self.handle = ctypes.c_void_p(handle)

    def info(self) -> dict:
        return pip_set_info(self)

    def free(self):
        if self.handle and self.handle.value:
            _native.check(lib().pip_set_free(self.handle))
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _load(fn, vx, vy, ring_off, poly_ring_off, parents, opts, stream, allocator=None):
    ring_off = np.ascontiguousarray(ring_off, np.int64) if isinstance(ring_off, np.ndarray) else ring_off
    poly_ring_off = (np.ascontiguousarray(poly_ring_off, np.int64)
                     if isinstance(poly_ring_off, np.ndarray) else poly_ring_off)
    parents = list(parents or [])
    parents = [np.ascontiguousarray(p, np.int32) if isinstance(p, np.ndarray) else p for p in parents]
    par_arr = (ctypes.c_void_p * max(1, len(parents)))(*[_ptr(p).value for p in parents]) if parents else None
    handle = ctypes.c_void_p(0)
    o = _opts(opts)
    st = fn(_ptr(vx), _ptr(vy), int(len(vx)), _ptr(ring_off), int(len(ring_off) - 1), _ptr(poly_ring_off),
            int(len(poly_ring_off) - 1), par_arr, len(parents), ctypes.byref(o) if o else None,
            ctypes.byref(allocator) if allocator is not None else None, _stream(stream),
            ctypes.byref(handle))
    _native.check(st)
    ps = PolygonSet(handle.value)
    ps._allocator = allocator  # the set calls it until freed
    return ps


def pip_set_load_i32(vx, vy, ring_off, poly_ring_off, parents=None, opts=None, stream=None,
                     allocator=None) -> PolygonSet:
    """Load int32 lattice vertices (numpy host arrays or torch tensors).
    allocator: optional _native.Allocator (device memory hook)."""
    if isinstance(vx, np.ndarray):
        vx = np.ascontiguousarray(vx, np.int32)
        vy = np.ascontiguousarray(vy, np.int32)
    return _load(lib().pip_set_load_i32, vx, vy, ring_off, poly_ring_off, parents, opts, stream, allocator)


def pip_set_load_f64(vx, vy, ring_off, poly_ring_off, parents=None, opts=None, stream=None) -> PolygonSet:
    """Load double vertices in degrees (quantized by Q on the device)."""
    if isinstance(vx, np.ndarray):
        vx = np.ascontiguousarray(vx, np.float64)
        vy = np.ascontiguousarray(vy, np.float64)
    return _load(lib().pip_set_load_f64, vx, vy, ring_off, poly_ring_off, parents, opts, stream)


def load_polygon_set(pset, opts=None, stream=None, allocator=None) -> PolygonSet:
    """Load a synth.PolygonSet-like object (vx, vy, ring_off, poly_ring_off, parents)."""
    return pip_set_load_i32(pset.vx, pset.vy, pset.ring_off, pset.poly_ring_off,
                            parents=getattr(pset, "parents", None), opts=opts, stream=stream,
                            allocator=allocator)


def pip_set_info(s: PolygonSet) -> dict:
    info = SetInfo()
    _native.check(lib().pip_set_info(s.handle, ctypes.byref(info)))
    d = {k: getattr(info, k) for k, _ in SetInfo._fields_}
    d["compact_by_edges"] = list(d["compact_by_edges"])
    d["nodes_by_level"] = list(d["nodes_by_level"])
    return d


LOC_KINDS = {0: "empty", 1: "interior", 2: "residual", 3: "compact", 4: "outside"}


def pip_locate(s: PolygonSet, qx, qy, stream=None):
    """Kind (bits 0-7) and trie depth (bits 8-15) of the index cell that
    answers each lattice point (int32 device tensors); see LOC_KINDS."""
    import torch
    code = torch.empty(int(qx.shape[0]), dtype=torch.int32, device=qx.device)
    _native.check(lib().pip_locate(s.handle, _ptr(qx), _ptr(qy), int(qx.shape[0]), _ptr(code), _stream(stream)))
    return code


def pip_set_rebuild(s: PolygonSet, opts=None, stream=None):
    o = _opts(opts)
    _native.check(lib().pip_set_rebuild(s.handle, ctypes.byref(o) if o else None, _stream(stream)))


def pip_set_free(s: PolygonSet):
    s.free()


def pip_set_check(s: PolygonSet, stream=None):
    _native.check(lib().pip_set_check(s.handle, _stream(stream)))


def pip_project(s: PolygonSet, lon, lat, out=None, stream=None):
    """out[i] = block id of (lon[i], lat[i]) (-1 outside). Device tensors:
    asynchronous on the stream; host arrays (numpy / CPU tensors): streamed
    through the device, returns when out is written."""
    import torch
    n = int(lon.shape[0])
    if out is None:
        if isinstance(lon, np.ndarray):
            out = np.empty(n, np.int32)
        else:
            out = torch.empty(n, dtype=torch.int32, device=lon.device)
    _native.check(lib().pip_project(s.handle, _ptr(lon), _ptr(lat), n, _ptr(out), _stream(stream)))
    return out


def pip_project_ex(s: PolygonSet, lon, lat, out=None, stream=None):
    """pip_project plus counters (synchronises the stream)."""
    import torch
    n = int(lon.shape[0])
    if out is None:
        if isinstance(lon, np.ndarray):
            out = np.empty(n, np.int32)
        else:
            out = torch.empty(n, dtype=torch.int32, device=lon.device)
    st = ProjectStats()
    _native.check(lib().pip_project_ex(s.handle, _ptr(lon), _ptr(lat), n, _ptr(out), _stream(stream),
                                       ctypes.byref(st)))
    return out, {"n": st.n, "residual": st.residual, "items": st.items}


def pip_project_noalloc(s: PolygonSet, lon, lat, out, stream=None):
    """pip_project without any device allocation (device tensors; at most
    262144 points; the scratch is a fixed array inside the library shared by
    all calls, so calls must not overlap on the GPU)."""
    _native.check(lib().pip_project_noalloc(s.handle, _ptr(lon), _ptr(lat), int(lon.shape[0]), _ptr(out),
                                            _stream(stream)))
    return out


def pip_parent_ids(s: PolygonSet, ids, level: int, stream=None):
    """Level-`level` ancestors of block ids (1 = tract, 2 = county, ...)."""
    import torch
    out = torch.empty_like(ids)
    _native.check(lib().pip_parent_ids(s.handle, _ptr(ids), int(ids.shape[0]), int(level), _ptr(out),
                                       _stream(stream)))
    return out


def pip_quantize(v, stream=None):
    """Device quantizer Q (diagnostic): returns (q int32, valid uint8) tensors."""
    import torch
    q = torch.empty(v.shape[0], dtype=torch.int32, device=v.device)
    ok = torch.empty(v.shape[0], dtype=torch.uint8, device=v.device)
    _native.check(lib().pip_quantize(_ptr(v), int(v.shape[0]), _ptr(q), _ptr(ok), _stream(stream)))
    return q, ok


def pip_selftest_bounded_wait(limit_ns: int, stream=None) -> int:
    """Run the bounded-wait failure path once (diagnostic): returns the
    status code, PIP_ETIMEOUT (5) when the wait ran out as designed."""
    return int(lib().pip_selftest_bounded_wait(int(limit_ns), _stream(stream)))


def pip_set_top_candidates(s: PolygonSet, mode: int):
    info = pip_set_info(s)
    cells = int(info["grid_nx"] * info["grid_ny"])
    off = np.zeros(cells + 1, np.int64)
    st = lib().pip_set_top_candidates(s.handle, mode, _ptr(off), None, 0)
    need = int(off[-1])
    ids = np.zeros(max(1, need), np.int32)
    _native.check(lib().pip_set_top_candidates(s.handle, mode, _ptr(off), _ptr(ids), need))
    del st
    return off, ids[:need]


def _queries(qs):
    arr = (Query * len(qs))()
    keep = []
    for i, (s, lon, lat, out) in enumerate(qs):
        arr[i].set = s.handle
        arr[i].lon = _ptr(lon)
        arr[i].lat = _ptr(lat)
        arr[i].n = int(lon.shape[0])
        arr[i].out = _ptr(out)
        keep.append((lon, lat, out))
    return arr, keep


class Queries:
    """A query list marshalled once into the C ABI's pip_query array, for
    runs that repeat it: building the array from Python costs about 2 us a
    query, more than a batched launch's kernel time per query. It keeps the
    tensors alive; their pointers must stay valid while it is used."""

    def __init__(self, qs):
        self.arr, self._keep = _queries(qs)
        self.n = len(qs)


def _marshalled(qs):
    if isinstance(qs, Queries):
        return qs.arr, qs.n, qs
    arr, keep = _queries(qs)
    return arr, len(qs), (arr, keep)


def pip_project_batch(qs, stream=None):
    """qs: list of (set, lon, lat, out) device tensors, or Queries; one launch (synchronous)."""
    arr, n, keep = _marshalled(qs)
    _native.check(lib().pip_project_batch(arr, n, _stream(stream)))


class Plan:
    """Batched launch plan: one persistent work-stealing kernel in a CUDA graph."""

    def __init__(self, max_points: int, max_queries: int, stream=None):
        h = ctypes.c_void_p(0)
        _native.check(lib().pip_plan_create(int(max_points), int(max_queries), _stream(stream),
                                            ctypes.byref(h)))
        self.handle = h

    def run(self, qs, stream=None):
        """qs: list of (set, lon, lat, out) device tensors, or a Queries built once."""
        arr, n, keep = _marshalled(qs)
        self._keep = keep
        _native.check(lib().pip_plan_run(self.handle, arr, n, _stream(stream)))

    def check(self, stream=None):
        _native.check(lib().pip_plan_check(self.handle, _stream(stream)))

    def tune(self, qs, stream=None):
        arr, n, keep = _marshalled(qs)
        ppc, st = ctypes.c_int32(0), ctypes.c_int32(0)
        _native.check(lib().pip_plan_tune(self.handle, arr, n, _stream(stream),
                                          ctypes.byref(ppc), ctypes.byref(st)))
        return {"pts_per_cta": ppc.value, "staged": st.value}

    def destroy(self):
        if self.handle and self.handle.value:
            _native.check(lib().pip_plan_destroy(self.handle))
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def pip_set_tune(s: PolygonSet, lon, lat, stream=None) -> dict:
    o = BuildOpts()
    _native.check(lib().pip_set_tune(s.handle, _ptr(lon), _ptr(lat), int(lon.shape[0]), _stream(stream),
                                     ctypes.byref(o)))
    return {k: getattr(o, k) for k, _ in BuildOpts._fields_}


class Server:
    """Continuous-batching serving loop over resident sets (host buffers)."""

    def __init__(self, sets, opts=None):
        arr = (ctypes.c_void_p * len(sets))(*[s.handle.value for s in sets])
        o = ServerOpts()
        for k, v in dict(opts or {}).items():
            setattr(o, k, int(v))
        h = ctypes.c_void_p(0)
        _native.check(lib().pip_server_create(arr, len(sets), ctypes.byref(o), ctypes.byref(h)))
        self.handle = h
        self._sets = sets

    def submit(self, set_index, lon, lat, out) -> int:
        t = ctypes.c_uint64(0)
        _native.check(lib().pip_server_submit(self.handle, int(set_index), _ptr(lon), _ptr(lat),
                                              int(lon.shape[0]), _ptr(out), ctypes.byref(t)))
        return t.value

    def try_submit(self, set_index, lon, lat, out):
        t = ctypes.c_uint64(0)
        st = lib().pip_server_submit(self.handle, int(set_index), _ptr(lon), _ptr(lat),
                                     int(lon.shape[0]), _ptr(out), ctypes.byref(t))
        return st, t.value

    def wait(self, ticket: int, timeout_us: int = -1):
        _native.check(lib().pip_server_wait(self.handle, ctypes.c_uint64(ticket), int(timeout_us)))

    def stats(self, reset: bool = False) -> dict:
        st = ServerStats()
        _native.check(lib().pip_server_stats(self.handle, ctypes.byref(st), 1 if reset else 0))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self.handle and self.handle.value:
            lib().pip_server_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pip_profile_enable(s: PolygonSet, capacity: int):
    _native.check(lib().pip_profile_enable(s.handle, int(capacity)))


def pip_profile_read(s: PolygonSet, capacity: int):
    """Per-call stage times (ms) recorded since enabling: dict of arrays."""
    k1 = np.zeros(max(1, capacity))
    bn = np.zeros(max(1, capacity))
    k3 = np.zeros(max(1, capacity))
    n = ctypes.c_int32(int(capacity))
    _native.check(lib().pip_profile_read(s.handle, _ptr(k1), _ptr(bn), _ptr(k3), ctypes.byref(n)))
    m = n.value
    return {"k1_ms": k1[:m], "bin_ms": bn[:m], "k3_ms": k3[:m]}


def pip_kernel_launches() -> int:
    return int(lib().pip_kernel_launches())
