"""Plain CPU oracle for the point-in-polygon join (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg and reference arm may import this package. The product library never loads it, and the two
share no code.

The oracle follows the paper (Kepner et al., "Fast Mapping onto Census
Blocks"): Sec. II for the data model (double lon/lat points, polygon rings,
bounding boxes in a hierarchy), Sec. III-A for the crossing-number test and
Sec. III / Appendix A for the hierarchical bounding-box filter with
lowest-index claims. The C++ source ``pip_oracle.cpp`` states the readings
taken where the paper is silent (lattice quantization Q, the half-open tie
rule, closed filter boxes, -1 for "no polygon").

Functions:
  quantize(v)            -> (q int32 array, valid bool array)      exact Q
  edge_crossing(...)     -> 0/1 for one edge and one lattice point
  inside(pset, p, x, y)  -> 0/1 crossing parity of polygon p
  join_bruteforce(...)   -> O0: every point against every polygon
  join_hier(...)         -> O1: hierarchical closed-box filter + crossing test
  count_owners_q(...)    -> number of containing polygons per lattice point
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pip_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction, plain -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = [
            "g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
            "-ffp-contract=off", "-o", tmp, _SRC,
        ]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I32 = ctypes.c_int32
    lib.orc_quantize.argtypes = [ctypes.c_double, P]
    lib.orc_quantize.restype = ctypes.c_int
    lib.orc_quantize_many.argtypes = [P, I64, P, P]
    lib.orc_quantize_many.restype = None
    lib.orc_edge_crossing.argtypes = [I32] * 6
    lib.orc_edge_crossing.restype = ctypes.c_int
    lib.orc_inside.argtypes = [P, P, P, P, I64, I64, I32, I32]
    lib.orc_inside.restype = ctypes.c_int
    lib.orc_count_owners_q.argtypes = [P, P, P, P, I64, P, P, I64, P, ctypes.c_int]
    lib.orc_count_owners_q.restype = None
    lib.orc_join_bruteforce_q.argtypes = [P, P, P, P, I64, P, P, I64, P, ctypes.c_int]
    lib.orc_join_bruteforce_q.restype = None
    lib.orc_join_bruteforce.argtypes = [P, P, P, P, I64, P, P, I64, P, ctypes.c_int]
    lib.orc_join_bruteforce.restype = None
    lib.orc_join_hier.argtypes = [P, P, P, P, I64, P, P, ctypes.c_int, P, P, I64, P, ctypes.c_int]
    lib.orc_join_hier.restype = None
    lib.orc_hier_create.argtypes = [P, P, P, P, I64, P, P, ctypes.c_int]
    lib.orc_hier_create.restype = P
    lib.orc_hier_join.argtypes = [P, P, P, I64, P, ctypes.c_int]
    lib.orc_hier_join.restype = None
    lib.orc_hier_free.argtypes = [P]
    lib.orc_hier_free.restype = None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def load_variant(source_text: str, tag: str):
    """Compile a modified copy of the oracle source (used by the tests that
    plant a mistake in the oracle to show the pins catch it). Returns an
    object with the same functions as this module."""
    import types
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_BUILD, f"variant_{tag}.cpp")
    so = os.path.join(_BUILD, f"libvariant_{tag}_{os.getpid()}.so")
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                           "-ffp-contract=off", "-o", so, src])
    lib = _bind(ctypes.CDLL(so))
    mod = types.SimpleNamespace()
    g = globals()
    for name in ("quantize", "edge_crossing", "inside", "count_owners_q",
                 "join_bruteforce_q", "join_bruteforce", "join_hier"):
        fn = g[name]
        mod.__dict__[name] = (lambda f: (lambda *a, **k: f(*a, _use=lib, **k)))(fn)
    return mod


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _poly_args(pset):
    vx = _c(pset.vx, np.int32)
    vy = _c(pset.vy, np.int32)
    ro = _c(pset.ring_off, np.int64)
    pro = _c(pset.poly_ring_off, np.int64)
    keep = (vx, vy, ro, pro)
    return keep, [_ptr(vx), _ptr(vy), _ptr(ro), _ptr(pro), ctypes.c_int64(len(pro) - 1)]


def quantize(v, _use=None) -> tuple[np.ndarray, np.ndarray]:
    """Q(v): nearest integer to v*1e7 (ties to even), and validity."""
    v = _c(np.atleast_1d(v), np.float64)
    q = np.zeros(v.shape, np.int32)
    ok = np.zeros(v.shape, np.uint8)
    (_use or _load()).orc_quantize_many(_ptr(v), v.size, _ptr(q), _ptr(ok))
    return q, ok.astype(bool)


def edge_crossing(ax, ay, bx, by, px, py, _use=None) -> int:
    return int((_use or _load()).orc_edge_crossing(int(ax), int(ay), int(bx), int(by), int(px), int(py)))


def inside(pset, poly: int, px: int, py: int, _use=None) -> int:
    keep, args = _poly_args(pset)
    return int((_use or _load()).orc_inside(*args, int(poly), int(px), int(py)))


def count_owners_q(pset, qx, qy, threads: int | None = None, _use=None) -> np.ndarray:
    keep, args = _poly_args(pset)
    qx = _c(qx, np.int32)
    qy = _c(qy, np.int32)
    out = np.zeros(qx.shape, np.int32)
    (_use or _load()).orc_count_owners_q(*args, _ptr(qx), _ptr(qy), qx.size, _ptr(out),
                               threads or default_threads())
    return out


def join_bruteforce_q(pset, qx, qy, threads: int | None = None, _use=None) -> np.ndarray:
    keep, args = _poly_args(pset)
    qx = _c(qx, np.int32)
    qy = _c(qy, np.int32)
    out = np.zeros(qx.shape, np.int32)
    (_use or _load()).orc_join_bruteforce_q(*args, _ptr(qx), _ptr(qy), qx.size, _ptr(out),
                                  threads or default_threads())
    return out


def join_bruteforce(pset, lon, lat, threads: int | None = None, _use=None) -> np.ndarray:
    """O0: brute force over all polygons (no filter)."""
    keep, args = _poly_args(pset)
    lon = _c(lon, np.float64)
    lat = _c(lat, np.float64)
    out = np.zeros(lon.shape, np.int32)
    (_use or _load()).orc_join_bruteforce(*args, _ptr(lon), _ptr(lat), lon.size, _ptr(out),
                                threads or default_threads())
    return out


def _parents_flat(pset):
    parents = list(getattr(pset, "parents", None) or [])
    if not parents:
        return np.zeros(1, np.int32), np.zeros(1, np.int64), 0
    flat = np.concatenate([_c(p, np.int32) for p in parents])
    lens = np.array([len(p) for p in parents], np.int64)
    return flat, lens, len(parents)


def join_hier(pset, lon, lat, threads: int | None = None, flat: bool = False, _use=None) -> np.ndarray:
    """O1: hierarchical closed-box filter, then the crossing test."""
    keep, args = _poly_args(pset)
    pf, pl, nl = _parents_flat(pset)
    if flat:
        nl = 0
    lon = _c(lon, np.float64)
    lat = _c(lat, np.float64)
    out = np.zeros(lon.shape, np.int32)
    (_use or _load()).orc_join_hier(*args, _ptr(pf), _ptr(pl), nl, _ptr(lon), _ptr(lat), lon.size,
                          _ptr(out), threads or default_threads())
    return out


class Hier:
    """O1 with its box hierarchy prepared once (for repeated joins against
    the same set, e.g. the timed CPU baseline)."""

    def __init__(self, pset, threads: int | None = None):
        self._keep, args = _poly_args(pset)
        self._pf, self._pl, nl = _parents_flat(pset)
        self._lib = _load()
        self.threads = threads or default_threads()
        self.h = self._lib.orc_hier_create(*args, _ptr(self._pf), _ptr(self._pl), nl)

    def join(self, lon, lat, threads: int | None = None) -> np.ndarray:
        lon = _c(lon, np.float64)
        lat = _c(lat, np.float64)
        out = np.zeros(lon.shape, np.int32)
        self._lib.orc_hier_join(self.h, _ptr(lon), _ptr(lat), lon.size, _ptr(out),
                                threads or self.threads)
        return out

    def __del__(self):
        if getattr(self, "h", None):
            self._lib.orc_hier_free(self.h)
            self.h = None
