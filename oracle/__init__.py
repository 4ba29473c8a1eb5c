"""CPU oracle for the hierarchy-cut-code hot path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
and reference legs may import this package.  The product library
(``paper_2305_16652_gb300``) never imports, links or calls it; the two share
no code.  Functions take and return numpy arrays and run single-threaded in
``hcc_oracle.cpp`` (built with g++, no FMA contraction).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hcc_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhcc_oracle.so")
_lib = None

HIT_DTYPE = np.dtype([("prim", np.int32), ("t", np.float32), ("u", np.float32), ("v", np.float32)])


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    u32, u64, i32, f64, f32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_float
    lib.oracle_surface_area.argtypes = [P, P]
    lib.oracle_surface_area.restype = f64
    lib.oracle_had.argtypes = [u32, P, P, P, P, P, f64, P]
    lib.oracle_had.restype = None
    lib.oracle_select_cut.argtypes = [u32, P, P, P, P, P, u32, f64, P]
    lib.oracle_select_cut.restype = u32
    lib.oracle_encode_hcc.argtypes = [u64, P, P, u32, P, P, u32, P]
    lib.oracle_encode_hcc.restype = None
    lib.oracle_key_margin.argtypes = [u64, P, P, u32, P, P, u32, P]
    lib.oracle_key_margin.restype = None
    lib.oracle_select_cut_ml.argtypes = [u32, P, P, P, P, P, u32, u32, f64, P, P]
    lib.oracle_select_cut_ml.restype = u32
    lib.oracle_encode_mlhcc.argtypes = [u64, P, P, u32, u32, P, P, u32, P, P, u32, P]
    lib.oracle_encode_mlhcc.restype = None
    lib.oracle_grid_cells.argtypes = [P, P, u32, P, P, P]
    lib.oracle_grid_cells.restype = u32
    lib.oracle_encode_ppc.argtypes = [u64, P, P, u32, P, P, P, P, u32, P]
    lib.oracle_encode_ppc.restype = None
    lib.oracle_encode_twopoint.argtypes = [u64, P, P, P, P, u32, P]
    lib.oracle_encode_twopoint_frac.argtypes = [u64, P, P, P, P, f32, u32, P]
    lib.oracle_encode_twopoint_frac.restype = None
    lib.oracle_encode_twopoint.restype = None
    lib.oracle_encode_origin.argtypes = [u64, P, P, P, u32, P]
    lib.oracle_encode_origin.restype = None
    lib.oracle_encode_origin_dir.argtypes = [u64, P, P, P, P, u32, P]
    lib.oracle_encode_origin_dir.restype = None
    lib.oracle_octahedral.argtypes = [P, P, P]
    lib.oracle_octahedral.restype = None
    lib.oracle_anc.argtypes = [u64, P, P]
    lib.oracle_anc.restype = f64
    lib.oracle_spawn.argtypes = [u64, P, P, P, P, u32, u64, f32, u64, P, P]
    lib.oracle_spawn.restype = None
    lib.oracle_stable_sort.argtypes = [u64, P, P]
    lib.oracle_stable_sort.restype = None
    lib.oracle_gather.argtypes = [u64, P, P, P, P, P]
    lib.oracle_gather.restype = None
    lib.oracle_intersect.argtypes = [P, P, f32, f32, P, P, P, P]
    lib.oracle_intersect.restype = i32
    lib.oracle_trace_brute.argtypes = [u32, P, u64, P, P, i32, P]
    lib.oracle_trace_brute.restype = None
    lib.oracle_trace_bvh.argtypes = [u32, P, P, P, P, P, P, P, P, u64, P, P, i32, P]
    lib.oracle_trace_bvh.restype = None
    _lib = lib
    return lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def surface_area(lo, hi) -> float:
    lo, hi = _c(lo, np.float32), _c(hi, np.float32)
    return float(_load().oracle_surface_area(_p(lo), _p(hi)))


def _tree(bvh):
    return (_c(bvh.lo, np.float32), _c(bvh.hi, np.float32), _c(bvh.left, np.int32), _c(bvh.right, np.int32),
            _c(bvh.count, np.uint32))


def had(bvh, lam: float = 0.125) -> np.ndarray:
    lo, hi, left, right, count = _tree(bvh)
    out = np.zeros(lo.shape[0], np.float64)
    _load().oracle_had(lo.shape[0], _p(lo), _p(hi), _p(left), _p(right), _p(count), lam, _p(out))
    return out


def select_cut(bvh, cut_size: int, lam: float = 0.125) -> np.ndarray:
    """Cut node ids in key order (HAD descending)."""
    lo, hi, left, right, count = _tree(bvh)
    out = np.zeros(max(cut_size, 1), np.int32)
    m = _load().oracle_select_cut(lo.shape[0], _p(lo), _p(hi), _p(left), _p(right), _p(count), cut_size, lam,
                                  _p(out))
    return out[:m].copy()


def encode_hcc(org, dir, cut_lo, cut_hi, key_bits: int) -> np.ndarray:
    org, dir = _c(org, np.float32), _c(dir, np.float32)
    cut_lo, cut_hi = _c(cut_lo, np.float32), _c(cut_hi, np.float32)
    n = org.shape[0]
    keys = np.zeros(n, np.uint64)
    _load().oracle_encode_hcc(n, _p(org), _p(dir), cut_lo.shape[0], _p(cut_lo), _p(cut_hi), key_bits, _p(keys))
    return keys


def key_margin(org, dir, cut_lo, cut_hi, key_bits: int) -> np.ndarray:
    org, dir = _c(org, np.float32), _c(dir, np.float32)
    cut_lo, cut_hi = _c(cut_lo, np.float32), _c(cut_hi, np.float32)
    n = org.shape[0]
    out = np.zeros(n, np.float64)
    _load().oracle_key_margin(n, _p(org), _p(dir), cut_lo.shape[0], _p(cut_lo), _p(cut_hi), key_bits, _p(out))
    return out


def select_cut_ml(bvh, top_size: int, low_size: int, lam: float = 0.125):
    """Two-level MLHCC cut: (top ids in HAD order, low ids of shape (ntop, low_size))."""
    lo, hi, left, right, count = _tree(bvh)
    top = np.zeros(max(top_size, 1), np.int32)
    low = np.zeros(max(top_size * low_size, 1), np.int32)
    m = _load().oracle_select_cut_ml(lo.shape[0], _p(lo), _p(hi), _p(left), _p(right), _p(count), top_size,
                                     low_size, lam, _p(top), _p(low))
    return top[:m].copy(), low[:m * low_size].reshape(m, low_size).copy()


def encode_mlhcc(org, dir, top_field: int, top_lo, top_hi, low_lo, low_hi, key_bits: int) -> np.ndarray:
    """low_lo/low_hi: (ntop, low_field, 3) boxes of each top node's low cut."""
    org, dir = _c(org, np.float32), _c(dir, np.float32)
    top_lo, top_hi = _c(top_lo, np.float32).reshape(-1, 3), _c(top_hi, np.float32).reshape(-1, 3)
    low_lo, low_hi = _c(low_lo, np.float32), _c(low_hi, np.float32)
    ntop = top_lo.shape[0]
    low_field = low_lo.shape[1] if low_lo.ndim == 3 else 0
    n = org.shape[0]
    keys = np.zeros(n, np.uint64)
    _load().oracle_encode_mlhcc(n, _p(org), _p(dir), top_field, ntop, _p(top_lo), _p(top_hi), low_field,
                                _p(low_lo), _p(low_hi), key_bits, _p(keys))
    return keys


def grid_cells(scene_lo, scene_hi, max_cells: int):
    """Regular-grid cells: (lo (m, 3), hi (m, 3), dims (3,))."""
    slo, shi = _c(scene_lo, np.float32), _c(scene_hi, np.float32)
    cap = 1
    while cap * 2 <= max(max_cells, 1):
        cap *= 2
    lo = np.zeros((cap, 3), np.float32)
    hi = np.zeros((cap, 3), np.float32)
    dims = np.zeros(3, np.uint32)
    m = _load().oracle_grid_cells(_p(slo), _p(shi), max_cells, _p(lo), _p(hi), _p(dims))
    return lo[:m].copy(), hi[:m].copy(), dims


def encode_ppc(org, dir, bvh, key_bits: int) -> np.ndarray:
    lo, hi, left, right, _ = _tree(bvh)
    org, dir = _c(org, np.float32), _c(dir, np.float32)
    n = org.shape[0]
    keys = np.zeros(n, np.uint64)
    _load().oracle_encode_ppc(n, _p(org), _p(dir), lo.shape[0], _p(lo), _p(hi), _p(left), _p(right), key_bits,
                              _p(keys))
    return keys


def encode_twopoint(org, dir, scene_lo, scene_hi, key_bits: int, fraction=None) -> np.ndarray:
    """TwoPoint keys; fraction = estimated ray length / largest scene extent (None: Sec. 5's 0.25)."""
    org, dir = _c(org, np.float32), _c(dir, np.float32)
    lo, hi = _c(scene_lo, np.float32), _c(scene_hi, np.float32)
    n = org.shape[0]
    keys = np.zeros(n, np.uint64)
    if fraction is None:
        _load().oracle_encode_twopoint(n, _p(org), _p(dir), _p(lo), _p(hi), key_bits, _p(keys))
    else:
        _load().oracle_encode_twopoint_frac(n, _p(org), _p(dir), _p(lo), _p(hi), fraction, key_bits, _p(keys))
    return keys


def encode_origin(org, scene_lo, scene_hi, key_bits: int) -> np.ndarray:
    org = _c(org, np.float32)
    lo, hi = _c(scene_lo, np.float32), _c(scene_hi, np.float32)
    n = org.shape[0]
    keys = np.zeros(n, np.uint64)
    _load().oracle_encode_origin(n, _p(org), _p(lo), _p(hi), key_bits, _p(keys))
    return keys


def encode_origin_dir(org, dir, scene_lo, scene_hi, key_bits: int) -> np.ndarray:
    org, dir = _c(org, np.float32), _c(dir, np.float32)
    lo, hi = _c(scene_lo, np.float32), _c(scene_hi, np.float32)
    n = org.shape[0]
    keys = np.zeros(n, np.uint64)
    _load().oracle_encode_origin_dir(n, _p(org), _p(dir), _p(lo), _p(hi), key_bits, _p(keys))
    return keys


def octahedral(d):
    d = _c(d, np.float32)
    u, v = ctypes.c_float(), ctypes.c_float()
    _load().oracle_octahedral(_p(d), ctypes.byref(u), ctypes.byref(v))
    return u.value, v.value


def anc(keys, perm) -> float:
    keys, perm = _c(keys, np.uint64), _c(perm, np.uint32)
    return float(_load().oracle_anc(keys.shape[0], _p(keys), _p(perm)))


def spawn(org, dir, hits, tris, seed: int, tmin: float, first_index: int = 0):
    """Next-bounce rays from hit records (structured HIT_DTYPE array); ray k is
    ray first_index + k of its batch."""
    org, dir, tris = _c(org, np.float32), _c(dir, np.float32), _c(tris, np.float32)
    hits = np.ascontiguousarray(hits, dtype=HIT_DTYPE)
    n = org.shape[0]
    oo = np.zeros((n, 4), np.float32)
    od = np.zeros((n, 4), np.float32)
    _load().oracle_spawn(n, _p(org), _p(dir), _p(hits), _p(tris), tris.shape[0], seed, tmin, first_index, _p(oo),
                         _p(od))
    return oo, od


def stable_sort(keys) -> np.ndarray:
    keys = _c(keys, np.uint64)
    n = keys.shape[0]
    perm = np.zeros(n, np.uint32)
    _load().oracle_stable_sort(n, _p(keys), _p(perm))
    return perm


def gather(org, dir, perm):
    org, dir, perm = _c(org, np.float32), _c(dir, np.float32), _c(perm, np.uint32)
    n = perm.shape[0]
    oo = np.zeros((n, 4), np.float32)
    od = np.zeros((n, 4), np.float32)
    _load().oracle_gather(n, _p(org), _p(dir), _p(perm), _p(oo), _p(od))
    return oo, od


def intersect(o, d, tmin, tmax, tri):
    o, d, tri = _c(o, np.float32), _c(d, np.float32), _c(tri, np.float32)
    t, u, v = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    hit = _load().oracle_intersect(_p(o), _p(d), tmin, tmax, _p(tri), ctypes.byref(t), ctypes.byref(u),
                                   ctypes.byref(v))
    return (bool(hit), t.value, u.value, v.value)


def trace_brute(tris, org, dir, any_hit: bool = False) -> np.ndarray:
    tris, org, dir = _c(tris, np.float32), _c(org, np.float32), _c(dir, np.float32)
    n = org.shape[0]
    hits = np.zeros(n, HIT_DTYPE)
    _load().oracle_trace_brute(tris.shape[0], _p(tris), n, _p(org), _p(dir), int(any_hit), _p(hits))
    return hits


def trace_bvh(bvh, org, dir, any_hit: bool = False) -> np.ndarray:
    lo, hi, left, right, count = _tree(bvh)
    first, order = _c(bvh.first, np.uint32), _c(bvh.order, np.uint32)
    tris, org, dir = _c(bvh.tris, np.float32), _c(org, np.float32), _c(dir, np.float32)
    n = org.shape[0]
    hits = np.zeros(n, HIT_DTYPE)
    _load().oracle_trace_bvh(lo.shape[0], _p(lo), _p(hi), _p(left), _p(right), _p(first), _p(count), _p(order),
                             _p(tris), n, _p(org), _p(dir), int(any_hit), _p(hits))
    return hits
