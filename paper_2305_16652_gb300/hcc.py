"""Python binding of the hcc C ABI (include/hcc.h): argument marshalling only.

Every function has the name of the C entry point it calls and takes torch
tensors (device memory) or numpy arrays (host memory) in place of pointers.
All computation happens in libhcc.so; if that library is missing or fails
to load, every call raises -- there is no fallback path.

Tensor conventions:
  rays: two contiguous (n, 4) float32 CUDA tensors (org_tmin, dir_tmax)
  keys: (n,) int32 (key_bits <= 32) or int64 (key_bits > 32) CUDA tensor,
        read as unsigned by the library
  perm: (n,) int32 CUDA tensor (unsigned ray ids)
  hits: (n, 4) int32 CUDA tensor: prim, then the bits of t, u, v
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "csrc", "_build", "libhcc.so")

HCC_METHOD_NOSORT, HCC_METHOD_HCC, HCC_METHOD_TWOPOINT, HCC_METHOD_ORIGIN, HCC_METHOD_ORIGIN_DIR = 0, 1, 2, 3, 4
HCC_METHOD_PPC, HCC_METHOD_MLHCC = 5, 6
METHODS = {"nosort": HCC_METHOD_NOSORT, "hcc": HCC_METHOD_HCC, "twopoint": HCC_METHOD_TWOPOINT,
           "origin": HCC_METHOD_ORIGIN, "origin_dir": HCC_METHOD_ORIGIN_DIR, "ppc": HCC_METHOD_PPC,
           "mlhcc": HCC_METHOD_MLHCC}
STATUS = {0: "HCC_OK", 1: "HCC_ERR_INVALID_ARG", 2: "HCC_ERR_OOM", 3: "HCC_ERR_CUDA", 4: "HCC_ERR_UNSUPPORTED",
          5: "HCC_ERR_STACK_OVERFLOW", 6: "HCC_ERR_TIMEOUT"}
HIT_DTYPE = np.dtype([("prim", np.int32), ("t", np.float32), ("u", np.float32), ("v", np.float32)])


class HccError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Rays(ctypes.Structure):
    _fields_ = [("org_tmin", ctypes.c_void_p), ("dir_tmax", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("stride", ctypes.c_uint64)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("method", ctypes.c_int), ("key_bits", ctypes.c_uint32),
                ("hbm_budget", ctypes.c_uint64)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64), ("rays", ctypes.c_uint64),
                ("max_in_flight", ctypes.c_uint32), ("queued", ctypes.c_uint32), ("budget", ctypes.c_uint64),
                ("peak_bytes", ctypes.c_uint64)]


class _BvhDesc(ctypes.Structure):
    _fields_ = [("num_nodes", ctypes.c_uint32), ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p),
                ("left", ctypes.c_void_p), ("right", ctypes.c_void_p), ("first", ctypes.c_void_p),
                ("count", ctypes.c_void_p), ("num_tris", ctypes.c_uint32), ("tris", ctypes.c_void_p),
                ("order", ctypes.c_void_p)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libhcc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    P, u32, u64, i32, f64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "hcc_create": [PP, i32, P],
        "hcc_destroy": [P],
        "hcc_set_stream": [P, P],
        "hcc_set_trace_schedule": [P, i32],
        "hcc_set_twopoint_distance": [P, ctypes.c_float],
        "hcc_set_sort_wait_limit": [P, u32],
        "hcc_set_trace_shape": [P, u32, u32],
        "hcc_test_sort_withhold_tile": [P, u32],
        "hcc_reserve": [P, u64, u32],
        "hcc_sync": [P],
        "hcc_bvh_upload": [P, ctypes.POINTER(_BvhDesc), PP],
        "hcc_bvh_upload_layout": [P, ctypes.POINTER(_BvhDesc), i32, PP],
        "hcc_bvh_info": [P, P, P, P, P, P],
        "hcc_bvh_destroy": [P],
        "hcc_select_cut": [P, P, u32, f64, PP],
        "hcc_cut_info": [P, P, P],
        "hcc_cut_destroy": [P],
        "hcc_select_cut_ml": [P, P, u32, u32, f64, PP],
        "hcc_cut_ml_info": [P, P, P, P, P],
        "hcc_select_grid": [P, P, u32, PP],
        "hcc_cut_boxes": [P, P, P],
        "hcc_encode": [P, i32, P, P, ctypes.POINTER(_Rays), u32, P],
        "hcc_sort": [P, P, u32, u64, P],
        "hcc_gather": [P, ctypes.POINTER(_Rays), P, ctypes.POINTER(_Rays)],
        "hcc_trace": [P, P, ctypes.POINTER(_Rays), i32, P, P],
        "hcc_run": [P, i32, P, P, ctypes.POINTER(_Rays), u32, i32, P],
        "hcc_run_host": [P, i32, P, P, P, P, u64, u32, i32, P],
        "hcc_trace_counts": [P, P, ctypes.POINTER(_Rays), P, i32, P],
        "hcc_key_stats": [P, P, u32, P, u64, P, P],
        "hcc_trace_sorted": [P, P, ctypes.POINTER(_Rays), P, i32, P],
        "hcc_sort_noalloc": [P, u32, u64, P, P, P],
        "hcc_batch_create": [P, u32, P, P, P, PP],
        "hcc_batch_destroy": [P],
        "hcc_batch_run": [P, P, i32, ctypes.POINTER(_Rays), u32, i32, P],
        "hcc_batch_spawn": [P, P, ctypes.POINTER(_Rays), P, u64, ctypes.c_float, ctypes.POINTER(_Rays)],
        "hcc_graph_capture_batch": [P, P, i32, ctypes.POINTER(_Rays), u32, i32, P, PP],
        "hcc_graph_launch": [P, P],
        "hcc_graph_destroy": [P],
        "hcc_graph_begin": [P],
        "hcc_graph_end": [P, PP],
        "hcc_server_create": [i32, u32, P, P, ctypes.POINTER(_ServerConfig), PP],
        "hcc_server_submit": [P, u32, P, P, u64, i32, P, ctypes.POINTER(u64)],
        "hcc_server_query": [P, u64, ctypes.POINTER(i32)],
        "hcc_server_wait": [P, u64, ctypes.POINTER(f64)],
        "hcc_server_stats_get": [P, ctypes.POINTER(_ServerStats)],
        "hcc_server_destroy": [P],
        "hcc_server_request_bytes": [P, u64, ctypes.POINTER(u64)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.hcc_last_error.argtypes = [P]
    lib.hcc_last_error.restype = ctypes.c_char_p
    lib.hcc_status_string.argtypes = [ctypes.c_int]
    lib.hcc_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int, ctx=None):
    if status != 0:
        msg = load().hcc_last_error(ctx).decode() if ctx else ""
        raise HccError(status, msg)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(t.data_ptr())


def _row_stride_bytes(t) -> int:
    """Bytes between consecutive rays of an (n, 4) float32 view (torch or numpy)."""
    if isinstance(t, np.ndarray):
        if t.ndim != 2 or t.shape[1] != 4 or t.strides[1] != 4:
            raise ValueError("rays must be (n, 4) float32 views with contiguous rows")
        return int(t.strides[0])
    if t.dim() != 2 or t.shape[1] != 4 or t.stride(1) != 1:
        raise ValueError("rays must be (n, 4) float32 views with contiguous rows")
    return int(t.stride(0)) * t.element_size()


def _rays(org, dir_):
    """Ray descriptor of two (n, 4) views: two packed arrays, or the halves of
    an (n, 8) tensor of 32-byte records (rec[:, :4], rec[:, 4:])."""
    n = int(org.shape[0])
    if dir_.shape[0] != n:
        raise ValueError("org_tmin and dir_tmax differ in length")
    so, sd = (_row_stride_bytes(org), _row_stride_bytes(dir_)) if n > 1 else (16, 16)
    if so != sd:
        raise ValueError("org_tmin and dir_tmax must have the same row stride")
    return _Rays(_ptr(org), _ptr(dir_), n, so)


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


# ------------------------------------------------------------------ context

def hcc_create(device: int = 0, stream=None):
    h = ctypes.c_void_p()
    _check(load().hcc_create(ctypes.byref(h), device, _stream_handle(stream)))
    return h


def hcc_destroy(ctx):
    _check(load().hcc_destroy(ctx))


def hcc_set_stream(ctx, stream=None):
    _check(load().hcc_set_stream(ctx, _stream_handle(stream)), ctx)


def hcc_reserve(ctx, max_n: int, max_key_bits: int):
    _check(load().hcc_reserve(ctx, max_n, max_key_bits), ctx)


def hcc_sync(ctx):
    _check(load().hcc_sync(ctx), ctx)


# ---------------------------------------------------------------------- BVH

HCC_BVH_QUANTISED, HCC_BVH_EXACT, HCC_BVH_WIDE = 0, 1, 2
LAYOUTS = {"quantised": HCC_BVH_QUANTISED, "exact": HCC_BVH_EXACT, "wide": HCC_BVH_WIDE}


def hcc_bvh_upload(ctx, bvh, layout=None):
    """bvh: an object with lo, hi, left, right, first, count, order, tris numpy arrays.

    layout None calls hcc_bvh_upload (quantised nodes); "quantised", "exact" or
    "wide" calls hcc_bvh_upload_layout.
    """
    arrs = dict(lo=np.ascontiguousarray(bvh.lo, np.float32), hi=np.ascontiguousarray(bvh.hi, np.float32),
                left=np.ascontiguousarray(bvh.left, np.int32), right=np.ascontiguousarray(bvh.right, np.int32),
                first=np.ascontiguousarray(bvh.first, np.uint32), count=np.ascontiguousarray(bvh.count, np.uint32),
                tris=np.ascontiguousarray(bvh.tris, np.float32), order=np.ascontiguousarray(bvh.order, np.uint32))
    d = _BvhDesc(arrs["lo"].shape[0], _ptr(arrs["lo"]), _ptr(arrs["hi"]), _ptr(arrs["left"]), _ptr(arrs["right"]),
                 _ptr(arrs["first"]), _ptr(arrs["count"]), arrs["tris"].shape[0], _ptr(arrs["tris"]),
                 _ptr(arrs["order"]))
    h = ctypes.c_void_p()
    if layout is None:
        _check(load().hcc_bvh_upload(ctx, ctypes.byref(d), ctypes.byref(h)), ctx)
    else:
        _check(load().hcc_bvh_upload_layout(ctx, ctypes.byref(d), LAYOUTS.get(layout, layout), ctypes.byref(h)), ctx)
    return h


def hcc_bvh_upload_layout(ctx, bvh, layout):
    return hcc_bvh_upload(ctx, bvh, layout=layout)


def hcc_bvh_info(bvh):
    nn, nt, dep = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    lo, hi = (ctypes.c_float * 3)(), (ctypes.c_float * 3)()
    _check(load().hcc_bvh_info(bvh, ctypes.byref(nn), ctypes.byref(nt), ctypes.byref(dep), lo, hi))
    return dict(num_nodes=nn.value, num_tris=nt.value, depth=dep.value, scene_lo=list(lo), scene_hi=list(hi))


def hcc_bvh_destroy(bvh):
    _check(load().hcc_bvh_destroy(bvh))


# ---------------------------------------------------------------------- cut

TRACE_SCHEDULES = {"auto": 0, "per_ray": 1, "refill": 2}


def hcc_set_trace_schedule(ctx, schedule="auto"):
    """Ray scheduling of the context's traces: auto, per_ray or refill."""
    _check(load().hcc_set_trace_schedule(ctx, TRACE_SCHEDULES.get(schedule, schedule)), ctx)


def hcc_set_twopoint_distance(ctx, fraction: float = 0.25):
    """TwoPoint ray-length estimate as a fraction of the largest scene extent."""
    _check(load().hcc_set_twopoint_distance(ctx, fraction), ctx)


HCC_TRACE_STACK = 64  # default traversal-stack entries per ray (include/hcc.h)
TRACE_SHAPES = [(b, st) for b in (64, 128, 256) for st in (32, 48, 64)]


def hcc_set_trace_shape(ctx, block_threads: int = 0, stack_entries: int = 0):
    """Threads per block and stack entries per ray of the closest-hit persistent trace ((0, 0) = default)."""
    _check(load().hcc_set_trace_shape(ctx, block_threads, stack_entries), ctx)


def hcc_set_sort_wait_limit(ctx, status_reads: int = 0):
    """Look-back wait bound of the context's sorts (0 = the default 2^22 reads)."""
    _check(load().hcc_set_sort_wait_limit(ctx, status_reads), ctx)


def hcc_test_sort_withhold_tile(ctx, tile: int = 0xFFFFFFFF):
    """Test hook: tile `tile` of each digit pass never publishes its counts."""
    _check(load().hcc_test_sort_withhold_tile(ctx, tile), ctx)


def hcc_select_cut(ctx, bvh, cut_size: int, lam: float = 0.125):
    h = ctypes.c_void_p()
    _check(load().hcc_select_cut(ctx, bvh, cut_size, lam, ctypes.byref(h)), ctx)
    return h


def hcc_cut_info(cut) -> np.ndarray:
    n = ctypes.c_uint32()
    _check(load().hcc_cut_info(cut, ctypes.byref(n), None))
    ids = np.zeros(n.value, np.int32)
    _check(load().hcc_cut_info(cut, ctypes.byref(n), _ptr(ids)))
    return ids


def hcc_select_cut_ml(ctx, bvh, top_size: int, low_size: int, lam: float = 0.125):
    """Two-level MLHCC cut (Algorithm 3)."""
    h = ctypes.c_void_p()
    _check(load().hcc_select_cut_ml(ctx, bvh, top_size, low_size, lam, ctypes.byref(h)), ctx)
    return h


def hcc_cut_ml_info(cut):
    """(top ids, low ids (ntop, low_size), top_size, low_size) of a two-level cut."""
    ntop, tf, lf = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(load().hcc_cut_ml_info(cut, ctypes.byref(ntop), ctypes.byref(tf), ctypes.byref(lf), None))
    low = np.zeros(ntop.value * lf.value, np.int32)
    _check(load().hcc_cut_ml_info(cut, ctypes.byref(ntop), ctypes.byref(tf), ctypes.byref(lf), _ptr(low)))
    return hcc_cut_info(cut), low.reshape(ntop.value, lf.value), tf.value, lf.value


def hcc_select_grid(ctx, bvh, max_cells: int):
    """Regular-grid cells of the root box as a cut (Sec. 5)."""
    h = ctypes.c_void_p()
    _check(load().hcc_select_grid(ctx, bvh, max_cells, ctypes.byref(h)), ctx)
    return h


def hcc_cut_boxes(cut):
    """Host copy of the key-driving boxes: (lo (m, 3), hi (m, 3))."""
    m = min(len(hcc_cut_info(cut)), 64)
    lo = np.zeros((m, 3), np.float32)
    hi = np.zeros((m, 3), np.float32)
    _check(load().hcc_cut_boxes(cut, _ptr(lo), _ptr(hi)))
    return lo, hi


def hcc_cut_destroy(cut):
    _check(load().hcc_cut_destroy(cut))


# ------------------------------------------------------------- hot-path calls

def hcc_encode(ctx, method, bvh, cut, org, dir_, key_bits: int, keys):
    r = _rays(org, dir_)
    _check(load().hcc_encode(ctx, METHODS.get(method, method), bvh, cut, ctypes.byref(r), key_bits, _ptr(keys)), ctx)


def hcc_sort(ctx, keys, key_bits: int, n: int, perm):
    _check(load().hcc_sort(ctx, _ptr(keys), key_bits, n, _ptr(perm)), ctx)


HCC_SORT_NOALLOC_MAX_N = 524288


def hcc_sort_noalloc(keys, key_bits: int, n: int, perm, err_word=None, stream=None):
    """Sort without a context or any allocation (n <= HCC_SORT_NOALLOC_MAX_N)."""
    _check(load().hcc_sort_noalloc(_ptr(keys), key_bits, n, _ptr(perm), _ptr(err_word), _stream_handle(stream)))


def hcc_gather(ctx, in_org, in_dir, perm, out_org, out_dir):
    ri, ro = _rays(in_org, in_dir), _rays(out_org, out_dir)
    _check(load().hcc_gather(ctx, ctypes.byref(ri), _ptr(perm), ctypes.byref(ro)), ctx)


def hcc_trace(ctx, bvh, org, dir_, hits, any_hit: bool = False, scatter=None):
    r = _rays(org, dir_)
    _check(load().hcc_trace(ctx, bvh, ctypes.byref(r), int(any_hit), _ptr(scatter), _ptr(hits)), ctx)


def hcc_trace_sorted(ctx, bvh, org, dir_, perm, hits, any_hit: bool = False):
    """Trace ray perm[j] in slot j (fetch through the sorted ids); hits land in input order."""
    r = _rays(org, dir_)
    _check(load().hcc_trace_sorted(ctx, bvh, ctypes.byref(r), _ptr(perm), int(any_hit), _ptr(hits)), ctx)


def hcc_trace_counts(ctx, bvh, org, dir_, perm=None, any_hit: bool = False):
    """Diagnostic trace: node visits, triangle tests and warp-level node / leaf steps."""
    r = _rays(org, dir_)
    c = (ctypes.c_uint64 * 4)()
    _check(load().hcc_trace_counts(ctx, bvh, ctypes.byref(r), _ptr(perm), int(any_hit), c), ctx)
    return {"node_visits": int(c[0]), "tri_tests": int(c[1]), "warp_node_steps": int(c[2]),
            "warp_leaf_steps": int(c[3])}


def hcc_key_stats(ctx, keys, key_bits: int, perm, n: int):
    """Distinct keys and average distinct codes per warp of keys in sorted order."""
    anc, distinct = ctypes.c_double(), ctypes.c_uint64()
    _check(load().hcc_key_stats(ctx, _ptr(keys), key_bits, _ptr(perm), n, ctypes.byref(anc),
                                ctypes.byref(distinct)), ctx)
    return {"anc": anc.value, "distinct": int(distinct.value)}


# ------------------------------------------------------------------ batches

def hcc_batch_create(ctx, bvhs, cuts, offsets):
    """bvhs / cuts: lists of handles (cuts may be None or hold None); offsets: S + 1 ints."""
    S = len(bvhs)
    arr_b = (ctypes.c_void_p * S)(*[b.value if hasattr(b, "value") else b for b in bvhs])
    arr_c = None
    if cuts is not None:
        arr_c = (ctypes.c_void_p * S)(*[(c.value if hasattr(c, "value") else c) if c is not None else None
                                        for c in cuts])
    off = np.ascontiguousarray(offsets, np.uint64)
    h = ctypes.c_void_p()
    _check(load().hcc_batch_create(ctx, S, arr_b, arr_c, _ptr(off), ctypes.byref(h)), ctx)
    return h


def hcc_batch_destroy(batch):
    _check(load().hcc_batch_destroy(batch))


def hcc_batch_run(ctx, batch, method, org, dir_, key_bits: int, hits, any_hit: bool = False):
    r = _rays(org, dir_)
    _check(load().hcc_batch_run(ctx, batch, METHODS.get(method, method), ctypes.byref(r), key_bits, int(any_hit),
                                _ptr(hits)), ctx)


def hcc_batch_spawn(ctx, batch, in_org, in_dir, hits, seed: int, tmin: float, out_org, out_dir):
    ri, ro = _rays(in_org, in_dir), _rays(out_org, out_dir)
    _check(load().hcc_batch_spawn(ctx, batch, ctypes.byref(ri), _ptr(hits), seed, tmin, ctypes.byref(ro)), ctx)


def hcc_graph_capture_batch(ctx, batch, method, org, dir_, key_bits: int, hits, any_hit: bool = False):
    r = _rays(org, dir_)
    h = ctypes.c_void_p()
    _check(load().hcc_graph_capture_batch(ctx, batch, METHODS.get(method, method), ctypes.byref(r), key_bits,
                                          int(any_hit), _ptr(hits), ctypes.byref(h)), ctx)
    return h


def hcc_graph_begin(ctx):
    _check(load().hcc_graph_begin(ctx), ctx)


def hcc_graph_end(ctx):
    h = ctypes.c_void_p()
    _check(load().hcc_graph_end(ctx, ctypes.byref(h)), ctx)
    return h


def hcc_graph_launch(ctx, graph):
    _check(load().hcc_graph_launch(ctx, graph), ctx)


def hcc_graph_destroy(graph):
    _check(load().hcc_graph_destroy(graph))


def hcc_run(ctx, method, bvh, cut, org, dir_, key_bits: int, hits, any_hit: bool = False):
    r = _rays(org, dir_)
    _check(load().hcc_run(ctx, METHODS.get(method, method), bvh, cut, ctypes.byref(r), key_bits, int(any_hit),
                          _ptr(hits)), ctx)


def hcc_run_host(ctx, method, bvh, cut, org: np.ndarray, dir_: np.ndarray, key_bits: int, hits: np.ndarray,
                 any_hit: bool = False):
    """Host buffers in and out (numpy arrays or pinned CPU tensors)."""
    n = int(org.shape[0])
    _check(load().hcc_run_host(ctx, METHODS.get(method, method), bvh, cut, _ptr(org), _ptr(dir_), n, key_bits,
                               int(any_hit), _ptr(hits)), ctx)


# ------------------------------------------------------------- serving loop

def hcc_server_create(device: int, bvhs, cuts, slots: int, method="hcc", key_bits: int = 32,
                      hbm_budget: int = 0):
    """A ray-query server over resident scenes (bvhs[s], cuts[s] for HCC)."""
    arr_b = (ctypes.c_void_p * len(bvhs))(*[b.value if isinstance(b, ctypes.c_void_p) else b for b in bvhs])
    arr_c = None
    if cuts is not None:
        arr_c = (ctypes.c_void_p * len(cuts))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in cuts])
    cfg = _ServerConfig(slots, METHODS.get(method, method), key_bits, hbm_budget)
    h = ctypes.c_void_p()
    _check(load().hcc_server_create(device, len(bvhs), arr_b, arr_c, ctypes.byref(cfg), ctypes.byref(h)))
    return h


def hcc_server_submit(server, scene: int, org, dir_, hits, any_hit: bool = False) -> int:
    """Queue a request; org/dir/hits are host arrays (page-locked for overlap)
    that must stay alive until hcc_server_wait returns."""
    n = int(org.shape[0])
    if dir_.shape[0] != n or hits.shape[0] != n:
        raise ValueError("org_tmin, dir_tmax and hits differ in length")
    t = ctypes.c_uint64()
    _check(load().hcc_server_submit(server, scene, _ptr(org), _ptr(dir_), n, int(any_hit), _ptr(hits),
                                    ctypes.byref(t)))
    return t.value


def hcc_server_query(server, ticket: int) -> bool:
    d = ctypes.c_int()
    _check(load().hcc_server_query(server, ticket, ctypes.byref(d)))
    return bool(d.value)


def hcc_server_wait(server, ticket: int) -> float:
    """Wait for a request; returns its latency in ms, raises HccError if it failed."""
    ms = ctypes.c_double()
    _check(load().hcc_server_wait(server, ticket, ctypes.byref(ms)))
    return ms.value


def hcc_server_stats_get(server) -> dict:
    st = _ServerStats()
    _check(load().hcc_server_stats_get(server, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in _ServerStats._fields_}


def hcc_server_request_bytes(server, n: int) -> int:
    b = ctypes.c_uint64()
    _check(load().hcc_server_request_bytes(server, n, ctypes.byref(b)))
    return b.value


def hcc_server_destroy(server):
    _check(load().hcc_server_destroy(server))


def hits_to_numpy(hits_tensor) -> np.ndarray:
    """(n, 4) int32 hit tensor -> structured numpy array with prim, t, u, v."""
    a = hits_tensor.detach().cpu().numpy() if hasattr(hits_tensor, "detach") else np.asarray(hits_tensor)
    return np.ascontiguousarray(a, dtype=np.int32).view(HIT_DTYPE).reshape(-1)
