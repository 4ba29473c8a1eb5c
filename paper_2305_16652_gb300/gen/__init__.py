"""Seeded synthetic inputs: scenes, BVH2, camera visibility and rays.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests.  It produces inputs only and holds none of the method's
arithmetic (no slab test, key encoding, sort or ray/triangle test); see
``gen.c`` for what each generator draws.

Workload recipes (the paper's scenes are not available; these synthetic
stand-ins copy their structure, Sec. 6: dense detail clustered in small
regions of a closed space, 1920x1080, 8 samples per pixel, two shadow rays
per bounce):

* ``tiny_workload`` -- 10k random triangles in the unit cube, 64x64 camera,
  the first 4096 samples that see a triangle each emit one cosine-weighted
  diffuse secondary ray (tmin 1e-4).
* ``room_workload`` -- a closed 10 x 3 x 8 m room with ~1M triangles of
  clustered procedural furniture, 1920x1080 x 8 spp (every sample hits),
  one secondary ray per sample plus two shadow rays toward four ceiling
  lights.  ``scale`` shrinks the image for quick tests.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhccgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator library in-tree with gcc (host code only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    u32, u64, i32, f64, f32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_float
    lib.gen_rng_u64.argtypes = [u64, u64, u64]
    lib.gen_rng_u64.restype = u64
    lib.gen_random_tris.argtypes = [u64, u32, f64, f64, P]
    lib.gen_random_tris.restype = None
    lib.gen_room_tris.argtypes = [u64, u32, u32, P, u32]
    lib.gen_room_tris.restype = u32
    lib.gen_build_bvh.argtypes = [P, u32, i32, i32, P, P, P, P, P, P, P, P]
    lib.gen_build_bvh.restype = u32
    lib.gen_camera_rays.argtypes = [P, u32, P, P, f64, i32, i32, i32, u64, i32, u64, f32, P, P, i32, P, i32,
                                    f64, P, P, P]
    lib.gen_camera_rays.restype = u64
    _lib = lib
    return lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def rng_u64(seed: int, purpose: int, index: int) -> int:
    return int(_load().gen_rng_u64(seed, purpose, index))


def random_tris(seed: int, n: int, mu: float = -4.0, sigma: float = 0.5) -> np.ndarray:
    out = np.empty((n, 9), np.float32)
    _load().gen_random_tris(seed, n, mu, sigma, _ptr(out))
    return out


def room_tris(seed: int, target_tris: int = 1_000_000, clusters: int = 40) -> np.ndarray:
    lib = _load()
    n = lib.gen_room_tris(seed, target_tris, clusters, None, 0)
    out = np.empty((n, 9), np.float32)
    m = lib.gen_room_tris(seed, target_tris, clusters, _ptr(out), n)
    assert m == n
    return out


@dataclass
class BVH:
    """A BVH2 in depth-first pre-order (root = node 0).

    lo, hi: (nodes, 3) float32 exact boxes; left, right: child node ids or -1
    for a leaf; first, count: a leaf's range in ``order``; order: triangle ids
    in leaf order; tris: (T, 9) float32 triangles in scene order.
    """
    lo: np.ndarray
    hi: np.ndarray
    left: np.ndarray
    right: np.ndarray
    first: np.ndarray
    count: np.ndarray
    order: np.ndarray
    tris: np.ndarray
    depth: int

    @property
    def num_nodes(self) -> int:
        return int(self.lo.shape[0])

    @property
    def num_tris(self) -> int:
        return int(self.tris.shape[0])


def build_bvh(tris: np.ndarray, bins: int = 32, max_leaf: int = 4) -> BVH:
    tris = np.ascontiguousarray(tris, np.float32)
    T = tris.shape[0]
    cap = max(2 * T, 1)
    lo = np.empty((cap, 3), np.float32)
    hi = np.empty((cap, 3), np.float32)
    left = np.empty(cap, np.int32)
    right = np.empty(cap, np.int32)
    first = np.empty(cap, np.uint32)
    count = np.empty(cap, np.uint32)
    order = np.empty(max(T, 1), np.uint32)
    depth = ctypes.c_uint32(0)
    n = _load().gen_build_bvh(_ptr(tris), T, bins, max_leaf, _ptr(lo), _ptr(hi), _ptr(left), _ptr(right),
                              _ptr(first), _ptr(count), _ptr(order), ctypes.byref(depth))
    return BVH(lo[:n].copy(), hi[:n].copy(), left[:n].copy(), right[:n].copy(), first[:n].copy(),
               count[:n].copy(), order[:T].copy(), tris, int(depth.value))


@dataclass
class Rays:
    """N rays as two float4 streams: (ox, oy, oz, tmin) and (dx, dy, dz, tmax)."""
    org: np.ndarray  # (N, 4) float32
    dir: np.ndarray  # (N, 4) float32

    @property
    def n(self) -> int:
        return int(self.org.shape[0])

    def take(self, idx) -> "Rays":
        return Rays(np.ascontiguousarray(self.org[idx]), np.ascontiguousarray(self.dir[idx]))


def camera_rays(tris: np.ndarray, cam_pos, cam_target, vfov_deg: float, W: int, H: int, spp: int, seed: int,
                sample_major: bool, max_rays: int | None = None, tmin: float = 1e-4, n_shadow: int = 0,
                lights=None, light_half: float = 0.25):
    """Secondary (and optional shadow) rays leaving the camera's visible points."""
    tris = np.ascontiguousarray(tris, np.float32)
    ns = W * H * spp
    m = ns if max_rays is None else min(ns, max_rays)
    sec_o = np.empty((m, 4), np.float32)
    sec_d = np.empty((m, 4), np.float32)
    prim = np.empty(m, np.int32)
    if n_shadow:
        lights = np.ascontiguousarray(np.asarray(lights, np.float64).reshape(-1, 3))
        sh_o = np.empty((m * n_shadow, 4), np.float32)
        sh_d = np.empty((m * n_shadow, 4), np.float32)
        nl = lights.shape[0]
    else:
        lights, sh_o, sh_d, nl = None, None, None, 0
    cp = np.asarray(cam_pos, np.float64)
    ct = np.asarray(cam_target, np.float64)
    n = _load().gen_camera_rays(_ptr(tris), tris.shape[0], _ptr(cp), _ptr(ct), vfov_deg, W, H, spp, seed,
                                int(sample_major), m, tmin, _ptr(sec_o), _ptr(sec_d), n_shadow, _ptr(lights), nl,
                                light_half, _ptr(sh_o), _ptr(sh_d), _ptr(prim))
    sec = Rays(sec_o[:n], sec_d[:n])
    sh = Rays(sh_o[: n * n_shadow], sh_d[: n * n_shadow]) if n_shadow else None
    return sec, sh, prim[:n]


@dataclass
class Workload:
    name: str
    tris: np.ndarray
    bvh: BVH
    rays: Rays             # secondary rays (closest hit)
    shadow: Rays | None    # shadow rays (any hit)
    primary_prim: np.ndarray


def tiny_workload(seed: int = 0, ntris: int = 10_000, nrays: int = 4096) -> Workload:
    """10k random triangles in the unit cube; 4096 diffuse secondary rays."""
    tris = random_tris(seed, ntris)
    bvh = build_bvh(tris)
    # Iterate (pixel = i mod 4096, sample = i div 4096) until nrays primaries hit.
    sec, _, prim = camera_rays(tris, (0.5, 0.5, -1.2), (0.5, 0.5, 0.5), 45.0, 64, 64, 64, seed,
                               sample_major=True, max_rays=nrays)
    if sec.n < nrays:
        raise RuntimeError(f"only {sec.n} primary hits")
    return Workload("tiny-10k-tris-4096-rays", tris, bvh, sec, None, prim)


ROOM_LIGHTS = ((2.5, 2.95, 2.0), (7.5, 2.95, 2.0), (2.5, 2.95, 6.0), (7.5, 2.95, 6.0))
P_BATCH_TRIS, P_BATCH_RAYS = 100, 101
P_SERVE_SCENE, P_SERVE_SIZE, P_SERVE_OFFSET, P_SERVE_GAP = 102, 103, 104, 105


def _unit(seed: int, purpose: int, index: int) -> float:
    """Uniform double in [0, 1) from the counter-based generator."""
    return (rng_u64(seed, purpose, index) >> 11) * (1.0 / 9007199254740992.0)


def _log_uniform(seed: int, purpose: int, lo: float, hi: float, index: int = 0) -> int:
    u = _unit(seed, purpose, index)
    return int(round(float(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo))))))


def batch_workloads(seeds=range(2, 18), tris_range=(50_000, 2_000_000), rays_range=(65_536, 8_388_608),
                    scale: float = 1.0):
    """One furnished room per seed with a log-uniform triangle count and a
    log-uniform wavefront size (8 spp, 16:9 image, every sample hits).
    scale < 1 shrinks both ranges (quick runs)."""
    out = []
    for seed in seeds:
        nt = max(2_000, int(_log_uniform(seed, P_BATCH_TRIS, *tris_range) * scale))
        nr = max(1_024, int(_log_uniform(seed, P_BATCH_RAYS, *rays_range) * scale))
        H = int(np.ceil(np.sqrt(nr / 8 * 9 / 16)))
        W = int(np.ceil(H * 16 / 9))
        tris = room_tris(seed, nt, clusters=40)
        bvh = build_bvh(tris)
        sec, _, prim = camera_rays(tris, (5.0, 1.6, 0.4), (5.0, 1.2, 8.0), 60.0, W, H, 8, seed, sample_major=False,
                                   max_rays=nr)
        out.append(Workload(f"room-seed{seed}-{tris.shape[0]}-tris-{sec.n}-rays", tris, bvh, sec, None, prim))
    return out


def serve_scenes(seeds=range(30, 38), tris_range=(200_000, 4_000_000), W: int = 1920, H: int = 1080, spp: int = 2,
                 scale: float = 1.0):
    """Resident scenes of a ray-query server: one furnished room per seed with a
    log-uniform triangle count and a pool of W x H x spp diffuse secondary rays
    (pixel-major) from which requests take contiguous windows.  scale < 1
    shrinks the triangle counts and the image (quick runs)."""
    out = []
    for seed in seeds:
        nt = max(2_000, int(_log_uniform(seed, P_BATCH_TRIS, *tris_range) * scale))
        w, h = max(16, int(W * np.sqrt(scale))), max(9, int(H * np.sqrt(scale)))
        tris = room_tris(seed, nt, clusters=40)
        bvh = build_bvh(tris)
        sec, _, prim = camera_rays(tris, (5.0, 1.6, 0.4), (5.0, 1.2, 8.0), 60.0, w, h, spp, seed, sample_major=False)
        out.append(Workload(f"room-seed{seed}-{tris.shape[0]}-tris-{sec.n}-ray-pool", tris, bvh, sec, None, prim))
    return out


def serve_requests(seed: int, count: int, pool_sizes, rays_range=(65_536, 4_194_304)):
    """A request stream: request i goes to a uniformly drawn scene, asks for a
    log-uniform number of rays in rays_range (capped by the scene's pool) taken
    as a window at a uniform offset of the pool, and arrives a unit-mean
    exponential gap after request i-1 (Poisson arrivals at rate 1; scale the
    gaps by 1/rate).  Returns arrays scene, n, offset, gap."""
    S = len(pool_sizes)
    scene = np.empty(count, np.int64)
    n = np.empty(count, np.int64)
    off = np.empty(count, np.int64)
    gap = np.empty(count, np.float64)
    for i in range(count):
        s = min(int(_unit(seed, P_SERVE_SCENE, i) * S), S - 1)
        k = min(_log_uniform(seed, P_SERVE_SIZE, *rays_range, index=i), int(pool_sizes[s]))
        scene[i], n[i] = s, k
        off[i] = min(int(_unit(seed, P_SERVE_OFFSET, i) * (pool_sizes[s] - k + 1)), pool_sizes[s] - k)
        gap[i] = -np.log1p(-_unit(seed, P_SERVE_GAP, i))
    return {"scene": scene, "n": n, "offset": off, "gap": gap}


ROOM_CAMERA = ((5.0, 1.6, 0.4), (5.0, 1.2, 8.0), 60.0)
# a limited viewport (Sec. 6.3): a narrow view of the floor from the same eye point
LIMITED_CAMERA = ((5.0, 1.6, 0.4), (5.5, 0.0, 4.0), 10.0)


def room_workload(seed: int = 1, target_tris: int = 1_000_000, W: int = 1920, H: int = 1080, spp: int = 8,
                  shadow: bool = True, bvh: BVH | None = None, tris: np.ndarray | None = None,
                  camera=ROOM_CAMERA) -> Workload:
    """Closed furnished room, one diffuse bounce plus 2 shadow rays per sample.
    camera = (eye, target, vertical FOV in degrees)."""
    if tris is None:
        tris = room_tris(seed, target_tris)
    if bvh is None:
        bvh = build_bvh(tris)
    eye, target, vfov = camera
    sec, sh, prim = camera_rays(tris, eye, target, vfov, W, H, spp, seed,
                                sample_major=False, n_shadow=2 if shadow else 0, lights=ROOM_LIGHTS,
                                light_half=0.25)
    tag = "" if camera == ROOM_CAMERA else f"-fov{vfov:g}"
    return Workload(f"room-{tris.shape[0]}-tris-{W}x{H}x{spp}spp{tag}", tris, bvh, sec, sh, prim)
