"""CUDA path against the CPU oracle, element by element (needs a GB300).

Every check goes through the C ABI (libhcc.so via the ctypes binding).
Integer results (cut ids, keys, permutations, gathered bytes) must be equal
bit for bit.  Keys may differ only on rays within 1e-6 (relative) of a cut
box boundary; hit records must be bit-identical except on near-edge ties
(the oracle's hit within 1e-6 of a triangle edge in barycentric terms, and t
within 1e-5 relative); the rules are in parity.py.  Such exceptions are
counted, bounded and printed at the end of the run.
"""
import numpy as np
import pytest

import oracle
from paper_2305_16652_gb300 import gen, hcc
from parity import compare_hits, compare_keys

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


# ------------------------------------------------------------------ fixtures

@pytest.fixture(scope="module")
def ctx():
    c = hcc.hcc_create(0)
    yield c
    hcc.hcc_destroy(c)


class Scene:
    def __init__(self, ctx, w):
        self.w = w
        self.bvh = hcc.hcc_bvh_upload(ctx, w.bvh)
        self.bvh_exact = hcc.hcc_bvh_upload(ctx, w.bvh, layout="exact")
        self.bvh_wide = hcc.hcc_bvh_upload(ctx, w.bvh, layout="wide")
        self.org = torch.from_numpy(w.rays.org).to(DEV)
        self.dir = torch.from_numpy(w.rays.dir).to(DEV)
        self.n = w.rays.n


def _dense_workload(seed=4, ntris=3000, nrays=3000):
    tris = gen.random_tris(seed, ntris, mu=-2.0)
    b = gen.build_bvh(tris)
    sec, _, prim = gen.camera_rays(tris, (0.5, 0.5, -1.2), (0.5, 0.5, 0.5), 45.0, 48, 48, 16, seed,
                                   sample_major=True, max_rays=nrays)
    return gen.Workload("dense", tris, b, sec, None, prim)


@pytest.fixture(scope="module")
def tiny(ctx):
    return Scene(ctx, gen.tiny_workload(0))


@pytest.fixture(scope="module")
def dense(ctx):
    return Scene(ctx, _dense_workload())


@pytest.fixture(scope="module")
def room(ctx):
    return Scene(ctx, gen.room_workload(1, target_tris=60_000, W=160, H=90, spp=2))


def _keys_tensor(n, k):
    return torch.zeros(n, dtype=torch.int32 if k <= 32 else torch.int64, device=DEV)


def _u64(keys_t, k):
    a = keys_t.cpu().numpy()
    return (a.view(np.uint32) if k <= 32 else a.view(np.uint64)).astype(np.uint64)


def gpu_encode(ctx, sc, method, k, cut=None, org=None, dir_=None):
    org = sc.org if org is None else org
    dir_ = sc.dir if dir_ is None else dir_
    keys = _keys_tensor(org.shape[0], k)
    hcc.hcc_encode(ctx, method, sc.bvh, cut, org, dir_, k, keys)
    hcc.hcc_sync(ctx)
    return _u64(keys, k)


def gpu_sort(ctx, keys_u64, k):
    n = keys_u64.shape[0]
    if k <= 32:
        kt = torch.from_numpy(keys_u64.astype(np.uint32).view(np.int32)).to(DEV)
    else:
        kt = torch.from_numpy(keys_u64.view(np.int64)).to(DEV)
    perm = torch.full((max(n, 1),), -7, dtype=torch.int32, device=DEV)
    hcc.hcc_sort(ctx, kt, k, n, perm)
    hcc.hcc_sync(ctx)
    return perm[:n].cpu().numpy().view(np.uint32)


def gpu_trace(ctx, sc, org, dir_, any_hit=False, scatter=None, layout="quantised"):
    hits = torch.zeros((org.shape[0], 4), dtype=torch.int32, device=DEV)
    bvh = {"quantised": sc.bvh, "exact": sc.bvh_exact, "wide": sc.bvh_wide}[layout]
    hcc.hcc_trace(ctx, bvh, org, dir_, hits, any_hit=any_hit, scatter=scatter)
    hcc.hcc_sync(ctx)
    return hcc.hits_to_numpy(hits)


# --------------------------------------------------------------------- cut

@pytest.mark.parametrize("which", ["tiny", "room"])
def test_cut_matches_oracle(ctx, which, request):
    sc = request.getfixturevalue(which)
    nleaves = int(np.sum(sc.w.bvh.left < 0))
    for C in (1, 2, 3, 32, 64, 256, 4096, nleaves, nleaves + 5):
        for lam in (0.125, 0.0, 1.0):
            cut = hcc.hcc_select_cut(ctx, sc.bvh, C, lam)
            try:
                assert np.array_equal(hcc.hcc_cut_info(cut), oracle.select_cut(sc.w.bvh, C, lam)), (C, lam)
            finally:
                hcc.hcc_cut_destroy(cut)


# ------------------------------------------------------------------ encode

@pytest.mark.parametrize("k", [1, 16, 24, 31, 32, 33, 48, 64])
@pytest.mark.parametrize("C", [32, 64])
@pytest.mark.parametrize("which", ["tiny", "room"])
def test_encode_hcc_matches_oracle(ctx, which, C, k, request):
    sc = request.getfixturevalue(which)
    cut = hcc.hcc_select_cut(ctx, sc.bvh, C, 0.125)
    ids = hcc.hcc_cut_info(cut)
    try:
        g = gpu_encode(ctx, sc, "hcc", k, cut=cut)
    finally:
        hcc.hcc_cut_destroy(cut)
    lo, hi = sc.w.bvh.lo[ids], sc.w.bvh.hi[ids]
    o = oracle.encode_hcc(sc.w.rays.org, sc.w.rays.dir, lo, hi, k)
    compare_keys(g, o, lambda b: oracle.key_margin(sc.w.rays.org[b], sc.w.rays.dir[b], lo, hi, k))
    assert np.all(g < (np.uint64(1) << np.uint64(k)) if k < 64 else True)
    if k >= 16:
        assert len(np.unique(g)) > 1


@pytest.mark.parametrize("k", [16, 32, 64])
@pytest.mark.parametrize("C", [256, 4096])
def test_encode_hcc_large_cuts_use_the_highest_had_nodes(ctx, room, C, k):
    """A cut larger than the key: the key's bits come from the min(C, k) cut
    nodes of highest HAD, in the oracle's order."""
    cut = hcc.hcc_select_cut(ctx, room.bvh, C, 0.125)
    ids = hcc.hcc_cut_info(cut)
    try:
        assert len(ids) == C
        g = gpu_encode(ctx, room, "hcc", k, cut=cut)
    finally:
        hcc.hcc_cut_destroy(cut)
    lo, hi = room.w.bvh.lo[ids], room.w.bvh.hi[ids]
    o = oracle.encode_hcc(room.w.rays.org, room.w.rays.dir, lo, hi, k)
    o_first = oracle.encode_hcc(room.w.rays.org, room.w.rays.dir, lo[:k], hi[:k], k)
    assert np.array_equal(o, o_first)  # the oracle reads only the first k nodes
    compare_keys(g, o, lambda b: oracle.key_margin(room.w.rays.org[b], room.w.rays.dir[b], lo, hi, k))
    assert len(np.unique(g)) > 1


@pytest.mark.parametrize("k", [1, 5, 6, 16, 30, 32, 33, 60, 64])
def test_encode_twopoint_matches_oracle(ctx, room, k):
    g = gpu_encode(ctx, room, "twopoint", k)
    o = oracle.encode_twopoint(room.w.rays.org, room.w.rays.dir, room.w.bvh.lo[0], room.w.bvh.hi[0], k)
    assert np.array_equal(g, o)


@pytest.mark.parametrize("k", [1, 3, 6, 16, 24, 31, 32, 33, 48, 64])
def test_encode_origin_keys_match_oracle(ctx, room, k):
    lo, hi = room.w.bvh.lo[0], room.w.bvh.hi[0]
    g = gpu_encode(ctx, room, "origin", k)
    assert np.array_equal(g, oracle.encode_origin(room.w.rays.org, lo, hi, k))
    g = gpu_encode(ctx, room, "origin_dir", k)
    assert np.array_equal(g, oracle.encode_origin_dir(room.w.rays.org, room.w.rays.dir, lo, hi, k))


@pytest.mark.parametrize("method,k", [("hcc", 16), ("hcc", 32), ("hcc", 64), ("twopoint", 32), ("origin_dir", 24)])
def test_key_stats_match_oracle(ctx, room, method, k):
    cut = hcc.hcc_select_cut(ctx, room.bvh, max(k, 32), 0.125) if method == "hcc" else None
    keys = _keys_tensor(room.n, k)
    perm = torch.zeros(room.n, dtype=torch.int32, device=DEV)
    try:
        hcc.hcc_encode(ctx, method, room.bvh, cut, room.org, room.dir, k, keys)
        hcc.hcc_sort(ctx, keys, k, room.n, perm)
        st = hcc.hcc_key_stats(ctx, keys, k, perm, room.n)
    finally:
        if cut is not None:
            hcc.hcc_cut_destroy(cut)
    ku, pu = _u64(keys, k), perm.cpu().numpy().view(np.uint32)
    assert st["distinct"] == len(np.unique(ku))
    assert abs(st["anc"] - oracle.anc(ku, pu)) < 1e-12


def test_trace_counts_are_consistent(ctx, room):
    """Visits depend on the warp a ray shares (a lane holding a parked leaf keeps descending),
    so the two orders may differ in work, never in the counts' internal consistency."""
    rng = np.random.default_rng(8)
    perm = torch.from_numpy(rng.permutation(room.n).astype(np.int32)).to(DEV)
    for c in (hcc.hcc_trace_counts(ctx, room.bvh_exact, room.org, room.dir),
              hcc.hcc_trace_counts(ctx, room.bvh_exact, room.org, room.dir, perm=perm)):
        assert c["node_visits"] > 0 and c["tri_tests"] > 0
        assert c["warp_node_steps"] <= c["node_visits"] <= 32 * c["warp_node_steps"]
        assert c["warp_leaf_steps"] > 0


def test_encode_special_rays(ctx, tiny):
    """Zero direction components, origins on box faces, NaN and Inf inputs."""
    cut = hcc.hcc_select_cut(ctx, tiny.bvh, 32, 0.125)
    ids = hcc.hcc_cut_info(cut)
    lo, hi = tiny.w.bvh.lo[ids], tiny.w.bvh.hi[ids]
    rng = np.random.default_rng(0)
    n = 600
    org = np.concatenate([rng.uniform(0, 1, (n, 3)), np.full((n, 1), 1e-4)], 1).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d[: n // 3, rng.integers(0, 3)] = 0.0
    d[n // 3: n // 2, :2] = 0.0
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    dir_ = np.concatenate([d, np.full((n, 1), np.inf)], 1).astype(np.float32)
    org[:50, :3] = lo[np.arange(50) % len(ids)]  # origins exactly on box corners
    org[50:60, 0] = np.nan
    dir_[60:70, 1] = np.inf
    dir_[70:80, 3] = np.nan
    o_t, d_t = torch.from_numpy(org).to(DEV), torch.from_numpy(dir_).to(DEV)
    try:
        for k in (32, 64):
            g = gpu_encode(ctx, tiny, "hcc", k, cut=cut, org=o_t, dir_=d_t)
            assert np.array_equal(g, oracle.encode_hcc(org, dir_, lo, hi, k))
        g = gpu_encode(ctx, tiny, "twopoint", 32, org=o_t, dir_=d_t)
        assert np.array_equal(g, oracle.encode_twopoint(org, dir_, tiny.w.bvh.lo[0], tiny.w.bvh.hi[0], 32))
        for k in (24, 64):
            g = gpu_encode(ctx, tiny, "origin_dir", k, org=o_t, dir_=d_t)
            assert np.array_equal(g, oracle.encode_origin_dir(org, dir_, tiny.w.bvh.lo[0], tiny.w.bvh.hi[0], k))
    finally:
        hcc.hcc_cut_destroy(cut)


# -------------------------------------------------------------------- sort

def _keys(kind, n, k, rng):
    top = (1 << k) - 1 if k < 64 else (1 << 64) - 1
    if kind == "uniform":
        return rng.integers(0, top, n, dtype=np.uint64, endpoint=True)
    if kind == "few":
        return rng.integers(0, min(4, top + 1), n, dtype=np.uint64)
    if kind == "equal":
        return np.full(n, min(top, 12345), np.uint64)
    if kind == "high_only":  # only the top digit varies: lower passes are skipped
        return (rng.integers(0, 256, n, dtype=np.uint64) << np.uint64(max(k - 8, 0))) & np.uint64(top)
    if kind == "distinct":
        return (rng.permutation(n).astype(np.uint64) * np.uint64(2654435761)) & np.uint64(top)
    raise ValueError(kind)


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 3583, 3584, 3585, 4096, 7169, 10752, 65537, 300_001])
def test_sort_sizes(ctx, n):
    rng = np.random.default_rng(n)
    for k in (32, 17):
        keys = _keys("uniform", n, k, rng)
        assert np.array_equal(gpu_sort(ctx, keys, k), oracle.stable_sort(keys))


@pytest.mark.parametrize("k", [1, 8, 16, 24, 31, 32, 33, 48, 64])
@pytest.mark.parametrize("kind", ["uniform", "few", "equal", "high_only", "distinct"])
def test_sort_key_widths(ctx, k, kind):
    rng = np.random.default_rng(k * 31 + len(kind))
    n = 100_003
    keys = _keys(kind, n, k, rng)
    assert np.array_equal(gpu_sort(ctx, keys, k), oracle.stable_sort(keys))


@pytest.mark.parametrize("k", [32, 64])
@pytest.mark.parametrize("n", [5, 622_591, 622_593, 2_490_369])
def test_sort_keys_not_16_byte_aligned(ctx, k, n):
    """Keys that start one element past a 16-byte boundary (the histogram
    then reads them one at a time) and sizes around the histogram's whole
    vector steps (608 blocks x 256 threads x 4 loads of 16 bytes)."""
    rng = np.random.default_rng(n + k)
    keys = _keys("uniform", n, k, rng)
    keys[::5] = keys[0]
    dt = np.int32 if k <= 32 else np.int64
    raw = np.zeros(n + 1, dtype=np.uint32 if k <= 32 else np.uint64)
    raw[1:] = keys.astype(raw.dtype)
    base = torch.from_numpy(raw.view(dt)).to(DEV)
    for kt in (base[1:], base[:n]):
        perm = torch.full((n,), -7, dtype=torch.int32, device=DEV)
        hcc.hcc_sort(ctx, kt, k, n, perm)
        hcc.hcc_sync(ctx)
        ref = kt.cpu().numpy().view(np.uint32 if k <= 32 else np.uint64).astype(np.uint64)
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), oracle.stable_sort(ref))


def test_sort_ignores_bits_above_key_bits(ctx):
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 2 ** 32 - 1, 50_000, dtype=np.uint64)
    k = 20
    g = gpu_sort(ctx, keys, k)
    assert np.array_equal(g, oracle.stable_sort(keys & np.uint64((1 << k) - 1)))


def test_sort_hcc_keys(ctx, room):
    cut = hcc.hcc_select_cut(ctx, room.bvh, 32, 0.125)
    try:
        g = gpu_encode(ctx, room, "hcc", 32, cut=cut)
    finally:
        hcc.hcc_cut_destroy(cut)
    assert np.array_equal(gpu_sort(ctx, g, 32), oracle.stable_sort(g))


@pytest.mark.parametrize("k", [32, 64])
@pytest.mark.parametrize("tile", [0, 5])
def test_sort_bounded_wait_runs_out_and_the_context_recovers(ctx, tile, k):
    """A tile that never publishes its counts (test hook) makes the next
    tile's look-back wait run out: hcc_sync reports HCC_ERR_TIMEOUT, every
    tile returns (the sort ends), and the next sort on the same context is
    the oracle's stable sort again."""
    rng = np.random.default_rng(77 + tile + k)
    n = 300_001  # 84 tiles of 3584 keys
    keys = _keys("uniform", n, k, rng)
    try:
        hcc.hcc_set_sort_wait_limit(ctx, 256)
        hcc.hcc_test_sort_withhold_tile(ctx, tile)
        with pytest.raises(hcc.HccError) as ei:
            gpu_sort(ctx, keys, k)
        assert ei.value.status == 6  # HCC_ERR_TIMEOUT
    finally:
        hcc.hcc_test_sort_withhold_tile(ctx)
        hcc.hcc_set_sort_wait_limit(ctx, 0)
    assert np.array_equal(gpu_sort(ctx, keys, k), oracle.stable_sort(keys))


# ------------------------------------------------------------------ gather

@pytest.mark.parametrize("n", [1, 33, 1000, 65_541])
def test_gather_bit_exact(ctx, n):
    rng = np.random.default_rng(n)
    org = rng.integers(-2 ** 31, 2 ** 31 - 1, (n, 4), dtype=np.int64).astype(np.int32).view(np.float32)
    dir_ = rng.integers(-2 ** 31, 2 ** 31 - 1, (n, 4), dtype=np.int64).astype(np.int32).view(np.float32)
    perm = rng.permutation(n).astype(np.uint32)
    oo, od = oracle.gather(org, dir_, perm)
    ti, td = torch.from_numpy(org.copy()).to(DEV), torch.from_numpy(dir_.copy()).to(DEV)
    po, pd = torch.zeros_like(ti), torch.zeros_like(td)
    hcc.hcc_gather(ctx, ti, td, torch.from_numpy(perm.view(np.int32)).to(DEV), po, pd)
    hcc.hcc_sync(ctx)
    assert po.cpu().numpy().tobytes() == oo.tobytes() and pd.cpu().numpy().tobytes() == od.tobytes()


# ------------------------------------------------------------- ray layouts

def _record_views(org, dir_, width=8, at=4):
    """The rays as rows of `width` floats: origin at 0..3, direction at at..at+3."""
    n = org.shape[0]
    rec = torch.full((n, width), float("nan"), dtype=torch.float32, device=DEV)
    rec[:, :4] = org
    rec[:, at:at + 4] = dir_
    return rec, rec[:, :4], rec[:, at:at + 4]


@pytest.mark.parametrize("width,at", [(8, 4), (12, 8)])
def test_strided_ray_layouts_give_the_same_keys_and_hits(ctx, room, width, at):
    """32-byte records (origin, direction) and a wider stride give bit for bit
    the keys, the gathered rays and the hit records of two packed arrays."""
    rec, o, d = _record_views(room.org, room.dir, width, at)
    cut = hcc.hcc_select_cut(ctx, room.bvh, 32, 0.125)
    try:
        for method, k in (("hcc", 32), ("twopoint", 30), ("origin", 30), ("origin_dir", 48)):
            c = cut if method == "hcc" else None
            assert np.array_equal(gpu_encode(ctx, room, method, k, cut=c, org=o, dir_=d),
                                  gpu_encode(ctx, room, method, k, cut=c)), method
        for kind in ("ppc", "mlhcc"):
            a, b = _keys_tensor(room.n, 32), _keys_tensor(room.n, 32)
            h = room.bvh_exact if kind == "ppc" else room.bvh
            c = hcc.hcc_select_cut_ml(ctx, room.bvh, 8, 8, 0.125) if kind == "mlhcc" else None
            try:
                hcc.hcc_encode(ctx, kind, h, c, o, d, 32, a)
                hcc.hcc_encode(ctx, kind, h, c, room.org, room.dir, 32, b)
                hcc.hcc_sync(ctx)
            finally:
                if c is not None:
                    hcc.hcc_cut_destroy(c)
            assert torch.equal(a, b), kind
        keys = _keys_tensor(room.n, 32)
        hcc.hcc_encode(ctx, "hcc", room.bvh, cut, o, d, 32, keys)
        perm = torch.empty(room.n, dtype=torch.int32, device=DEV)
        hcc.hcc_sort(ctx, keys, 32, room.n, perm)
    finally:
        hcc.hcc_cut_destroy(cut)
    ref = oracle.trace_bvh(room.w.bvh, room.w.rays.org, room.w.rays.dir)
    for layout in ("quantised", "exact", "wide"):
        compare_hits(gpu_trace(ctx, room, o, d, layout=layout), ref)
        bvh = {"quantised": room.bvh, "exact": room.bvh_exact, "wide": room.bvh_wide}[layout]
        hits = torch.zeros((room.n, 4), dtype=torch.int32, device=DEV)
        hcc.hcc_trace_sorted(ctx, bvh, o, d, perm, hits)
        hcc.hcc_sync(ctx)
        compare_hits(hcc.hits_to_numpy(hits), ref)
    # gathers between every pair of layouts: the oracle's gathered records, bit for bit
    p = perm.cpu().numpy().view(np.uint32)
    oo, od = oracle.gather(room.w.rays.org, room.w.rays.dir, p)
    packed_out = (torch.zeros_like(room.org), torch.zeros_like(room.dir))
    _, ro, rd = _record_views(torch.zeros_like(room.org), torch.zeros_like(room.dir), width, at)
    for src in ((room.org, room.dir), (o, d)):
        for dst in (packed_out, (ro, rd)):
            dst[0].zero_()
            dst[1].zero_()
            hcc.hcc_gather(ctx, src[0], src[1], perm, dst[0], dst[1])
            hcc.hcc_sync(ctx)
            assert dst[0].cpu().numpy().tobytes() == oo.tobytes()
            assert dst[1].cpu().numpy().tobytes() == od.tobytes()
    # the whole pipeline on records
    hits = torch.zeros((room.n, 4), dtype=torch.int32, device=DEV)
    cut = hcc.hcc_select_cut(ctx, room.bvh, 32, 0.125)
    try:
        hcc.hcc_run(ctx, "hcc", room.bvh, cut, o, d, 32, hits)
        hcc.hcc_sync(ctx)
    finally:
        hcc.hcc_cut_destroy(cut)
    compare_hits(hcc.hits_to_numpy(hits), ref)


def test_ray_stride_must_be_a_multiple_of_16(ctx, room):
    bad = torch.zeros((room.n, 6), dtype=torch.float32, device=DEV)  # 24-byte rows
    keys = _keys_tensor(room.n, 32)
    with pytest.raises(hcc.HccError) as ei:
        hcc.hcc_encode(ctx, "twopoint", room.bvh, None, bad[:, :4], bad[:, 2:6], 32, keys)
    assert ei.value.status == 1


# ------------------------------------------------------------------- trace

@pytest.mark.parametrize("layout", ["quantised", "exact", "wide"])
@pytest.mark.parametrize("which", ["tiny", "dense", "room"])
def test_trace_closest_matches_oracle(ctx, which, layout, request):
    sc = request.getfixturevalue(which)
    g = gpu_trace(ctx, sc, sc.org, sc.dir, layout=layout)
    o = oracle.trace_bvh(sc.w.bvh, sc.w.rays.org, sc.w.rays.dir)
    compare_hits(g, o)
    assert (g["prim"] >= 0).mean() > 0.2


@pytest.mark.parametrize("layout", ["quantised", "exact", "wide"])
def test_trace_matches_brute_force_definition(ctx, dense, layout):
    g = gpu_trace(ctx, dense, dense.org, dense.dir, layout=layout)
    o = oracle.trace_brute(dense.w.tris, dense.w.rays.org, dense.w.rays.dir)
    compare_hits(g, o)


@pytest.mark.parametrize("layout", ["quantised", "exact", "wide"])
def test_trace_any_hit_shadow_rays(ctx, room, layout):
    sh = room.w.shadow
    org, dir_ = torch.from_numpy(sh.org).to(DEV), torch.from_numpy(sh.dir).to(DEV)
    g = gpu_trace(ctx, room, org, dir_, any_hit=True, layout=layout)
    o = oracle.trace_bvh(room.w.bvh, sh.org, sh.dir)
    occl_g, occl_o = g["prim"] >= 0, o["prim"] >= 0
    assert np.array_equal(occl_g, occl_o)
    assert 0.01 < occl_g.mean() < 0.99
    for i in np.nonzero(occl_g)[0][:500]:
        ok, t, u, v = oracle.intersect(sh.org[i, :3], sh.dir[i, :3], sh.org[i, 3], sh.dir[i, 3],
                                       room.w.tris[g["prim"][i]])
        assert ok and np.float32(t) == g["t"][i]


@pytest.mark.parametrize("layout", ["quantised", "exact", "wide"])
def test_trace_special_rays(ctx, dense, layout):
    rng = np.random.default_rng(1)
    n = 400
    org = np.concatenate([rng.uniform(0, 1, (n, 3)), np.full((n, 1), 1e-4)], 1).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d[:100, 0] = 0.0
    d[100:150, :2] = 0.0
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    dir_ = np.concatenate([d, np.full((n, 1), np.inf)], 1).astype(np.float32)
    dir_[150:200, 3] = 0.3          # finite tmax
    org[200:210, 1] = np.nan        # invalid inputs are misses on both sides
    dir_[210:220, 2] = np.nan
    org[220:230, 3] = np.inf        # empty interval
    g = gpu_trace(ctx, dense, torch.from_numpy(org).to(DEV), torch.from_numpy(dir_).to(DEV), layout=layout)
    o = oracle.trace_bvh(dense.w.bvh, org, dir_)
    compare_hits(g, o)
    assert np.all(g["prim"][200:230] == -1)


def test_trace_scatter_and_reorder_invariance(ctx, room):
    rng = np.random.default_rng(3)
    perm = rng.permutation(room.n).astype(np.uint32)
    po, pd = oracle.gather(room.w.rays.org, room.w.rays.dir, perm)
    plain = gpu_trace(ctx, room, room.org, room.dir)
    perm_t = torch.from_numpy(perm.view(np.int32)).to(DEV)
    scattered = gpu_trace(ctx, room, torch.from_numpy(po).to(DEV), torch.from_numpy(pd).to(DEV), scatter=perm_t)
    assert plain.tobytes() == scattered.tobytes()
    # fetch through the permutation (no separate gather): same records
    hits = torch.zeros((room.n, 4), dtype=torch.int32, device=DEV)
    hcc.hcc_trace_sorted(ctx, room.bvh_exact, room.org, room.dir, perm_t, hits)
    hcc.hcc_sync(ctx)
    assert hcc.hits_to_numpy(hits).tobytes() == plain.tobytes()


# ---------------------------------------------------------------- pipeline

def run_pipeline(ctx, sc, method, k=32, C=32, any_hit=False):
    cut = hcc.hcc_select_cut(ctx, sc.bvh, C, 0.125) if method == "hcc" else None
    hits = torch.zeros((sc.n, 4), dtype=torch.int32, device=DEV)
    try:
        hcc.hcc_run(ctx, method, sc.bvh, cut, sc.org, sc.dir, k, hits, any_hit=any_hit)
        hcc.hcc_sync(ctx)
    finally:
        if cut is not None:
            hcc.hcc_cut_destroy(cut)
    return hcc.hits_to_numpy(hits)


@pytest.mark.parametrize("which", ["tiny", "room"])
def test_pipeline_methods_agree_bit_for_bit(ctx, which, request):
    sc = request.getfixturevalue(which)
    base = run_pipeline(ctx, sc, "nosort")
    for method, k, C in (("hcc", 32, 32), ("hcc", 32, 256), ("hcc", 64, 64), ("hcc", 16, 4096), ("twopoint", 32, 0),
                         ("twopoint", 64, 0), ("origin", 30, 0), ("origin_dir", 48, 0)):
        assert run_pipeline(ctx, sc, method, k, C).tobytes() == base.tobytes(), (method, k, C)
    compare_hits(base, oracle.trace_bvh(sc.w.bvh, sc.w.rays.org, sc.w.rays.dir))


def test_pipeline_host_buffers(ctx, room):
    cut = hcc.hcc_select_cut(ctx, room.bvh, 32, 0.125)
    try:
        out = np.zeros(room.n, hcc.HIT_DTYPE)
        hcc.hcc_run_host(ctx, "hcc", room.bvh, cut, room.w.rays.org, room.w.rays.dir, 32, out)
    finally:
        hcc.hcc_cut_destroy(cut)
    assert out.tobytes() == run_pipeline(ctx, room, "nosort").tobytes()


def test_deterministic(ctx, room):
    a = run_pipeline(ctx, room, "hcc")
    b = run_pipeline(ctx, room, "hcc")
    assert a.tobytes() == b.tobytes()


# ------------------------------------------------------------- edge cases

def test_empty_inputs_are_noops(ctx, tiny):
    e = torch.zeros((0, 4), dtype=torch.float32, device=DEV)
    k = torch.zeros(0, dtype=torch.int32, device=DEV)
    h = torch.zeros((0, 4), dtype=torch.int32, device=DEV)
    cut = hcc.hcc_select_cut(ctx, tiny.bvh, 32, 0.125)
    hcc.hcc_encode(ctx, "hcc", tiny.bvh, cut, e, e, 32, k)
    hcc.hcc_sort(ctx, k, 32, 0, k)
    hcc.hcc_gather(ctx, e, e, k, e, e)
    hcc.hcc_trace(ctx, tiny.bvh, e, e, h)
    hcc.hcc_run(ctx, "hcc", tiny.bvh, cut, e, e, 32, h)
    hcc.hcc_sync(ctx)
    hcc.hcc_cut_destroy(cut)


def test_invalid_arguments_are_rejected(ctx, tiny):
    cut = hcc.hcc_select_cut(ctx, tiny.bvh, 32, 0.125)
    keys = torch.zeros(tiny.n, dtype=torch.int32, device=DEV)
    try:
        for bad_k in (0, 65):
            with pytest.raises(hcc.HccError) as ei:
                hcc.hcc_encode(ctx, "hcc", tiny.bvh, cut, tiny.org, tiny.dir, bad_k, keys)
            assert ei.value.status == 1
        with pytest.raises(hcc.HccError):
            hcc.hcc_encode(ctx, "hcc", tiny.bvh, None, tiny.org, tiny.dir, 32, keys)  # HCC without a cut
        with pytest.raises(hcc.HccError):
            hcc.hcc_encode(ctx, "nosort", tiny.bvh, cut, tiny.org, tiny.dir, 32, keys)
        with pytest.raises(hcc.HccError):
            hcc.hcc_select_cut(ctx, tiny.bvh, 0, 0.125)
        with pytest.raises(hcc.HccError):
            hcc.hcc_select_cut(ctx, tiny.bvh, 8, -1.0)
        with pytest.raises(hcc.HccError):  # keys and perm overlap
            hcc.hcc_sort(ctx, keys, 32, tiny.n, keys)
        with pytest.raises(hcc.HccError):  # misaligned ray stream
            hcc.hcc_trace(ctx, tiny.bvh, tiny.org.view(-1)[1:].view(-1)[: 4 * (tiny.n - 1)].view(-1, 4), tiny.dir[1:],
                          torch.zeros((tiny.n - 1, 4), dtype=torch.int32, device=DEV))
    finally:
        hcc.hcc_cut_destroy(cut)
    hcc.hcc_sync(ctx)  # nothing was launched by the rejected calls


def _chain_bvh(depth):
    """Every node's box is the whole scene; left = deeper internal node, right = leaf."""
    tris = gen.random_tris(1, depth + 1, mu=-1.0)
    lo = np.tile(tris.reshape(-1, 3).min(0), (2 * depth + 1, 1)).astype(np.float32)
    hi = np.tile(tris.reshape(-1, 3).max(0), (2 * depth + 1, 1)).astype(np.float32)
    left = np.full(2 * depth + 1, -1, np.int32)
    right = np.full(2 * depth + 1, -1, np.int32)
    first = np.zeros(2 * depth + 1, np.uint32)
    count = np.zeros(2 * depth + 1, np.uint32)
    # internal nodes 0..depth-1 at even ids 2i; leaves at odd ids
    for i in range(depth):
        node = 2 * i
        left[node] = 2 * (i + 1) if i + 1 < depth else 2 * depth
        right[node] = 2 * i + 1
        first[2 * i + 1], count[2 * i + 1] = i, 1
    first[2 * depth], count[2 * depth] = depth, 1
    return gen.BVH(lo, hi, left, right, first, count, np.arange(depth + 1, dtype=np.uint32), tris, depth)


@pytest.mark.parametrize("layout", ["quantised", "exact", "wide"])
def test_stack_overflow_is_reported_and_context_survives(ctx, tiny, layout):
    deep = _chain_bvh(100)
    h = hcc.hcc_bvh_upload(ctx, deep, layout=layout)
    assert hcc.hcc_bvh_info(h)["depth"] == 100
    c = deep.tris.reshape(-1, 3).mean(0)
    org = torch.tensor([[c[0], c[1], c[2] - 5.0, 0.0]], dtype=torch.float32, device=DEV)
    dir_ = torch.tensor([[0.0, 0.0, 1.0, float("inf")]], dtype=torch.float32, device=DEV)
    hits = torch.zeros((1, 4), dtype=torch.int32, device=DEV)
    hcc.hcc_trace(ctx, h, org, dir_, hits)
    with pytest.raises(hcc.HccError) as ei:
        hcc.hcc_sync(ctx)
    assert ei.value.status == 5
    assert int(hits[0, 0]) == -1
    hcc.hcc_bvh_destroy(h)
    # the context keeps working
    g = gpu_trace(ctx, tiny, tiny.org, tiny.dir)
    compare_hits(g, oracle.trace_bvh(tiny.w.bvh, tiny.w.rays.org, tiny.w.rays.dir))


@pytest.mark.parametrize("layout", ["quantised", "exact"])
def test_trace_shape_stack_depth_is_honoured(ctx, tiny, layout):
    """A 40-level chain fits 48 or 64 stack entries but not 32: the shallow
    shape reports the overflow (and a miss), the deeper ones find the hit."""
    deep = _chain_bvh(40)
    h = hcc.hcc_bvh_upload(ctx, deep, layout=layout)
    c = deep.tris.reshape(-1, 3).mean(0)
    org = torch.tensor([[c[0], c[1], c[2] - 5.0, 0.0]], dtype=torch.float32, device=DEV)
    dir_ = torch.tensor([[0.0, 0.0, 1.0, float("inf")]], dtype=torch.float32, device=DEV)
    ref = oracle.trace_bvh(deep, org.cpu().numpy(), dir_.cpu().numpy())
    try:
        for block in (64, 128, 256):
            for stack in (32, 48, 64):
                hcc.hcc_set_trace_shape(ctx, block, stack)
                hits = torch.zeros((1, 4), dtype=torch.int32, device=DEV)
                hcc.hcc_trace(ctx, h, org, dir_, hits)
                if stack == 32:
                    with pytest.raises(hcc.HccError) as ei:
                        hcc.hcc_sync(ctx)
                    assert ei.value.status == 5 and int(hits[0, 0]) == -1
                else:
                    hcc.hcc_sync(ctx)
                    compare_hits(hcc.hits_to_numpy(hits), ref)
    finally:
        hcc.hcc_set_trace_shape(ctx, 0, 0)
        hcc.hcc_bvh_destroy(h)


@pytest.mark.parametrize("which", ["tiny", "room"])
def test_trace_schedules_give_the_same_records(ctx, which, request):
    """One thread per ray and the persistent trace with ray replacement return
    the same closest-hit records (and the same occlusion for any hit)."""
    sc = request.getfixturevalue(which)
    ref = oracle.trace_bvh(sc.w.bvh, sc.w.rays.org, sc.w.rays.dir)
    ref_any = oracle.trace_bvh(sc.w.bvh, sc.w.rays.org, sc.w.rays.dir, any_hit=True)
    keys = torch.empty(sc.n, dtype=torch.int32, device=DEV)
    perm = torch.empty(sc.n, dtype=torch.int32, device=DEV)
    cut = hcc.hcc_select_cut(ctx, sc.bvh_exact, 32, 0.125)
    hcc.hcc_encode(ctx, "hcc", sc.bvh_exact, cut, sc.org, sc.dir, 32, keys)
    hcc.hcc_sort(ctx, keys, 32, sc.n, perm)
    try:
        for schedule in ("per_ray", "refill", "auto"):
            hcc.hcc_set_trace_schedule(ctx, schedule)
            for bvh in (sc.bvh, sc.bvh_exact, sc.bvh_wide):
                hits = torch.zeros((sc.n, 4), dtype=torch.int32, device=DEV)
                hcc.hcc_trace(ctx, bvh, sc.org, sc.dir, hits)
                hcc.hcc_sync(ctx)
                assert hcc.hits_to_numpy(hits).tobytes() == ref.tobytes(), schedule
                hits.zero_()
                hcc.hcc_trace_sorted(ctx, bvh, sc.org, sc.dir, perm, hits)
                hcc.hcc_sync(ctx)
                assert hcc.hits_to_numpy(hits).tobytes() == ref.tobytes(), schedule
                hits.zero_()
                hcc.hcc_trace(ctx, bvh, sc.org, sc.dir, hits, any_hit=True)
                hcc.hcc_sync(ctx)
                assert np.array_equal(hcc.hits_to_numpy(hits)["prim"] >= 0, ref_any["prim"] >= 0), schedule
            c = hcc.hcc_trace_counts(ctx, sc.bvh_exact, sc.org, sc.dir, perm=perm)
            assert c["warp_node_steps"] <= c["node_visits"] <= 32 * c["warp_node_steps"]
        with pytest.raises(hcc.HccError):
            hcc.hcc_set_trace_schedule(ctx, 7)
    finally:
        hcc.hcc_set_trace_schedule(ctx, "auto")
        hcc.hcc_cut_destroy(cut)


@pytest.fixture(scope="module")
def chunk_room():
    w = gen.room_workload(2, target_tris=60_000, W=1024, H=576, spp=8, shadow=False)
    assert w.rays.n >= 1 << 22
    return w


# the whole wavefront (chunks of 2^20, 2^21, then 2^22 and the rest), one ray
# more than a single pass (2^20 + 2^21 + 2^20 + 1), and four chunks with a
# 5-ray tail
@pytest.mark.parametrize("n_rays", [None, (1 << 22) + 1, (1 << 20) + (1 << 21) + (1 << 22) + 5])
def test_run_host_pipeline_over_chunks(ctx, chunk_room, n_rays):
    """Rays above 2^22 go through the two-stream chunked host pipeline: every
    hit equals the device pipeline's, and a sample equals the oracle's."""
    w = chunk_room
    org_np, dir_np = w.rays.org, w.rays.dir
    if n_rays is not None:  # repeat the wavefront's rays to reach n_rays
        reps = -(-n_rays // w.rays.n)
        org_np = np.ascontiguousarray(np.concatenate([org_np] * reps)[:n_rays])
        dir_np = np.ascontiguousarray(np.concatenate([dir_np] * reps)[:n_rays])
    n = org_np.shape[0]
    bvh = hcc.hcc_bvh_upload(ctx, w.bvh, layout="exact")
    cut = hcc.hcc_select_cut(ctx, bvh, 32, 0.125)
    try:
        org = torch.from_numpy(org_np).pin_memory()
        dir_ = torch.from_numpy(dir_np).pin_memory()
        for method in ("hcc", "nosort"):
            h_host = torch.zeros((n, 4), dtype=torch.int32).pin_memory()
            hcc.hcc_run_host(ctx, method, bvh, cut, org, dir_, 32, h_host)
            d_hits = torch.zeros((n, 4), dtype=torch.int32, device=DEV)
            hcc.hcc_run(ctx, method, bvh, cut, org.to(DEV), dir_.to(DEV), 32, d_hits)
            hcc.hcc_sync(ctx)
            assert torch.equal(h_host, d_hits.cpu()), method
        idx = np.random.default_rng(5).choice(n, 3000, replace=False)
        idx = np.concatenate([idx, np.arange(n - 5, n)])  # the last chunk's rays
        ref = oracle.trace_bvh(w.bvh, org_np[idx], dir_np[idx])
        assert hcc.hits_to_numpy(h_host)[idx].tobytes() == ref.tobytes()
        # the chunked path reports errors like the one-pass path
        with pytest.raises(hcc.HccError):
            hcc.hcc_run_host(ctx, "hcc", bvh, None, org, dir_, 32, h_host)
    finally:
        hcc.hcc_cut_destroy(cut)
        hcc.hcc_bvh_destroy(bvh)


def test_encode_with_an_inverted_cut_box_takes_the_general_test(ctx, tiny):
    """A cut box with lo > hi on an axis voids the sign-selected slab bounds
    (they assume lo <= hi); the encoder must notice and give the oracle's keys."""
    import copy
    b = copy.deepcopy(tiny.w.bvh)
    b.lo[0, 1], b.hi[0, 1] = b.hi[0, 1], b.lo[0, 1]  # root box inverted on y
    h = hcc.hcc_bvh_upload(ctx, b, layout="exact")
    cut = hcc.hcc_select_cut(ctx, h, 1, 0.125)  # the cut is the root alone
    try:
        assert hcc.hcc_cut_info(cut).tolist() == [0]
        keys = torch.zeros(tiny.n, dtype=torch.int32, device=DEV)
        hcc.hcc_encode(ctx, "hcc", h, cut, tiny.org, tiny.dir, 8, keys)
        hcc.hcc_sync(ctx)
        g = keys.cpu().numpy().view(np.uint32).astype(np.uint64)
        o = oracle.encode_hcc(tiny.w.rays.org, tiny.w.rays.dir, b.lo[[0]], b.hi[[0]], 8)
        assert np.array_equal(g, o)
        # min/max make the test symmetric in lo and hi, so every ray still meets the box;
        # near/far bounds picked by direction sign (lo near for a positive direction)
        # would have missed it for most rays
        assert np.count_nonzero(o) == tiny.n
    finally:
        hcc.hcc_cut_destroy(cut)
        hcc.hcc_bvh_destroy(h)


def test_full_size_headline_configuration():
    """The benchmark's workload and launch configuration (1920x1080x8spp room,
    16,588,800 rays, ~1M triangles, cut 32, 32-bit keys, exact nodes): keys on a
    sample against the oracle, the whole permutation by the properties of a
    stable sort, hits on a sample against the oracle and all hits against NoSort."""
    w = gen.room_workload(1, target_tris=1_000_000, W=1920, H=1080, spp=8, shadow=False)
    n = w.rays.n
    assert n == 16_588_800
    c = hcc.hcc_create(0)
    bvh = hcc.hcc_bvh_upload(c, w.bvh, layout="exact")
    cut = hcc.hcc_select_cut(c, bvh, 32, 0.125)
    try:
        ids = hcc.hcc_cut_info(cut)
        assert ids.tolist() == oracle.select_cut(w.bvh, 32).tolist()
        org = torch.from_numpy(w.rays.org).to(DEV)
        dir_ = torch.from_numpy(w.rays.dir).to(DEV)
        keys = torch.empty(n, dtype=torch.int32, device=DEV)
        perm = torch.empty(n, dtype=torch.int32, device=DEV)
        hcc.hcc_encode(c, "hcc", bvh, cut, org, dir_, 32, keys)
        hcc.hcc_sort(c, keys, 32, n, perm)
        hits = torch.empty((n, 4), dtype=torch.int32, device=DEV)
        hcc.hcc_trace_sorted(c, bvh, org, dir_, perm, hits)
        hits0 = torch.empty_like(hits)
        hcc.hcc_trace(c, bvh, org, dir_, hits0)
        hcc.hcc_sync(c)
        assert torch.equal(hits, hits0)
        k = keys.cpu().numpy().view(np.uint32).astype(np.uint64)
        p = perm.cpu().numpy().view(np.uint32).astype(np.int64)
        rng = np.random.default_rng(11)
        idx = rng.choice(n, 20_000, replace=False)
        ref_k = oracle.encode_hcc(w.rays.org[idx], w.rays.dir[idx], w.bvh.lo[ids], w.bvh.hi[ids], 32)
        compare_keys(k[idx], ref_k, lambda b: oracle.key_margin(w.rays.org[idx[b]], w.rays.dir[idx[b]],
                                                                 w.bvh.lo[ids], w.bvh.hi[ids], 32))
        # the permutation: every id once, keys non-decreasing, equal keys in id order
        assert np.array_equal(np.sort(p), np.arange(n))
        ks = k[p]
        assert np.all(ks[1:] >= ks[:-1])
        same = ks[1:] == ks[:-1]
        assert np.all(p[1:][same] > p[:-1][same])
        sample = idx[:3000]
        ref_h = oracle.trace_bvh(w.bvh, w.rays.org[sample], w.rays.dir[sample])
        compare_hits(hcc.hits_to_numpy(hits)[sample], ref_h)
    finally:
        hcc.hcc_cut_destroy(cut)
        hcc.hcc_bvh_destroy(bvh)
        hcc.hcc_destroy(c)


@pytest.mark.parametrize("fraction", [0.0, 0.1, 0.5, 1.0])
def test_twopoint_distance_fraction_matches_oracle(ctx, room, fraction):
    try:
        hcc.hcc_set_twopoint_distance(ctx, fraction)
        g = gpu_encode(ctx, room, "twopoint", 48)
    finally:
        hcc.hcc_set_twopoint_distance(ctx, 0.25)
    o = oracle.encode_twopoint(room.w.rays.org, room.w.rays.dir, room.w.bvh.lo[0], room.w.bvh.hi[0], 48,
                               fraction=fraction)
    assert np.array_equal(g, o)
    with pytest.raises(hcc.HccError):
        hcc.hcc_set_twopoint_distance(ctx, -1.0)
