"""Method variants on the GPU against the CPU oracle (needs a GB300): the
multi-level hierarchy cut code (Sec. 4.3, Algorithm 3), regular grid
encoding (Sec. 5) and the prefix path code (Sec. 4.1).

Cut ids and grid boxes must be identical; keys bit-exact except on rays whose
slab-test margin against a box that drives a bit is below 1e-6 (counted, at
most one in a thousand); every reordered pipeline must give the NoSort hits.
"""
import numpy as np
import pytest

import oracle
from paper_2305_16652_gb300 import gen, hcc
from parity import compare_hits, compare_keys
from test_gpu_parity import Scene, _chain_bvh, gpu_encode

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    c = hcc.hcc_create(0)
    yield c
    hcc.hcc_destroy(c)


@pytest.fixture(scope="module")
def tiny(ctx):
    return Scene(ctx, gen.tiny_workload(0))


@pytest.fixture(scope="module")
def room(ctx):
    return Scene(ctx, gen.room_workload(1, target_tris=60_000, W=160, H=90, spp=2))


def _margin_all(org, dir_, lo, hi):
    """Smallest slab margin of each ray over all given boxes."""
    m = np.full(org.shape[0], np.inf)
    for c in range(0, lo.shape[0], 64):
        m = np.minimum(m, oracle.key_margin(org, dir_, lo[c:c + 64], hi[c:c + 64], 64))
    return m


def _check_keys(g, o, org, dir_, lo, hi, n):
    assert len(g) == n
    compare_keys(g, o, lambda b: _margin_all(org[b], dir_[b], lo, hi))


# --------------------------------------------------------------------- MLHCC

@pytest.mark.parametrize("T,L", [(8, 8), (16, 16), (4, 32), (32, 2), (1, 8), (2, 40), (32, 32)])
@pytest.mark.parametrize("which", ["tiny", "room"])
def test_mlhcc_cut_matches_oracle(ctx, which, T, L, request):
    sc = request.getfixturevalue(which)
    cut = hcc.hcc_select_cut_ml(ctx, sc.bvh, T, L, 0.125)
    try:
        top, low, tf, lf = hcc.hcc_cut_ml_info(cut)
    finally:
        hcc.hcc_cut_destroy(cut)
    ref_top, ref_low = oracle.select_cut_ml(sc.w.bvh, T, L)
    assert (tf, lf) == (T, L)
    assert top.tolist() == ref_top.tolist()
    assert np.array_equal(low, ref_low)


@pytest.mark.parametrize("T,L,k", [(8, 8, 16), (16, 16, 32), (8, 8, 24), (16, 16, 48), (32, 32, 64), (4, 28, 32)])
@pytest.mark.parametrize("which", ["tiny", "room"])
def test_mlhcc_keys_match_oracle(ctx, which, T, L, k, request):
    sc = request.getfixturevalue(which)
    cut = hcc.hcc_select_cut_ml(ctx, sc.bvh, T, L, 0.125)
    try:
        top, low, _, _ = hcc.hcc_cut_ml_info(cut)
        g = gpu_encode(ctx, sc, "mlhcc", k, cut=cut)
    finally:
        hcc.hcc_cut_destroy(cut)
    b = sc.w.bvh
    o = oracle.encode_mlhcc(sc.w.rays.org, sc.w.rays.dir, T, b.lo[top], b.hi[top], b.lo[low], b.hi[low], k)
    boxes = np.concatenate([top, low.reshape(-1)])
    _check_keys(g, o, sc.w.rays.org, sc.w.rays.dir, b.lo[boxes], b.hi[boxes], sc.n)
    assert len(np.unique(g)) > 1
    if k > T + L:
        assert np.all(g % (np.uint64(1) << np.uint64(k - T - L)) == 0)


def test_mlhcc_special_rays_and_bad_arguments(ctx, tiny):
    rng = np.random.default_rng(3)
    n = 500
    org = np.concatenate([rng.uniform(0, 1, (n, 3)), np.full((n, 1), 1e-4)], 1).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d[: n // 3, 1] = 0.0
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    dir_ = np.concatenate([d, np.full((n, 1), np.inf)], 1).astype(np.float32)
    org[40:50, 2] = np.nan
    dir_[50:60, 3] = np.nan
    cut = hcc.hcc_select_cut_ml(ctx, tiny.bvh, 16, 16, 0.125)
    o_t, d_t = torch.from_numpy(org).to(DEV), torch.from_numpy(dir_).to(DEV)
    try:
        top, low, _, _ = hcc.hcc_cut_ml_info(cut)
        g = gpu_encode(ctx, tiny, "mlhcc", 32, cut=cut, org=o_t, dir_=d_t)
        b = tiny.w.bvh
        assert np.array_equal(g, oracle.encode_mlhcc(org, dir_, 16, b.lo[top], b.hi[top], b.lo[low], b.hi[low], 32))
        keys = torch.zeros(n, dtype=torch.int32, device=DEV)
        with pytest.raises(hcc.HccError):  # 16 + 16 bits do not fit 24
            hcc.hcc_encode(ctx, "mlhcc", tiny.bvh, cut, o_t, d_t, 24, keys)
        one = hcc.hcc_select_cut(ctx, tiny.bvh, 32, 0.125)
        with pytest.raises(hcc.HccError):  # a one-level cut
            hcc.hcc_encode(ctx, "mlhcc", tiny.bvh, one, o_t, d_t, 32, keys)
        with pytest.raises(hcc.HccError):
            hcc.hcc_cut_ml_info(one)
        hcc.hcc_cut_destroy(one)
    finally:
        hcc.hcc_cut_destroy(cut)
    for T, L in ((0, 8), (8, 0), (40, 25)):
        with pytest.raises(hcc.HccError):
            hcc.hcc_select_cut_ml(ctx, tiny.bvh, T, L, 0.125)
    # no node holds enough leaves: an empty top level, every key 0
    cut = hcc.hcc_select_cut_ml(ctx, tiny.bvh, 2, 62, 0.125)
    try:
        top, low, _, _ = hcc.hcc_cut_ml_info(cut)
        assert top.size == oracle.select_cut_ml(tiny.w.bvh, 2, 62)[0].size
    finally:
        hcc.hcc_cut_destroy(cut)


# ---------------------------------------------------------------- grid

@pytest.mark.parametrize("cells,k", [(1, 8), (7, 8), (32, 32), (64, 64), (48, 40)])
@pytest.mark.parametrize("which", ["tiny", "room"])
def test_grid_matches_oracle(ctx, which, cells, k, request):
    sc = request.getfixturevalue(which)
    b = sc.w.bvh
    cut = hcc.hcc_select_grid(ctx, sc.bvh, cells)
    try:
        lo, hi = hcc.hcc_cut_boxes(cut)
        g = gpu_encode(ctx, sc, "hcc", k, cut=cut)
    finally:
        hcc.hcc_cut_destroy(cut)
    rlo, rhi, _ = oracle.grid_cells(b.lo[0], b.hi[0], cells)
    assert lo.tobytes() == rlo.tobytes() and hi.tobytes() == rhi.tobytes()
    o = oracle.encode_hcc(sc.w.rays.org, sc.w.rays.dir, rlo, rhi, k)
    _check_keys(g, o, sc.w.rays.org, sc.w.rays.dir, rlo, rhi, sc.n)
    with pytest.raises(hcc.HccError):
        hcc.hcc_select_grid(ctx, sc.bvh, 65)


# ----------------------------------------------------------------- PPC

@pytest.mark.parametrize("k", [1, 2, 16, 31, 32, 33, 48, 64])
@pytest.mark.parametrize("which", ["tiny", "room"])
def test_ppc_matches_oracle(ctx, which, k, request):
    sc = request.getfixturevalue(which)
    keys = torch.zeros(sc.n, dtype=torch.int32 if k <= 32 else torch.int64, device=DEV)
    hcc.hcc_encode(ctx, "ppc", sc.bvh_exact, None, sc.org, sc.dir, k, keys)
    hcc.hcc_sync(ctx)
    g = keys.cpu().numpy().view(np.uint32 if k <= 32 else np.uint64).astype(np.uint64)
    o = oracle.encode_ppc(sc.w.rays.org, sc.w.rays.dir, sc.w.bvh, k)
    b = sc.w.bvh
    compare_keys(g, o, lambda i: _margin_all(sc.w.rays.org[i], sc.w.rays.dir[i], b.lo, b.hi))
    if k >= 16:
        assert len(np.unique(g)) > 10


def test_ppc_deep_and_degenerate_trees(ctx, tiny):
    # a chain 100 levels deep: the walk is cut off by the key length, never by a stack
    deep = _chain_bvh(100)
    h = hcc.hcc_bvh_upload(ctx, deep, layout="exact")
    c = deep.tris.reshape(-1, 3).mean(0)
    org = np.array([[c[0], c[1], c[2] - 5.0, 0.0], [c[0] + 50, c[1], c[2], 0.0]], np.float32)
    dir_ = np.array([[0.0, 0.0, 1.0, np.inf], [0.0, 1.0, 0.0, np.inf]], np.float32)
    keys = torch.zeros(2, dtype=torch.int64, device=DEV)
    hcc.hcc_encode(ctx, "ppc", h, None, torch.from_numpy(org).to(DEV), torch.from_numpy(dir_).to(DEV), 64, keys)
    hcc.hcc_sync(ctx)
    g = keys.cpu().numpy().view(np.uint64)
    assert np.array_equal(g, oracle.encode_ppc(org, dir_, deep, 64))
    assert int(g[0]) == (1 << 64) - 1 and int(g[1]) == 0
    hcc.hcc_bvh_destroy(h)
    # a single leaf: one test
    one = gen.build_bvh(gen.random_tris(0, 1))
    h = hcc.hcc_bvh_upload(ctx, one, layout="exact")
    org = tiny.w.rays.org[:64]
    dir_ = tiny.w.rays.dir[:64]
    keys = torch.zeros(64, dtype=torch.int32, device=DEV)
    hcc.hcc_encode(ctx, "ppc", h, None, torch.from_numpy(org).to(DEV), torch.from_numpy(dir_).to(DEV), 16, keys)
    hcc.hcc_sync(ctx)
    assert np.array_equal(keys.cpu().numpy().view(np.uint32), oracle.encode_ppc(org, dir_, one, 16).astype(np.uint32))
    hcc.hcc_bvh_destroy(h)
    # the quantised layout has no exact boxes to test
    with pytest.raises(hcc.HccError) as ei:
        hcc.hcc_encode(ctx, "ppc", tiny.bvh, None, tiny.org, tiny.dir, 32,
                       torch.zeros(tiny.n, dtype=torch.int32, device=DEV))
    assert ei.value.status == 4


# ------------------------------------------------------------ pipelines

@pytest.mark.parametrize("layout", ["exact", "quantised", "wide"])
def test_variant_pipelines_give_the_nosort_hits(ctx, room, layout):
    bvh = {"exact": room.bvh_exact, "quantised": room.bvh, "wide": room.bvh_wide}[layout]
    hits0 = torch.zeros((room.n, 4), dtype=torch.int32, device=DEV)
    hcc.hcc_run(ctx, "nosort", bvh, None, room.org, room.dir, 32, hits0)
    ml = hcc.hcc_select_cut_ml(ctx, bvh, 16, 16, 0.125)
    grid = hcc.hcc_select_grid(ctx, bvh, 32)
    cases = [("mlhcc", ml, 32), ("mlhcc", ml, 48), ("hcc", grid, 32)]
    if layout == "exact":
        cases += [("ppc", None, 32), ("ppc", None, 64)]
    else:  # the prefix path code walks exact BVH2 nodes only
        keys = torch.zeros(room.n, dtype=torch.int32, device=DEV)
        with pytest.raises(hcc.HccError) as ei:
            hcc.hcc_encode(ctx, "ppc", bvh, None, room.org, room.dir, 32, keys)
        assert ei.value.status == 4
    try:
        for method, cut, k in cases:
            hits = torch.zeros_like(hits0)
            hcc.hcc_run(ctx, method, bvh, cut, room.org, room.dir, k, hits)
            hcc.hcc_sync(ctx)
            assert torch.equal(hits, hits0), (method, k)
        ref = oracle.trace_bvh(room.w.bvh, room.w.rays.org, room.w.rays.dir)
        compare_hits(hcc.hits_to_numpy(hits0), ref)
        # batches take only the keys of the batched kernels
        offsets = np.array([0, room.n], np.uint64)
        batch = hcc.hcc_batch_create(ctx, [bvh], [ml], offsets)
        try:
            with pytest.raises(hcc.HccError) as ei:
                hcc.hcc_batch_run(ctx, batch, "mlhcc", room.org, room.dir, 32, hits0)
            assert ei.value.status == 4
        finally:
            hcc.hcc_batch_destroy(batch)
    finally:
        hcc.hcc_cut_destroy(ml)
        hcc.hcc_cut_destroy(grid)
