"""Node layouts on small and unusual trees (needs a GB300).

The quantised and exact BVH2 layouts and the 4-ary layout collapsed from the
BVH2 must give the closest-hit records of the definition -- brute force over
all triangles (Sec. 3.1 closest hit, Moller-Trumbore) -- on trees whose root
is a leaf, whose 4-ary nodes hold two or three children, and whose boxes are
given with lo > hi on an axis (the same slab to a min/max slab test; the
upload stores them swapped).  Any-hit answers must agree with the definition
on whether a ray is occluded and report a triangle the ray really meets.
"""
import numpy as np
import pytest

import oracle
from paper_2305_16652_gb300 import gen, hcc
from parity import compare_hits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
LAYOUTS = ("quantised", "exact", "wide")


@pytest.fixture(scope="module")
def ctx():
    c = hcc.hcc_create(0)
    yield c
    hcc.hcc_destroy(c)


def _rays(seed, n, tris, shadow=False):
    """Rays from around the scene: half aimed at a triangle's centroid, half
    in uniform directions; shadow rays stop short of a random distance."""
    rng = np.random.default_rng(seed)
    v = tris.reshape(-1, 3).astype(np.float64)
    lo, hi = v.min(0), v.max(0)
    ext = max(float((hi - lo).max()), 1e-3)
    o = (lo + hi) / 2 + (rng.random((n, 3)) - 0.5) * 2.0 * ext
    cen = tris.reshape(-1, 3, 3).astype(np.float64).mean(1)
    aim = cen[rng.integers(0, cen.shape[0], n)] + rng.normal(scale=0.01 * ext, size=(n, 3))
    d = np.where((np.arange(n) % 2 == 0)[:, None], aim - o, rng.normal(size=(n, 3)))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    tmax = rng.random(n) * 2.0 * ext if shadow else np.full(n, np.inf)
    org = np.concatenate([o, np.full((n, 1), 1e-4)], 1).astype(np.float32)
    dir_ = np.concatenate([d, tmax[:, None]], 1).astype(np.float32)
    return org, dir_


def _trace(ctx, bvh_h, org, dir_, any_hit=False):
    o, d = torch.from_numpy(org).to(DEV), torch.from_numpy(dir_).to(DEV)
    hits = torch.zeros((org.shape[0], 4), dtype=torch.int32, device=DEV)
    hcc.hcc_trace(ctx, bvh_h, o, d, hits, any_hit=any_hit)
    hcc.hcc_sync(ctx)
    return hcc.hits_to_numpy(hits)


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("ntris", [1, 2, 3, 4, 5, 7, 9, 17, 33, 100, 1000])
def test_small_trees_match_brute_force(ctx, layout, ntris):
    tris = gen.random_tris(40 + ntris, ntris, mu=-1.5)
    bvh = gen.build_bvh(tris)
    h = hcc.hcc_bvh_upload(ctx, bvh, layout=layout)
    try:
        org, dir_ = _rays(ntris, 2000, tris)
        ref = oracle.trace_brute(tris, org, dir_)
        assert (ref["prim"] >= 0).any()
        compare_hits(_trace(ctx, h, org, dir_), ref)
    finally:
        hcc.hcc_bvh_destroy(h)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_any_hit_matches_the_definition(ctx, layout):
    tris = gen.random_tris(7, 800, mu=-2.0)
    bvh = gen.build_bvh(tris)
    h = hcc.hcc_bvh_upload(ctx, bvh, layout=layout)
    try:
        org, dir_ = _rays(3, 4000, tris, shadow=True)
        g = _trace(ctx, h, org, dir_, any_hit=True)
        ref = oracle.trace_brute(tris, org, dir_, any_hit=True)
        occl = g["prim"] >= 0
        assert np.array_equal(occl, ref["prim"] >= 0)
        assert 0.05 < occl.mean() < 0.95
        for i in np.nonzero(occl)[0]:
            ok, t, _, _ = oracle.intersect(org[i, :3], dir_[i, :3], org[i, 3], dir_[i, 3], tris[g["prim"][i]])
            assert ok and np.float32(t) == g["t"][i]
    finally:
        hcc.hcc_bvh_destroy(h)


def _inverted(bvh, seed):
    """The same tree with lo and hi exchanged on one random axis of half the
    nodes: a min/max slab test sees the same slabs."""
    rng = np.random.default_rng(seed)
    lo, hi = bvh.lo.copy(), bvh.hi.copy()
    for k in np.nonzero(rng.random(lo.shape[0]) < 0.5)[0]:
        a = rng.integers(0, 3)
        lo[k, a], hi[k, a] = hi[k, a], lo[k, a]
    return gen.BVH(lo, hi, bvh.left, bvh.right, bvh.first, bvh.count, bvh.order, bvh.tris, bvh.depth)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_boxes_given_inverted_trace_the_same(ctx, layout):
    tris = gen.random_tris(11, 500, mu=-2.0)
    bvh = gen.build_bvh(tris)
    inv = _inverted(bvh, 5)
    assert (inv.lo > inv.hi).any()
    org, dir_ = _rays(9, 3000, tris)
    ref = oracle.trace_brute(tris, org, dir_)
    # the oracle's traversal reads the inverted boxes as the same slabs
    assert oracle.trace_bvh(inv, org, dir_).tobytes() == oracle.trace_bvh(bvh, org, dir_).tobytes()
    h0 = hcc.hcc_bvh_upload(ctx, bvh, layout=layout)
    h1 = hcc.hcc_bvh_upload(ctx, inv, layout=layout)
    try:
        g0 = _trace(ctx, h0, org, dir_)
        g1 = _trace(ctx, h1, org, dir_)
        assert g0.tobytes() == g1.tobytes()
        compare_hits(g1, ref)
    finally:
        hcc.hcc_bvh_destroy(h0)
        hcc.hcc_bvh_destroy(h1)


def test_wide_nodes_visit_fewer_nodes(ctx):
    """The 4-ary tree holds every BVH2 box, so a ray tests the same boxes
    and triangles in fewer node visits (the diagnostic counters)."""
    w = gen.room_workload(1, target_tris=60_000, W=160, H=90, spp=2)
    org, dir_ = torch.from_numpy(w.rays.org).to(DEV), torch.from_numpy(w.rays.dir).to(DEV)
    counts = {}
    for layout in ("exact", "wide"):
        h = hcc.hcc_bvh_upload(ctx, w.bvh, layout=layout)
        try:
            counts[layout] = hcc.hcc_trace_counts(ctx, h, org, dir_)
        finally:
            hcc.hcc_bvh_destroy(h)
    assert counts["wide"]["node_visits"] < 0.75 * counts["exact"]["node_visits"]
    # the same leaves are reached (up to the order-dependent pruning)
    assert abs(counts["wide"]["tri_tests"] - counts["exact"]["tri_tests"]) < 0.1 * counts["exact"]["tri_tests"]
