"""Input generators: determinism and BVH well-formedness (no GPU)."""
import numpy as np

from paper_2305_16652_gb300 import gen


def test_rng_is_counter_based_and_deterministic():
    a = [gen.rng_u64(1, 2, i) for i in range(100)]
    b = [gen.rng_u64(1, 2, i) for i in range(100)]
    assert a == b and len(set(a)) == 100
    assert gen.rng_u64(1, 2, 5) != gen.rng_u64(2, 2, 5) != gen.rng_u64(1, 3, 5)


def test_random_scene_centroids_and_sizes():
    t = gen.random_tris(0, 10_000).reshape(-1, 3, 3).astype(np.float64)
    c = t.mean(axis=1)
    assert np.all(c > -1e-6) and np.all(c < 1 + 1e-6)
    edge = np.linalg.norm(t[:, 1] - t[:, 0], axis=1)
    assert 0.005 < np.median(edge) < 0.05
    assert np.array_equal(gen.random_tris(0, 100), gen.random_tris(0, 100))


def _check_bvh(b):
    n = b.num_nodes
    assert n == 2 * int(np.sum(b.left < 0)) - 1
    leaves = np.nonzero(b.left < 0)[0]
    assert np.all(b.count[leaves] >= 1) and np.all(b.count[leaves] <= 4)
    # every triangle is in exactly one leaf
    seen = np.zeros(b.num_tris, np.int64)
    for l in leaves:
        seen[b.order[b.first[l]:b.first[l] + b.count[l]]] += 1
    assert np.all(seen == 1)
    # boxes are tight unions: leaf boxes bound their triangles, parents bound children
    tris = b.tris.reshape(-1, 3, 3)
    for l in leaves[:2000]:
        ids = b.order[b.first[l]:b.first[l] + b.count[l]]
        v = tris[ids].reshape(-1, 3)
        assert np.array_equal(b.lo[l], v.min(0)) and np.array_equal(b.hi[l], v.max(0))
    inner = np.nonzero(b.left >= 0)[0]
    lo_c = np.minimum(b.lo[b.left[inner]], b.lo[b.right[inner]])
    hi_c = np.maximum(b.hi[b.left[inner]], b.hi[b.right[inner]])
    assert np.array_equal(b.lo[inner], lo_c) and np.array_equal(b.hi[inner], hi_c)
    # pre-order numbering: the left child follows its parent
    assert np.all(b.left[inner] == inner + 1) and np.all(b.right[inner] > inner + 1)


def test_bvh_random_scene():
    _check_bvh(gen.build_bvh(gen.random_tris(3, 5000)))


def test_bvh_room_scene():
    tris = gen.room_tris(1, target_tris=50_000, clusters=10)
    assert tris.shape[0] >= 50_000
    _check_bvh(gen.build_bvh(tris))


def test_bvh_degenerate_inputs():
    one = gen.random_tris(0, 1)
    b = gen.build_bvh(one)
    assert b.num_nodes == 1 and b.left[0] == -1 and b.count[0] == 1
    same = np.tile(gen.random_tris(0, 1), (37, 1))  # identical centroids: falls back to halving
    _check_bvh(gen.build_bvh(same))


def test_tiny_workload_shape():
    w = gen.tiny_workload(0)
    assert w.rays.n == 4096 and w.tris.shape == (10_000, 9)
    assert np.all(w.rays.org[:, 3] == np.float32(1e-4)) and np.all(np.isinf(w.rays.dir[:, 3]))
    nrm = np.linalg.norm(w.rays.dir[:, :3].astype(np.float64), axis=1)
    assert np.all(np.abs(nrm - 1) < 1e-6)
    w2 = gen.tiny_workload(0)
    assert w.rays.org.tobytes() == w2.rays.org.tobytes() and w.rays.dir.tobytes() == w2.rays.dir.tobytes()


def test_room_workload_small_image():
    w = gen.room_workload(1, target_tris=30_000, W=96, H=54, spp=2)
    assert w.rays.n == 96 * 54 * 2  # closed room: every sample sees a surface
    assert w.shadow.n == 2 * w.rays.n
    assert np.all(w.shadow.dir[:, 3] > 0) and np.all(np.isfinite(w.shadow.dir[:, 3]))
    o = w.rays.org[:, :3]
    assert np.all(o > -1e-3) and np.all(o[:, 0] < 10.001) and np.all(o[:, 1] < 3.001) and np.all(o[:, 2] < 8.001)


def test_serve_request_stream():
    pools = [4_147_200, 3_000_000, 500_000]
    r = gen.serve_requests(1, 4000, pools)
    assert np.all((r["n"] >= 65_536) & (r["n"] <= 4_194_304))
    caps = np.array(pools)[r["scene"]]
    assert np.all(r["n"] <= caps) and np.all(r["offset"] >= 0) and np.all(r["offset"] + r["n"] <= caps)
    assert set(np.unique(r["scene"])) == {0, 1, 2}
    # log-uniform sizes: log n uniform on [log 64k, log 4M] where the pool does not cap it
    ln = np.log(r["n"][r["scene"] == 0])
    assert abs(ln.mean() - (np.log(65_536) + np.log(4_194_304)) / 2) < 0.1
    # Poisson arrivals at rate 1: exponential gaps with mean 1 and variance 1
    assert abs(r["gap"].mean() - 1) < 0.06 and abs(r["gap"].var() - 1) < 0.15 and np.all(r["gap"] >= 0)
    r2 = gen.serve_requests(1, 4000, pools)
    assert all(np.array_equal(r[k], r2[k]) for k in r)
