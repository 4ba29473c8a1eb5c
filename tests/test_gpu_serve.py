"""The serving loop: requests of uneven sizes against several resident scenes,
run alone and in a mix of concurrent requests (needs a GB300).

Every request's hits must be the same bit for bit whether it ran alone
(one slot, one request on the GPU at a time) or among others sharing the GPU,
and equal to the CPU oracle's trace of the same rays on the same scene.
"""
import threading

import numpy as np
import pytest

import oracle
from paper_2305_16652_gb300 import gen, hcc
from parity import compare_hits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [1, 3, 31, 32, 33, 257, 1000, 4097, 6000]


@pytest.fixture(scope="module")
def scenes():
    ws = [gen.tiny_workload(0, ntris=3000, nrays=6000),
          gen.room_workload(3, target_tris=40_000, W=80, H=45, spp=2, shadow=False),
          gen.tiny_workload(7, ntris=8000, nrays=6000)]
    ctx = hcc.hcc_create(0)
    up = {}
    for layout in ("exact", "quantised", "wide"):
        bvhs = [hcc.hcc_bvh_upload(ctx, w.bvh, layout=layout) for w in ws]
        cuts = [hcc.hcc_select_cut(ctx, b, 32, 0.125) for b in bvhs]
        up[layout] = (bvhs, cuts)
    torch.cuda.synchronize()
    yield ws, up
    for bvhs, cuts in up.values():
        for c in cuts:
            hcc.hcc_cut_destroy(c)
        for b in bvhs:
            hcc.hcc_bvh_destroy(b)
    hcc.hcc_destroy(ctx)


def _requests(ws, seed, count, any_hit_every=0):
    """(scene, org, dir, any_hit) with uneven sizes and shuffled ray subsets."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        s = i % len(ws)
        rays = ws[s].rays
        n = min(SIZES[int(rng.integers(len(SIZES)))], rays.n)
        idx = rng.permutation(rays.n)[:n]
        any_hit = bool(any_hit_every) and i % any_hit_every == any_hit_every - 1
        out.append((s, np.ascontiguousarray(rays.org[idx]), np.ascontiguousarray(rays.dir[idx]), any_hit))
    return out


def _host(a, pinned):
    if not pinned:
        return a
    t = torch.from_numpy(a).pin_memory()
    return t


def _run_alone(server, reqs):
    res = []
    for k, (s, o, d, ah) in enumerate(reqs):
        oo, dd = _host(o, k % 2 == 0), _host(d, k % 2 == 0)
        hits = np.zeros(o.shape[0], oracle.HIT_DTYPE)
        t = hcc.hcc_server_submit(server, s, oo, dd, hits, any_hit=ah)
        hcc.hcc_server_wait(server, t)
        res.append(hits)
    return res


def _run_mix(server, reqs, threads=4):
    """Submit from several threads at once, then wait for every ticket."""
    res = [None] * len(reqs)
    keep = []
    tickets = [None] * len(reqs)
    bufs = []
    for k, (s, o, d, ah) in enumerate(reqs):
        pinned = k % 3 != 0
        hits = torch.zeros((o.shape[0], 4), dtype=torch.int32).pin_memory() if pinned else \
            np.zeros(o.shape[0], oracle.HIT_DTYPE)
        bufs.append((_host(o, pinned), _host(d, pinned), hits))
    go = threading.Barrier(threads)
    errors = []

    def worker(w):
        try:
            go.wait()
            for k in range(w, len(reqs), threads):
                oo, dd, hh = bufs[k]
                tickets[k] = hcc.hcc_server_submit(server, reqs[k][0], oo, dd, hh, any_hit=reqs[k][3])
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(e)

    th = [threading.Thread(target=worker, args=(w,)) for w in range(threads)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    lat = [hcc.hcc_server_wait(server, t) for t in tickets]
    for k, (_, _, hh) in enumerate(bufs):
        res[k] = hcc.hits_to_numpy(hh) if hasattr(hh, "numpy") else hh
    keep.append(bufs)
    return res, lat


def _oracle(ws, reqs):
    return [oracle.trace_bvh(ws[s].bvh, o, d, any_hit=ah) for s, o, d, ah in reqs]


@pytest.mark.parametrize("method,k,layout", [("hcc", 32, "exact"), ("hcc", 48, "quantised"),
                                             ("twopoint", 30, "exact"), ("nosort", 32, "quantised"),
                                             ("origin_dir", 24, "exact"), ("hcc", 32, "wide")])
def test_each_result_is_the_same_alone_and_in_the_mix(scenes, method, k, layout):
    ws, up = scenes
    bvhs, cuts = up[layout]
    reqs = _requests(ws, seed=11, count=36)
    ref = _oracle(ws, reqs)
    alone_srv = hcc.hcc_server_create(0, bvhs, cuts, slots=1, method=method, key_bits=k)
    try:
        alone = _run_alone(alone_srv, reqs)
        st = hcc.hcc_server_stats_get(alone_srv)
        assert st["max_in_flight"] == 1 and st["completed"] == len(reqs) and st["failed"] == 0
    finally:
        hcc.hcc_server_destroy(alone_srv)
    mix_srv = hcc.hcc_server_create(0, bvhs, cuts, slots=8, method=method, key_bits=k)
    try:
        mix, lat = _run_mix(mix_srv, reqs)
        st = hcc.hcc_server_stats_get(mix_srv)
        assert st["completed"] == len(reqs) and st["failed"] == 0 and st["queued"] == 0
        assert st["rays"] == sum(r[1].shape[0] for r in reqs)
        assert 1 <= st["max_in_flight"] <= 8
    finally:
        hcc.hcc_server_destroy(mix_srv)
    assert all(x > 0 for x in lat)
    for a, m, r in zip(alone, mix, ref):
        assert a.tobytes() == m.tobytes()
        compare_hits(a, r)


def test_any_hit_requests_in_the_mix(scenes):
    ws, up = scenes
    bvhs, cuts = up["exact"]
    reqs = _requests(ws, seed=12, count=24, any_hit_every=2)
    srv1 = hcc.hcc_server_create(0, bvhs, cuts, slots=1, method="hcc", key_bits=32)
    try:
        alone = _run_alone(srv1, reqs)
    finally:
        hcc.hcc_server_destroy(srv1)
    srv = hcc.hcc_server_create(0, bvhs, cuts, slots=6, method="hcc", key_bits=32)
    try:
        mix, _ = _run_mix(srv, reqs, threads=3)
    finally:
        hcc.hcc_server_destroy(srv)
    for (s, o, d, ah), a, m in zip(reqs, alone, mix):
        assert a.tobytes() == m.tobytes()
        ref = oracle.trace_bvh(ws[s].bvh, o, d, any_hit=ah)
        if ah:  # any hit is valid: compare occlusion only
            assert np.array_equal(a["prim"] >= 0, ref["prim"] >= 0)
        else:
            compare_hits(a, ref)


def test_failed_request_does_not_affect_others(scenes):
    """A request whose traversal overflows the stack fails alone; requests
    running beside it finish with correct hits."""
    from test_gpu_parity import _chain_bvh
    ws, up = scenes
    ctx = hcc.hcc_create(0)
    deep = _chain_bvh(100)
    hdeep = hcc.hcc_bvh_upload(ctx, deep, layout="exact")
    cdeep = hcc.hcc_select_cut(ctx, hdeep, 32, 0.125)
    bvhs, cuts = up["exact"]
    srv = hcc.hcc_server_create(0, list(bvhs) + [hdeep], list(cuts) + [cdeep], slots=4, method="hcc", key_bits=32)
    try:
        reqs = _requests(ws, seed=13, count=9)
        c = deep.tris.reshape(-1, 3).mean(0)
        bad_o = np.array([[c[0], c[1], c[2] - 5.0, 0.0]] * 64, np.float32)
        bad_d = np.array([[0.0, 0.0, 1.0, np.inf]] * 64, np.float32)
        bad_h = np.zeros(64, oracle.HIT_DTYPE)
        tickets, outs = [], []
        for k, (s, o, d, ah) in enumerate(reqs):
            if k == 4:
                bad = hcc.hcc_server_submit(srv, len(bvhs), bad_o, bad_d, bad_h)
            h = np.zeros(o.shape[0], oracle.HIT_DTYPE)
            tickets.append(hcc.hcc_server_submit(srv, s, o, d, h))
            outs.append(h)
        with pytest.raises(hcc.HccError) as ei:
            hcc.hcc_server_wait(srv, bad)
        assert ei.value.status == 5  # HCC_ERR_STACK_OVERFLOW
        for t in tickets:
            hcc.hcc_server_wait(srv, t)
        for (s, o, d, _), h in zip(reqs, outs):
            compare_hits(h, oracle.trace_bvh(ws[s].bvh, o, d))
        st = hcc.hcc_server_stats_get(srv)
        assert st["failed"] == 1 and st["completed"] == len(reqs)
    finally:
        hcc.hcc_server_destroy(srv)
        hcc.hcc_cut_destroy(cdeep)
        hcc.hcc_bvh_destroy(hdeep)
        hcc.hcc_destroy(ctx)


def test_admission_respects_the_memory_budget(scenes):
    ws, up = scenes
    bvhs, cuts = up["exact"]
    n = 6000
    reqs = [(s, ws[s].rays.org[:n], ws[s].rays.dir[:n], False) for s in (0, 2, 0, 2, 0)]
    probe = hcc.hcc_server_create(0, bvhs, cuts, slots=1, method="hcc", key_bits=32)
    one = hcc.hcc_server_request_bytes(probe, n)
    hcc.hcc_server_destroy(probe)
    assert one >= n * (32 + 16 + 4 + 4)
    # budget for 1.5 requests: slots are free but only one request fits at a time
    srv = hcc.hcc_server_create(0, bvhs, cuts, slots=8, method="hcc", key_bits=32, hbm_budget=one * 3 // 2)
    try:
        mix, _ = _run_mix(srv, reqs, threads=1)
        st = hcc.hcc_server_stats_get(srv)
        assert st["max_in_flight"] == 1
        assert st["peak_bytes"] == one
        for (s, o, d, _), m in zip(reqs, mix):
            compare_hits(m, oracle.trace_bvh(ws[s].bvh, o, d))
        # a request that could never fit is refused at submission
        big = 2 * n
        o, d = np.tile(ws[0].rays.org[:n], (2, 1)), np.tile(ws[0].rays.dir[:n], (2, 1))
        h = np.zeros(big, oracle.HIT_DTYPE)
        with pytest.raises(hcc.HccError) as ei:
            hcc.hcc_server_submit(srv, 0, o, d, h)
        assert ei.value.status == 2  # HCC_ERR_OOM
    finally:
        hcc.hcc_server_destroy(srv)


def test_server_rejects_bad_arguments(scenes):
    ws, up = scenes
    bvhs, cuts = up["exact"]
    qb, _ = up["quantised"]
    for kw in (dict(slots=0), dict(slots=65), dict(key_bits=0), dict(key_bits=65)):
        args = dict(slots=2, method="hcc", key_bits=32)
        args.update(kw)
        with pytest.raises(hcc.HccError):
            hcc.hcc_server_create(0, bvhs, cuts, **args)
    with pytest.raises(hcc.HccError):  # HCC needs cuts
        hcc.hcc_server_create(0, bvhs, None, slots=2, method="hcc", key_bits=32)
    with pytest.raises(hcc.HccError):  # mixed node layouts
        hcc.hcc_server_create(0, [bvhs[0], qb[1]], cuts[:2], slots=2, method="hcc", key_bits=32)
    srv = hcc.hcc_server_create(0, bvhs, None, slots=2, method="twopoint", key_bits=32)
    try:
        o, d = ws[0].rays.org[:10], ws[0].rays.dir[:10]
        h = np.zeros(10, oracle.HIT_DTYPE)
        with pytest.raises(hcc.HccError):  # scene index out of range
            hcc.hcc_server_submit(srv, 3, o, d, h)
        with pytest.raises(hcc.HccError):  # empty request
            hcc.hcc_server_submit(srv, 0, o[:0], d[:0], h[:0])
        with pytest.raises(hcc.HccError):  # unknown ticket
            hcc.hcc_server_wait(srv, 12345)
        t = hcc.hcc_server_submit(srv, 0, o, d, h)
        hcc.hcc_server_wait(srv, t)
        compare_hits(h, oracle.trace_bvh(ws[0].bvh, o, d))
        with pytest.raises(hcc.HccError):  # a ticket is released by its wait
            hcc.hcc_server_query(srv, t)
    finally:
        hcc.hcc_server_destroy(srv)
