"""Batches of wavefronts over several scenes, the next-bounce spawn and CUDA
graph capture, against the CPU oracle (needs a GB300).

The oracle traces each scene's rays on its own BVH; the batch must give the
same records bit for bit in every order (NoSort, HCC, TwoPoint, Origin-
Direction).  Bounce-2 rays are generated by the oracle from its own bounce-1
hits, never taken from the GPU.
"""
import numpy as np
import pytest

import oracle
from paper_2305_16652_gb300 import gen, hcc
from parity import compare_hits

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _scenes():
    ws = [gen.tiny_workload(0, ntris=3000, nrays=2048),
          gen.room_workload(3, target_tris=40_000, W=64, H=36, spp=2, shadow=False),
          gen.tiny_workload(5, ntris=6000, nrays=3000),
          gen.room_workload(4, target_tris=20_000, W=40, H=30, spp=1, shadow=False)]
    return ws


@pytest.fixture(scope="module")
def env():
    ctx = hcc.hcc_create(0)
    ws = _scenes()
    layouts = {}
    for layout in ("exact", "quantised", "wide"):
        bvhs = [hcc.hcc_bvh_upload(ctx, w.bvh, layout=layout) for w in ws]
        cuts = [hcc.hcc_select_cut(ctx, b, 32, 0.125) for b in bvhs]
        layouts[layout] = (bvhs, cuts)
    offsets = np.concatenate([[0], np.cumsum([w.rays.n for w in ws])]).astype(np.uint64)
    org = np.concatenate([w.rays.org for w in ws])
    dir_ = np.concatenate([w.rays.dir for w in ws])
    ref = [oracle.trace_bvh(w.bvh, w.rays.org, w.rays.dir) for w in ws]
    yield dict(ctx=ctx, ws=ws, layouts=layouts, offsets=offsets, org=org, dir=dir_, ref=np.concatenate(ref))
    for bvhs, cuts in layouts.values():
        for c in cuts:
            hcc.hcc_cut_destroy(c)
        for b in bvhs:
            hcc.hcc_bvh_destroy(b)
    hcc.hcc_destroy(ctx)


def _run(e, method, k, layout="exact", org=None, dir_=None):
    ctx = e["ctx"]
    bvhs, cuts = e["layouts"][layout]
    batch = hcc.hcc_batch_create(ctx, bvhs, cuts, e["offsets"])
    o = torch.from_numpy(e["org"] if org is None else org).to(DEV)
    d = torch.from_numpy(e["dir"] if dir_ is None else dir_).to(DEV)
    hits = torch.zeros((o.shape[0], 4), dtype=torch.int32, device=DEV)
    try:
        hcc.hcc_batch_run(ctx, batch, method, o, d, k, hits)
        hcc.hcc_sync(ctx)
    finally:
        hcc.hcc_batch_destroy(batch)
    return hcc.hits_to_numpy(hits)


@pytest.mark.parametrize("layout", ["exact", "quantised", "wide"])
@pytest.mark.parametrize("method,k", [("nosort", 32), ("hcc", 32), ("hcc", 62), ("twopoint", 30), ("origin_dir", 48),
                                      ("origin", 12)])
def test_batch_matches_per_scene_oracle(env, method, k, layout):
    g = _run(env, method, k, layout)
    compare_hits(g, env["ref"])
    assert (g["prim"] >= 0).mean() > 0.3


def test_batch_rejects_bad_arguments(env):
    ctx = env["ctx"]
    bvhs, cuts = env["layouts"]["exact"]
    with pytest.raises(hcc.HccError):  # decreasing offsets
        hcc.hcc_batch_create(ctx, bvhs, cuts, [0, 10, 5, 20, 30])
    with pytest.raises(hcc.HccError):  # mixed node layouts
        mixed = [bvhs[0], env["layouts"]["quantised"][0][1]] + bvhs[2:]
        hcc.hcc_batch_create(ctx, mixed, cuts, env["offsets"])
    batch = hcc.hcc_batch_create(ctx, bvhs, cuts, env["offsets"])
    try:
        o = torch.from_numpy(env["org"]).to(DEV)
        d = torch.from_numpy(env["dir"]).to(DEV)
        hits = torch.zeros((o.shape[0], 4), dtype=torch.int32, device=DEV)
        with pytest.raises(hcc.HccError):  # 63 key bits + 2 scene bits do not fit
            hcc.hcc_batch_run(ctx, batch, "hcc", o, d, 63, hits)
        with pytest.raises(hcc.HccError):  # ray count differs from the batch's
            hcc.hcc_batch_run(ctx, batch, "hcc", o[1:], d[1:], 32, hits)
    finally:
        hcc.hcc_batch_destroy(batch)
    hcc.hcc_sync(ctx)


@pytest.mark.parametrize("records", [False, True])
def test_spawn_matches_oracle_and_second_bounce(env, records):
    """Both bounces of the batch, on packed arrays or on 32-byte ray records
    (origin and direction adjacent) for the input and the spawned rays."""
    ctx = env["ctx"]
    bvhs, cuts = env["layouts"]["exact"]
    batch = hcc.hcc_batch_create(ctx, bvhs, cuts, env["offsets"])
    n = env["org"].shape[0]
    o = torch.from_numpy(env["org"]).to(DEV)
    d = torch.from_numpy(env["dir"]).to(DEV)
    hits = torch.zeros((n, 4), dtype=torch.int32, device=DEV)
    if records:
        rec1 = torch.cat([o, d], 1)
        rec2 = torch.zeros_like(rec1)
        o, d = rec1[:, :4], rec1[:, 4:]
        o2, d2 = rec2[:, :4], rec2[:, 4:]
    else:
        o2, d2 = torch.zeros_like(o), torch.zeros_like(d)
    hits2 = torch.zeros_like(hits)
    try:
        hcc.hcc_batch_run(ctx, batch, "hcc", o, d, 32, hits)
        hcc.hcc_batch_spawn(ctx, batch, o, d, hits, 1234, 1e-4, o2, d2)
        hcc.hcc_batch_run(ctx, batch, "hcc", o2, d2, 32, hits2)
        hcc.hcc_sync(ctx)
    finally:
        hcc.hcc_batch_destroy(batch)
    # oracle: its own bounce-1 hits, its own spawn, its own bounce-2 trace
    off = env["offsets"].astype(np.int64)
    ref_o, ref_d, ref_h2 = [], [], []
    for s, w in enumerate(env["ws"]):
        sl = slice(off[s], off[s + 1])
        h1 = env["ref"][sl]
        ro, rd = oracle.spawn(env["org"][sl], env["dir"][sl], h1, w.tris, 1234, 1e-4, first_index=int(off[s]))
        ref_o.append(ro)
        ref_d.append(rd)
        ref_h2.append(oracle.trace_bvh(w.bvh, ro, rd))
    assert o2.contiguous().cpu().numpy().tobytes() == np.concatenate(ref_o).tobytes()
    assert d2.contiguous().cpu().numpy().tobytes() == np.concatenate(ref_d).tobytes()
    g2 = hcc.hits_to_numpy(hits2)
    compare_hits(g2, np.concatenate(ref_h2))
    assert (g2["prim"] >= 0).mean() > 0.05


def test_graph_capture_replays_a_bounce(env):
    ctx_stream = torch.cuda.Stream()
    ctx = hcc.hcc_create(0, ctx_stream)
    bvhs, cuts = env["layouts"]["exact"]
    batch = hcc.hcc_batch_create(ctx, bvhs, cuts, env["offsets"])
    n = env["org"].shape[0]
    o = torch.from_numpy(env["org"]).to(DEV)
    d = torch.from_numpy(env["dir"]).to(DEV)
    hits = torch.zeros((n, 4), dtype=torch.int32, device=DEV)
    torch.cuda.synchronize()
    try:
        graph = hcc.hcc_graph_capture_batch(ctx, batch, "hcc", o, d, 32, hits)
        for _ in range(2):
            hits.zero_()
            torch.cuda.synchronize()
            hcc.hcc_graph_launch(ctx, graph)
            hcc.hcc_sync(ctx)
            compare_hits(hcc.hits_to_numpy(hits), env["ref"])
        hcc.hcc_graph_destroy(graph)
    finally:
        hcc.hcc_batch_destroy(batch)
        hcc.hcc_destroy(ctx)


@pytest.mark.parametrize("layout", ["exact", "quantised", "wide"])
def test_every_trace_shape_returns_the_oracle_hits(env, layout):
    """Each block size and stack depth the autotuner may pick (deep enough for
    the BVHs) gives the oracle's hits, on single wavefronts through the sorted
    ids and on the whole batch; a stack too shallow is reported, never silent."""
    from paper_2305_16652_gb300 import tune
    ctx = env["ctx"]
    bvhs, cuts = env["layouts"][layout]
    cands = tune.shape_candidates(bvhs, layout)
    assert cands and all(st >= tune.stack_bound(b, layout) for b in bvhs for _, st in cands)
    off = env["offsets"].astype(np.int64)
    o = torch.from_numpy(env["org"]).to(DEV)
    d = torch.from_numpy(env["dir"]).to(DEV)
    batch = hcc.hcc_batch_create(ctx, bvhs, cuts, env["offsets"])
    try:
        for shape in cands:
            hcc.hcc_set_trace_shape(ctx, *shape)
            hits = torch.zeros((o.shape[0], 4), dtype=torch.int32, device=DEV)
            hcc.hcc_batch_run(ctx, batch, "hcc", o, d, 32, hits)
            hcc.hcc_sync(ctx)
            compare_hits(hcc.hits_to_numpy(hits), env["ref"])
            s = 0
            n = int(off[1] - off[0])
            h1 = torch.zeros((n, 4), dtype=torch.int32, device=DEV)
            hcc.hcc_run(ctx, "hcc", bvhs[s], cuts[s], o[:n], d[:n], 32, h1)
            hcc.hcc_sync(ctx)
            compare_hits(hcc.hits_to_numpy(h1), env["ref"][:n])
    finally:
        hcc.hcc_set_trace_shape(ctx, 0, 0)
        hcc.hcc_batch_destroy(batch)
    with pytest.raises(hcc.HccError):
        hcc.hcc_set_trace_shape(ctx, 96, 64)
    with pytest.raises(hcc.HccError):
        hcc.hcc_set_trace_shape(ctx, 128, 40)


def test_autotuner_choices_are_valid_and_keep_the_results(env):
    from paper_2305_16652_gb300 import tune
    stream = torch.cuda.Stream()
    ctx = hcc.hcc_create(0, stream)
    bvhs, _ = env["layouts"]["exact"]
    off = env["offsets"].astype(np.int64)
    o = torch.from_numpy(env["org"]).to(DEV)
    d = torch.from_numpy(env["dir"]).to(DEV)
    per_scene = [(o[off[s]:off[s + 1]], d[off[s]:off[s + 1]]) for s in range(len(bvhs))]
    torch.cuda.synchronize()
    try:
        t = tune.tune_batch(ctx, stream, bvhs, per_scene, cut_sizes=(8, 32), key_bits=(16, 32),
                            lambdas=(0.0625, 0.125), schedules=("refill", "per_ray"), reps=1)
        assert t["key_bits"] in (16, 32) and t["schedule"] in ("refill", "per_ray")
        assert len(t["cut_sizes"]) == len(bvhs) and set(t["cut_sizes"]) <= {8, 32}
        assert set(t["lambdas"]) <= {0.0625, 0.125}
        assert tuple(t["shape"]) in tune.shape_candidates(bvhs, "exact")
        cuts = [hcc.hcc_select_cut(ctx, b, C, lam) for b, C, lam in zip(bvhs, t["cut_sizes"], t["lambdas"])]
        batch = hcc.hcc_batch_create(ctx, bvhs, cuts, env["offsets"])
        hits = torch.zeros((o.shape[0], 4), dtype=torch.int32, device=DEV)
        hcc.hcc_batch_run(ctx, batch, "hcc", o, d, t["key_bits"], hits)
        hcc.hcc_sync(ctx)
        compare_hits(hcc.hits_to_numpy(hits), env["ref"])
        hcc.hcc_batch_destroy(batch)
        for c in cuts:
            hcc.hcc_cut_destroy(c)
    finally:
        hcc.hcc_destroy(ctx)
