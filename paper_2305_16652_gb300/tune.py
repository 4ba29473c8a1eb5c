"""Autotuner for the batched wavefront path: per-scene cut size and HAD
weight, shared key length, trace schedule, and the trace's block shape and
traversal-stack depth.

For each trace schedule, candidate key length and scene it times, through
the C ABI, one HCC bounce (encode -> sort -> trace through the sorted ids) of
that scene's rays with every candidate (cut size, lambda), keeps each scene's
fastest pair, and picks the (schedule, key length) whose summed best times
are lowest.  It then times the trace of every scene (with its chosen cut and
the chosen key length) in each candidate shape -- threads per block and
stack entries per ray of the closest-hit persistent trace -- whose stack is
deep enough for every scene's BVH, and keeps the fastest total.  Timing uses
CUDA events on the context's stream; the result is a plain dict.
"""
from __future__ import annotations

import statistics

from . import hcc


def _time(stream, fn, reps):
    import torch
    times = []
    for _ in range(reps + 1):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times[1:])


def stack_bound(bvh, layout: str) -> int:
    """Stack entries a closest-hit traversal of this BVH can need: one per
    level for binary nodes (the farther child of each level descended); the
    4-ary layout can push three per level, so only the default depth is
    offered for it."""
    depth = int(hcc.hcc_bvh_info(bvh)["depth"])
    return depth + 1 if layout != "wide" else hcc.HCC_TRACE_STACK


def shape_candidates(bvhs, layout: str, shapes=None):
    """The supported (threads per block, stack entries) pairs deep enough for every BVH."""
    need = max(stack_bound(b, layout) for b in bvhs)
    return [(b, st) for b, st in (shapes or hcc.TRACE_SHAPES) if st >= need]


def tune_trace_shape(ctx, stream, bvhs, rays, cuts, key_bits, layout="exact", shapes=None, max_rays=1 << 20,
                     reps=3):
    """Time the trace through the sorted ids of every scene (its HCC keys from
    cuts[s] and key_bits) in each candidate shape; set the fastest on the
    context and return (shape, {shape: total ms})."""
    import torch
    cands = shape_candidates(bvhs, layout, shapes)
    prepared = []
    for s, (org, dir_) in enumerate(rays):
        n = min(int(org.shape[0]), max_rays)
        o, d = org[:n], dir_[:n]
        keys = torch.empty(n, dtype=torch.int32 if key_bits <= 32 else torch.int64, device=org.device)
        perm = torch.empty(n, dtype=torch.int32, device=org.device)
        hits = torch.empty((n, 4), dtype=torch.int32, device=org.device)
        hcc.hcc_encode(ctx, "hcc", bvhs[s], cuts[s], o, d, key_bits, keys)
        hcc.hcc_sort(ctx, keys, key_bits, n, perm)
        prepared.append((bvhs[s], o, d, perm, hits))
    totals = {}
    try:
        for shape in cands:
            hcc.hcc_set_trace_shape(ctx, *shape)
            totals[shape] = sum(_time(stream, lambda: hcc.hcc_trace_sorted(ctx, b, o, d, perm, hits), reps)
                                for b, o, d, perm, hits in prepared)
        hcc.hcc_sync(ctx)
    finally:
        hcc.hcc_set_trace_shape(ctx, 0, 0)
    best = min(totals, key=totals.get)
    hcc.hcc_set_trace_shape(ctx, *best)
    return best, totals


def tune_batch(ctx, stream, bvhs, rays, cut_sizes=(16, 32, 64, 128), key_bits=(24, 32, 48),
               lambdas=(0.0625, 0.125, 0.25), schedules=("auto",), max_rays=1 << 20, reps=3, layout="exact",
               shapes=None):
    """rays: list of (org, dir) CUDA tensor pairs, one per scene (the scene's wavefront).

    Searches each scene's cut size C and HAD weight lambda (Eq. 1), the key length shared by the
    batch, the trace shape (threads per block, stack entries; every supported shape deep enough for
    the BVHs unless `shapes` narrows it) and (when more than one is given) the trace schedule of
    the context.  The schedule is not searched by default: timed scene by scene on capped
    wavefronts it favoured one thread per ray, while the batched trace of all scenes at once runs
    faster with ray replacement.  Returns {"key_bits": k, "cut_sizes": [C per scene], "lambdas":
    [lambda per scene], "schedule": s, "shape": (threads, stack), "totals_ms": {...}, "shape_ms":
    {...}, "table": {...}} where table[schedule][k][scene][(C, lambda)] is the measured ms of that
    scene's bounce (first max_rays rays).  The context is left with the chosen schedule and shape.
    """
    import torch
    cuts = [{(C, lam): hcc.hcc_select_cut(ctx, bvhs[s], C, lam) for C in cut_sizes for lam in lambdas}
            for s in range(len(rays))]
    table = {}
    try:
        for sched in schedules:
            hcc.hcc_set_trace_schedule(ctx, sched)
            table[sched] = {}
            for k in key_bits:
                table[sched][k] = []
                for s, (org, dir_) in enumerate(rays):
                    n = min(int(org.shape[0]), max_rays)
                    o, d = org[:n], dir_[:n]
                    keys = torch.empty(n, dtype=torch.int32 if k <= 32 else torch.int64, device=org.device)
                    perm = torch.empty(n, dtype=torch.int32, device=org.device)
                    hits = torch.empty((n, 4), dtype=torch.int32, device=org.device)
                    row = {}
                    for key, cut in cuts[s].items():
                        def bounce():
                            hcc.hcc_encode(ctx, "hcc", bvhs[s], cut, o, d, k, keys)
                            hcc.hcc_sort(ctx, keys, k, n, perm)
                            hcc.hcc_trace_sorted(ctx, bvhs[s], o, d, perm, hits)
                        row[key] = _time(stream, bounce, reps)
                    table[sched][k].append(row)
    finally:
        for per_scene in cuts:
            for cut in per_scene.values():
                hcc.hcc_cut_destroy(cut)
    totals = {(sc, k): sum(min(r.values()) for r in rows) for sc, by_k in table.items() for k, rows in by_k.items()}
    best_sched, best_k = min(totals, key=totals.get)
    best = [min(r, key=r.get) for r in table[best_sched][best_k]]
    hcc.hcc_set_trace_schedule(ctx, best_sched)
    chosen = [hcc.hcc_select_cut(ctx, bvhs[s], C, lam) for s, (C, lam) in enumerate(best)]
    try:
        shape, shape_ms = tune_trace_shape(ctx, stream, bvhs, rays, chosen, best_k, layout, shapes, max_rays, reps)
    finally:
        for c in chosen:
            hcc.hcc_cut_destroy(c)
    return {"key_bits": best_k, "cut_sizes": [c for c, _ in best], "lambdas": [lam for _, lam in best],
            "schedule": best_sched, "shape": shape,
            "totals_ms": {f"{sc}/{k}": round(v, 3) for (sc, k), v in totals.items()},
            "shape_ms": {f"{b}x{st}": round(v, 3) for (b, st), v in shape_ms.items()}, "table": table}
