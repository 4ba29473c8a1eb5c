"""Autotuner for the batched wavefront path: per-scene cut size and HAD
weight, shared key length, trace schedule.

For each trace schedule, candidate key length and scene it times, through
the C ABI, one HCC bounce (encode -> sort -> trace through the sorted ids) of
that scene's rays with every candidate (cut size, lambda), keeps each scene's
fastest pair, and picks the (schedule, key length) whose summed best times
are lowest.  Timing uses CUDA events on the context's stream; the result is a
plain dict.  (Block shapes and the traversal stack depth are compile-time
constants of the kernels, so they are not searched: a 64-thread trace block
and tighter register bounds measured slower, and the stack needs 64 entries
for the deepest BVHs.)
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


def tune_batch(ctx, stream, bvhs, rays, cut_sizes=(16, 32, 64, 128), key_bits=(24, 32, 48),
               lambdas=(0.0625, 0.125, 0.25), schedules=("auto",), max_rays=1 << 20, reps=3):
    """rays: list of (org, dir) CUDA tensor pairs, one per scene (the scene's wavefront).

    Searches each scene's cut size C and HAD weight lambda (Eq. 1), the key length shared by the
    batch, and (when more than one is given) the trace schedule of the context.  The schedule is
    not searched by default: timed scene by scene on capped wavefronts it favoured one thread per
    ray, while the batched trace of all scenes at once runs faster with ray replacement.  Returns {"key_bits": k, "cut_sizes": [C per
    scene], "lambdas": [lambda per scene], "schedule": s, "totals_ms": {...}, "table": {...}}
    where table[schedule][k][scene][(C, lambda)] is the measured ms of that scene's bounce (first
    max_rays rays).  The context is left with the chosen schedule.
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
    return {"key_bits": best_k, "cut_sizes": [c for c, _ in best], "lambdas": [lam for _, lam in best],
            "schedule": best_sched, "totals_ms": {f"{sc}/{k}": round(v, 3) for (sc, k), v in totals.items()},
            "table": table}
