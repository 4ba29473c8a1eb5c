"""Autotuner for the batched wavefront path: per-scene cut size, shared key length.

For each candidate key length and each scene it times, through the C ABI,
one HCC bounce (encode -> sort -> trace through the sorted ids) of that
scene's rays with every candidate cut size, keeps each scene's fastest cut,
and picks the key length whose summed best times are lowest.  Timing uses
CUDA events on the context's stream; the result is a plain dict.  (Block
shapes and the traversal stack depth are compile-time constants of the
kernels, so they are not searched.)
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


def tune_batch(ctx, stream, bvhs, rays, cut_sizes=(16, 32, 64, 128), key_bits=(24, 32, 48), lam=0.125,
               max_rays=1 << 20, reps=3):
    """rays: list of (org, dir) CUDA tensor pairs, one per scene (the scene's wavefront).

    Returns {"key_bits": k, "cut_sizes": [C per scene], "table": {...}} where table[k][s][C]
    is the measured ms of scene s's bounce (first max_rays rays) with cut C and k-bit keys.
    """
    import torch
    table = {}
    for k in key_bits:
        table[k] = []
        for s, (org, dir_) in enumerate(rays):
            n = min(int(org.shape[0]), max_rays)
            o, d = org[:n], dir_[:n]
            keys = torch.empty(n, dtype=torch.int32 if k <= 32 else torch.int64, device=org.device)
            perm = torch.empty(n, dtype=torch.int32, device=org.device)
            hits = torch.empty((n, 4), dtype=torch.int32, device=org.device)
            row = {}
            for C in cut_sizes:
                cut = hcc.hcc_select_cut(ctx, bvhs[s], C, lam)
                try:
                    def bounce():
                        hcc.hcc_encode(ctx, "hcc", bvhs[s], cut, o, d, k, keys)
                        hcc.hcc_sort(ctx, keys, k, n, perm)
                        hcc.hcc_trace_sorted(ctx, bvhs[s], o, d, perm, hits)
                    row[C] = _time(stream, bounce, reps)
                finally:
                    hcc.hcc_cut_destroy(cut)
            table[k].append(row)
    totals = {k: sum(min(r.values()) for r in rows) for k, rows in table.items()}
    best_k = min(totals, key=totals.get)
    best_c = [min(r, key=r.get) for r in table[best_k]]
    return {"key_bits": best_k, "cut_sizes": best_c, "totals_ms": totals, "table": table}
