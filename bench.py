"""Benchmark: secondary-ray throughput of the hierarchy-cut-code pipeline.

One step = one pass of the whole hot path over one wavefront of secondary
rays of the 1920x1080, 8 spp furnished-room workload (16,588,800 rays,
~1M triangles): HCC encode (cut of 32 nodes, 32-bit keys) -> radix sort ->
gather -> closest-hit trace with the hits scattered back to input order.
The same wavefront is also run through the TwoPoint and NoSort orders.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (single-threaded) on a bounded sample
of the same workload and prints the same JSON line with "impl": "reference".
Under torchrun (N > 1) every rank traces its own wavefront (weak scaling);
rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "secondary Mrays/s incl. encode+sort, HCC vs NoSort/TwoPoint; p50/p99 latency"
UNIT = "Mrays/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "trace_room_1080p_dram.txt")
FALLBACK_HBM_GBS = 6800.0
SMS, LANES_PER_SM = 152, 128

# FP32/INT lane operations the trace kernel issues per unit of work, counted
# from trace.cu: one internal-node visit runs two slab tests (6 sub, 6 mul,
# 12 min/max, 1 mul, 1 min each = 26) and orders/pushes (~10); the quantised
# layout adds the decode of 12 bounds (byte select, convert, outward fma: 3
# ops each) and of the node frame (6); one triangle test is the
# Moller-Trumbore sequence (~45 ops incl. the reciprocal).  A 4-ary node
# visit (wide layout) runs four directed slab tests (6 fma, 5 min/max/mul,
# 4 to mark and clamp the met child = 15 each), selects its near/far rows
# (9), sorts the four entries (5 exchanges of 5 ops) and pushes (~12).
OPS_PER_NODE = {"exact": 2 * 26 + 10, "quantised": 36 + 6 + 2 * 26 + 10, "wide": 4 * 15 + 9 + 25 + 12}
OPS_PER_TRI = 45
# HBM bytes each stage must move per ray (32-bit keys; see the design notes)
BYTES_ENCODE = 32 + 4
BYTES_GATHER = 4 + 32 + 32
# FP32/INT lane operations of the HCC encode: about 20 per cut node that
# drives a bit (6 bound differences and products, 6 min/max to order and
# combine the slab ends, the tmin/tmax clamp, the compare and the bit) and
# about 10 per ray (reciprocal directions, key store): 650 at 32 nodes
ENCODE_OPS_PER_NODE, ENCODE_OPS_PER_RAY = 20, 10
LATENCY_STEPS = 200  # step latencies for p50/p99 are taken over at least this many timed steps


def sort_bytes_per_key(passes: int, key_bytes: int = 4) -> int:
    """Histogram read + first pass (ids synthesised) + middle passes + last pass (perm only)."""
    if passes <= 0:
        return key_bytes + 4
    if passes == 1:
        return key_bytes + key_bytes + 4
    return key_bytes + (key_bytes + key_bytes + 4) + (passes - 2) * 2 * (key_bytes + 4) + (key_bytes + 4 + 4)


def active_digit_passes(keys_t, key_bits: int) -> int:
    """8-bit digit passes whose digit is not the same for every key (the sort skips the others)."""
    k = keys_t.cpu().numpy().view(np.uint32 if key_bits <= 32 else np.uint64).astype(np.uint64)
    passes = 0
    for p in range((key_bits + 7) // 8):
        d = (k >> np.uint64(8 * p)) & np.uint64(255)
        passes += int(not np.all(d == d[0]))
    return passes


# ----------------------------------------------------------- distributed

def dist_env():
    """(rank, world, local_rank) from the torchrun environment (1 process by default)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def shard_seed(base_seed: int, rank: int) -> int:
    """Each rank traces its own wavefront: same scene, its own ray samples."""
    return base_seed + 1000 * rank


def reduce_max(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.dev = device_index
        self.path = os.path.join(tempfile.gettempdir(), f"hcc_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- workload

def make_workload(seed: int, quick: bool, shadow: bool = False, limited: bool = False):
    from paper_2305_16652_gb300 import gen
    camera = gen.LIMITED_CAMERA if limited else gen.ROOM_CAMERA
    if quick:
        return gen.room_workload(seed, target_tris=200_000, W=480, H=270, spp=8, shadow=shadow, camera=camera)
    return gen.room_workload(seed, target_tris=1_000_000, W=1920, H=1080, spp=8, shadow=shadow, camera=camera)


def peaks():
    try:
        p = json.load(open(PEAKS_FILE))
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, 2070.0, "fallback"


def recorded_trace_counters():
    """DRAM bytes and instruction counts of one HCC-order trace launch from the
    committed ncu summary, if trace.cu is unchanged (else an empty dict)."""
    try:
        rec = {}
        for line in open(TRAFFIC_FILE):
            if line.startswith("#") or ":" not in line:
                continue
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
        src = open(os.path.join(ROOT, "paper_2305_16652_gb300", "csrc", "trace.cu"), "rb").read()
        if rec.get("trace_cu_sha256") != hashlib.sha256(src).hexdigest():
            return {}
        return {k: int(rec[k]) for k in ("dram_bytes_per_launch", "warp_instructions", "lane_instructions") if k in rec}
    except Exception:
        return {}


# ------------------------------------------------------------- our path

def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2305_16652_gb300 import hcc

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = make_workload(shard_seed(1, rank), args.quick)
    n = w.rays.n
    K, C = args.key_bits, args.cut_size
    ctx = hcc.hcc_create(local_rank)
    bvh = hcc.hcc_bvh_upload(ctx, w.bvh, layout=args.layout)
    bvh_q = hcc.hcc_bvh_upload(ctx, w.bvh, layout="quantised")
    cut = hcc.hcc_select_cut(ctx, bvh, C, 0.125)
    hcc.hcc_reserve(ctx, n, K)
    org = torch.from_numpy(w.rays.org).to(dev)
    dir_ = torch.from_numpy(w.rays.dir).to(dev)
    keys = torch.empty(n, dtype=torch.int32, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    sorg, sdir = torch.empty_like(org), torch.empty_like(dir_)
    # the same rays as 32-byte records (origin then direction) for the record legs
    rec = torch.cat([org, dir_], 1)
    srec = torch.empty_like(rec)
    hits = torch.empty((n, 4), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    shapes = {"nosort": (128, hcc.HCC_TRACE_STACK), "sorted": (128, hcc.HCC_TRACE_STACK)}

    def step(method, ev=None, fused=True, bvh_h=None, schedule="auto", records=False):
        """One wavefront through the C ABI; ev = 5 events around encode/sort/gather/trace.
        records: the rays as 32-byte records instead of two float4 arrays."""
        b = bvh_h or bvh
        o, d = (rec[:, :4], rec[:, 4:]) if records else (org, dir_)
        so, sd = (srec[:, :4], srec[:, 4:]) if records else (sorg, sdir)
        hcc.hcc_set_trace_schedule(ctx, schedule)
        hcc.hcc_set_trace_shape(ctx, *shapes["nosort" if method == "nosort" else "sorted"])
        if ev:
            ev[0].record(stream)
        if method == "nosort":
            if ev:
                for e in ev[1:4]:
                    e.record(stream)
            hcc.hcc_trace(ctx, b, o, d, hits)
            if ev:
                ev[4].record(stream)
            return
        hcc.hcc_encode(ctx, method, b, cut if method == "hcc" else None, o, d, K, keys)
        if ev:
            ev[1].record(stream)
        hcc.hcc_sort(ctx, keys, K, n, perm)
        if ev:
            ev[2].record(stream)
        if fused:  # the trace fetches each ray through the sorted ids (Sec. 5)
            if ev:
                ev[3].record(stream)
            hcc.hcc_trace_sorted(ctx, b, o, d, perm, hits)
        else:
            hcc.hcc_gather(ctx, o, d, perm, so, sd)
            if ev:
                ev[3].record(stream)
            hcc.hcc_trace(ctx, b, so, sd, hits, scatter=perm)
        if ev:
            ev[4].record(stream)

    def timed(method, steps, warmup, **kw):
        for _ in range(warmup):
            step(method, **kw)
        hcc.hcc_sync(ctx)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(steps):
            step(method, evs[i], **kw)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        hcc.hcc_sync(ctx)
        barrier(world)
        per = [evs[i][0].elapsed_time(evs[i][4]) for i in range(steps)]
        stages = [[evs[i][s].elapsed_time(evs[i][s + 1]) for i in range(steps)] for s in range(4)]
        total_ms = evs[0][0].elapsed_time(evs[-1][4])
        return dict(per=per, stages=stages, total_ms=total_ms, wall_s=wall)

    # the trace shape (threads per block, stack entries) picked by the
    # autotuner, separately for the unsorted and the HCC-order trace
    shape_ms = tune_shapes(ctx, bvh, args.layout, org, dir_, keys, perm, hits, cut, K)
    shapes["nosort"] = min(shape_ms["nosort"], key=shape_ms["nosort"].get)
    shapes["sorted"] = min(shape_ms["hcc"], key=shape_ms["hcc"].get)

    # context for the headline: NoSort, TwoPoint, the split-gather HCC path and
    # the quantised node layout; then the HCC headline
    others = {}
    variants = [("nosort", "nosort", {}), ("twopoint", "twopoint", {}),
                ("hcc_split_gather", "hcc", {"fused": False}),
                ("hcc_records", "hcc", {"records": True}),
                ("hcc_split_gather_records", "hcc", {"fused": False, "records": True}),
                ("nosort_quantised", "nosort", {"bvh_h": bvh_q}), ("hcc_quantised", "hcc", {"bvh_h": bvh_q}),
                ("nosort_per_ray", "nosort", {"schedule": "per_ray"}), ("hcc_per_ray", "hcc", {"schedule": "per_ray"}),
                ("twopoint_per_ray", "twopoint", {"schedule": "per_ray"})]
    for name, method, kw in variants:
        r = timed(method, max(3, args.steps // 2), args.warmup, **kw)
        t_max = reduce_max(r["total_ms"], world)
        others[name] = dict(mrays_s=round(n * world * (len(r["per"])) / (t_max * 1e3), 2),
                            ms_per_step=round(t_max / len(r["per"]), 3),
                            stages_ms=dict(zip(("encode", "sort", "gather", "trace"),
                                               [round(statistics.mean(x), 4) for x in r["stages"]])))
    lat_steps = max(LATENCY_STEPS, args.steps)
    with ClockSampler(local_rank) as clk:
        r = timed("hcc", args.steps, args.warmup)
        # step latency: events around each of at least 200 back-to-back steps
        # (no host synchronisation inside), after the warm-up above
        lat = timed("hcc", lat_steps, 0)
    clocks = clk.summary()
    t_max = reduce_max(r["total_ms"], world)
    ms_step = t_max / args.steps
    value = n * world * args.steps / (t_max * 1e3)  # Mrays/s over all ranks
    per = sorted(lat["per"])
    p50 = statistics.median(per)
    p99 = per[min(len(per) - 1, int(round(0.99 * (len(per) - 1))))]
    st = [statistics.mean(x) for x in r["stages"]]
    g_split = others["hcc_split_gather"]["stages_ms"]["gather"]
    g_split_rec = others["hcc_split_gather_records"]["stages_ms"]["gather"]

    # e2e through the public host-buffer call: H2D rays, pipeline, D2H hits
    h_org = torch.empty((n, 4), dtype=torch.float32, pin_memory=True)
    h_dir = torch.empty((n, 4), dtype=torch.float32, pin_memory=True)
    h_org.copy_(torch.from_numpy(w.rays.org))
    h_dir.copy_(torch.from_numpy(w.rays.dir))
    h_hits = torch.empty((n, 4), dtype=torch.int32, pin_memory=True)
    a_org, a_dir, a_hits = h_org.numpy(), h_dir.numpy(), h_hits.numpy()
    for _ in range(2):
        hcc.hcc_run_host(ctx, "hcc", bvh, cut, a_org, a_dir, K, a_hits)
    e2e_steps = max(3, min(args.steps, 10))
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        hcc.hcc_run_host(ctx, "hcc", bvh, cut, a_org, a_dir, K, a_hits)
    e2e_s = reduce_max(time.perf_counter() - t0, world)
    e2e_value = n * world * e2e_steps / (e2e_s * 1e6)

    # a short serving leg on the same scene: Poisson arrivals at half the
    # 4-slot saturation, continuous admission against the unbatched path
    serving = (serve_leg(local_rank, bvh, cut, h_org, h_dir, K, args.serve_requests_bench)
               if args.serve_requests_bench else None)

    # parity of the timed path (sorted vs unsorted bit-identical)
    step("hcc")
    hcc.hcc_sync(ctx)
    h_hcc = hits.clone()
    gpu_keys = keys.cpu().numpy().view(np.uint32).astype(np.uint64)
    step("nosort")
    hcc.hcc_sync(ctx)
    identical = bool(torch.equal(h_hcc, hits))
    gpu_hits = hcc.hits_to_numpy(h_hcc)

    # work counts of the trace (order-independent per ray) for the ALU roofline
    counts = hcc.hcc_trace_counts(ctx, bvh, org, dir_, perm=perm)
    counts0 = hcc.hcc_trace_counts(ctx, bvh, org, dir_)
    hcc.hcc_bvh_destroy(bvh_q)
    hbm, sm_max, peak_kind = peaks()
    clk_mhz = clocks.get("sm_max_mhz") or sm_max
    alu_peak = SMS * LANES_PER_SM * clk_mhz * 1e6 / 1e12  # Tops/s
    trace_ms = st[3]
    work = counts["node_visits"] * OPS_PER_NODE[args.layout] + counts["tri_tests"] * OPS_PER_TRI
    achieved = work / (trace_ms * 1e-3) / 1e12
    tc = recorded_trace_counters() if args.layout == "exact" and C == 32 and K == 32 else {}
    measured = None
    if "lane_instructions" in tc:  # counters of the same launch (ncu), over this run's trace time
        measured = {"lane_instructions_per_ray": round(tc["lane_instructions"] / n, 1),
                    "active_lanes": round(tc["lane_instructions"] / tc["warp_instructions"], 2),
                    "issue_frac": round(tc["warp_instructions"] / (trace_ms * 1e-3) / (SMS * 4 * clk_mhz * 1e6), 3),
                    "lane_frac": round(tc["lane_instructions"] / (trace_ms * 1e-3) / 1e12 / alu_peak, 3),
                    "source": "ncu counters of one launch (profiles/trace_room_1080p_dram.txt)"}
    sort_passes = active_digit_passes(keys, K)
    sb = sort_bytes_per_key(sort_passes)
    enc_ops = (ENCODE_OPS_PER_NODE * min(C, K) + ENCODE_OPS_PER_RAY) * n
    enc_tops = enc_ops / (st[0] * 1e-3) / 1e12
    stages = {
        "encode": dict(ms=round(st[0], 4), bound="alu", ops_per_ray=ENCODE_OPS_PER_NODE * min(C, K) + ENCODE_OPS_PER_RAY,
                       achieved_tops=round(enc_tops, 3), frac=round(enc_tops / alu_peak, 3),
                       achieved_gbs=round(BYTES_ENCODE * n / (st[0] * 1e6), 1),
                       hbm_frac=round(BYTES_ENCODE * n / (st[0] * 1e6) / hbm, 3)),
        "sort": dict(ms=round(st[1], 4), bound="hbm", active_passes=sort_passes, bytes_per_key=sb,
                     achieved_gbs=round(sb * n / (st[1] * 1e6), 1), frac=round(sb * n / (st[1] * 1e6) / hbm, 3)),
        "gather": dict(ms=0.0, fused_into_trace=True, split_kernel_ms=round(g_split, 4), bound="hbm",
                       split_achieved_gbs=round(BYTES_GATHER * n / (g_split * 1e6), 1),
                       split_frac=round(BYTES_GATHER * n / (g_split * 1e6) / hbm, 3),
                       split_kernel_ms_records=round(g_split_rec, 4),
                       split_achieved_gbs_records=round(BYTES_GATHER * n / (g_split_rec * 1e6), 1),
                       split_frac_records=round(BYTES_GATHER * n / (g_split_rec * 1e6) / hbm, 3)),
        "trace": dict(ms=round(st[3], 4), bound="alu", achieved_tops=round(achieved, 3),
                      frac=round(achieved / alu_peak, 3),
                      node_visits_per_ray=round(counts["node_visits"] / n, 2),
                      tri_tests_per_ray=round(counts["tri_tests"] / n, 2),
                      warp_efficiency=round(counts["node_visits"] / (32.0 * max(1, counts["warp_node_steps"])), 4),
                      warp_efficiency_nosort=round(counts0["node_visits"] / (32.0 * max(1, counts0["warp_node_steps"])), 4),
                      measured=measured),
    }
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name + f" ({n} secondary rays), HCC cut {C}, {K}-bit keys, {args.layout} BVH nodes",
                   "bvh_layout": args.layout, "gather": "fused into the trace (rays fetched through the sorted ids)",
                   "trace_schedule": "auto (closest hit: persistent warps with ray replacement)",
                   "trace_shape": {"hcc": list(shapes["sorted"]), "nosort": list(shapes["nosort"]),
                                   "searched_ms": {o: {f"{b}x{st}": round(v, 4) for (b, st), v in t.items()}
                                                   for o, t in shape_ms.items()}},
                   "rays": n, "triangles": int(w.tris.shape[0]), "cut_size": C, "key_bits": K, "lambda": 0.125,
                   "l2": f"inputs larger than L2 ({n * 32 / 1e6:.0f} MB of rays per step)",
                   "parallelism": f"replica per GPU x{world}"},
        "p50_ms": round(p50, 4), "p99_ms": round(p99, 4), "latency_steps": len(per),
        "stages_ms": {"encode": round(st[0], 4), "sort": round(st[1], 4), "gather": round(st[2], 4),
                      "trace": round(st[3], 4)},
        "methods": {"hcc": {"mrays_s": round(value, 2), "ms_per_step": round(ms_step, 3)}, **others},
        "speedup_vs_nosort": round(value / others["nosort"]["mrays_s"], 3),
        "trace_speedup_vs_nosort": round(others["nosort"]["stages_ms"]["trace"] / st[3], 3),
        "speedup_vs_twopoint": round(value / others["twopoint"]["mrays_s"], 3),
        "hits_identical_hcc_vs_nosort": identical,
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": int(n * 32),
                "d2h_bytes_per_step": int(n * 16), "call": "hcc_run_host"},
        "gpu_launches": 7 * args.steps,  # per step: encode, sort histogram + 4 digit passes, trace
        "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(alu_peak, 2), "unit": "Tops/s",
                     "frac": round(achieved / alu_peak, 3), "traffic": tc.get("dram_bytes_per_launch"),
                     "kernel": f"k_trace_pool (closest hit, HCC order, {args.layout} nodes, ray replacement)",
                     "peak_source": f"{SMS} SMs x {LANES_PER_SM} lanes x {clk_mhz:.0f} MHz"},
        "stages": stages,
        "hbm_peak_gbs": hbm, "hbm_peak_source": peak_kind,
        "clocks": clocks,
    }
    if serving is not None:
        out["serving"] = serving
    hcc.hcc_cut_destroy(cut)
    hcc.hcc_bvh_destroy(bvh)
    hcc.hcc_destroy(ctx)
    return out, w, {"keys": gpu_keys, "hits": gpu_hits}


def tune_shapes(ctx, bvh, layout, org, dir_, keys, perm, hits, cut, key_bits, reps=3):
    """Trace time (ms, median of reps) of every trace shape the autotuner may
    pick for this BVH, for the unsorted wavefront and in HCC order."""
    import torch
    from paper_2305_16652_gb300 import hcc, tune
    hcc.hcc_encode(ctx, "hcc", bvh, cut, org, dir_, key_bits, keys)
    hcc.hcc_sort(ctx, keys, key_bits, int(org.shape[0]), perm)
    hcc.hcc_set_trace_schedule(ctx, "auto")
    out = {"nosort": {}, "hcc": {}}
    for shape in tune.shape_candidates([bvh], layout):
        hcc.hcc_set_trace_shape(ctx, *shape)
        for name, f in (("nosort", lambda: hcc.hcc_trace(ctx, bvh, org, dir_, hits)),
                        ("hcc", lambda: hcc.hcc_trace_sorted(ctx, bvh, org, dir_, perm, hits))):
            ts = []
            for _ in range(reps + 1):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                f()
                b.record()
                b.synchronize()
                ts.append(a.elapsed_time(b))
            out[name][shape] = statistics.median(ts[1:])
    hcc.hcc_sync(ctx)
    hcc.hcc_set_trace_shape(ctx, 0, 0)
    return out


# ------------------------------------------------------- oracle (CPU) leg

def oracle_indices(w, sample_n: int, seed: int = 7):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(w.rays.n, size=min(sample_n, w.rays.n), replace=False))


def oracle_sample(w, sample_n: int, seed: int = 7):
    idx = oracle_indices(w, sample_n, seed)
    return w.rays.org[idx].copy(), w.rays.dir[idx].copy()


def oracle_step(w, cut_ids, org, dir_, key_bits):
    """The whole path on the CPU oracle; returns the keys and the hits in input order."""
    import oracle
    keys = oracle.encode_hcc(org, dir_, w.bvh.lo[cut_ids], w.bvh.hi[cut_ids], key_bits)
    perm = oracle.stable_sort(keys)
    so, sd = oracle.gather(org, dir_, perm)
    hs = oracle.trace_bvh(w.bvh, so, sd)
    hits = np.empty_like(hs)
    hits[perm] = hs
    return keys, hits


def parity_counts(w, cut_ids, org, dir_, idx, keys_o, hits_o, gpu, key_bits):
    """GPU keys and hits of the sampled rays against the oracle's, with the
    tolerances of the parity tests: a key may differ only on a ray whose slab
    margin is below 1e-6; a hit only on a near-edge tie (the oracle's hit
    within 1e-6 of an edge, t within 1e-5 relative)."""
    import oracle
    lo, hi = w.bvh.lo[cut_ids], w.bvh.hi[cut_ids]
    kg = gpu["keys"][idx]
    kbad = np.nonzero(kg != keys_o)[0]
    kmarg = oracle.key_margin(org[kbad], dir_[kbad], lo, hi, key_bits) if len(kbad) else np.zeros(0)
    marginal_rays = int(np.sum(oracle.key_margin(org, dir_, lo, hi, key_bits) < 1e-6))
    hg = gpu["hits"][idx]
    gi, oi = hg.view(np.int32).reshape(-1, 4), hits_o.view(np.int32).reshape(-1, 4)
    hbad = np.nonzero(np.any(gi != oi, axis=1))[0]
    ties = 0
    for i in hbad:
        g, o = hg[i], hits_o[i]
        gh, oh = int(g["prim"]) >= 0, int(o["prim"]) >= 0
        ref = o if oh else g
        margin = min(float(ref["u"]), float(ref["v"]), 1.0 - float(ref["u"]) - float(ref["v"]))
        same_prim = gh and oh and int(g["prim"]) == int(o["prim"])
        t_ok = (not (gh and oh)) or abs(float(g["t"]) - float(o["t"])) <= 1e-5 * abs(float(o["t"]))
        ties += int(not same_prim and margin < 1e-6 and t_ok)
    return {"rays": int(len(idx)), "key_mismatches": int(len(kbad)),
            "key_mismatches_not_marginal": int(np.sum(kmarg >= 1e-6)), "marginal_rays": marginal_rays,
            "hit_mismatches": int(len(hbad)), "near_edge_ties": int(ties),
            "hit_mismatches_not_tolerated": int(len(hbad) - ties)}


def cpu_baseline(w, key_bits, cut_size, sample_n, gpu=None):
    import oracle
    cut_ids = oracle.select_cut(w.bvh, cut_size)
    idx = oracle_indices(w, sample_n)
    org, dir_ = w.rays.org[idx].copy(), w.rays.dir[idx].copy()
    t0 = time.perf_counter()
    keys_o, hits_o = oracle_step(w, cut_ids, org, dir_, key_bits)
    dt = time.perf_counter() - t0
    out = {"value": round(org.shape[0] / dt / 1e6, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{org.shape[0]} seeded random rays of the same wavefront, encode+sort+gather+trace, "
                     f"single-threaded C++ oracle, {dt:.1f} s"}
    parity = parity_counts(w, cut_ids, org, dir_, idx, keys_o, hits_o, gpu, key_bits) if gpu else None
    return out, parity


def run_reference(args, rank, world):
    if rank != 0:
        return None
    w = make_workload(1, args.quick)
    import oracle
    cut_ids = oracle.select_cut(w.bvh, args.cut_size)
    org, dir_ = oracle_sample(w, args.ref_sample)
    for _ in range(args.warmup):
        oracle_step(w, cut_ids, org[:1000], dir_[:1000], args.key_bits)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_step(w, cut_ids, org, dir_, args.key_bits)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = org.shape[0] * len(times) / tot / 1e6
    return {"metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * tot / len(times), 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name + f" ({w.rays.n} secondary rays), HCC cut {args.cut_size}, "
                                            f"{args.key_bits}-bit keys", "rays": w.rays.n},
            "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{org.shape[0]} seeded random rays per step, encode+sort+gather+trace"},
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_keylen_sweep(args):
    """Key-length study (Sec. 6.5, Tables 5-6): HCC (cut size = key bits), TwoPoint and
    Origin-Direction at 16/24/32/48/64 bits on the same wavefront; per point the stage
    times, ANC, distinct keys and the trace's warp execution efficiency."""
    import torch
    from paper_2305_16652_gb300 import build, hcc
    build()
    dev = torch.device("cuda", 0)
    w = make_workload(1, args.quick)
    n = w.rays.n
    ctx = hcc.hcc_create(0)
    bvh = hcc.hcc_bvh_upload(ctx, w.bvh, layout=args.layout)
    hcc.hcc_reserve(ctx, n, 64)
    org = torch.from_numpy(w.rays.org).to(dev)
    dir_ = torch.from_numpy(w.rays.dir).to(dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    hits = torch.empty((n, 4), dtype=torch.int32, device=dev)

    def tm(f, reps=5):
        ts = []
        for _ in range(reps + 2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            f()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts[2:])

    def eff(c):
        return round(c["node_visits"] / (32.0 * max(1, c["warp_node_steps"])), 4)

    c0 = hcc.hcc_trace_counts(ctx, bvh, org, dir_)
    nosort = {"trace_ms": round(tm(lambda: hcc.hcc_trace(ctx, bvh, org, dir_, hits)), 4),
              "warp_efficiency": eff(c0), "node_visits_per_ray": round(c0["node_visits"] / n, 3)}
    points = []
    for k in (16, 24, 32, 48, 64):
        keys = torch.empty(n, dtype=torch.int32 if k <= 32 else torch.int64, device=dev)
        for method in ("hcc", "twopoint", "origin_dir"):
            cut = hcc.hcc_select_cut(ctx, bvh, k, 0.125) if method == "hcc" else None
            te = tm(lambda: hcc.hcc_encode(ctx, method, bvh, cut, org, dir_, k, keys))
            ts = tm(lambda: hcc.hcc_sort(ctx, keys, k, n, perm))
            tt = tm(lambda: hcc.hcc_trace_sorted(ctx, bvh, org, dir_, perm, hits))
            st = hcc.hcc_key_stats(ctx, keys, k, perm, n)
            c = hcc.hcc_trace_counts(ctx, bvh, org, dir_, perm=perm)
            hcc.hcc_sync(ctx)
            tot = te + ts + tt
            points.append({"method": method, "key_bits": k, "encode_ms": round(te, 4), "sort_ms": round(ts, 4),
                           "trace_ms": round(tt, 4), "total_ms": round(tot, 4),
                           "mrays_s": round(n / (tot * 1e3), 2),
                           "trace_speedup_vs_nosort": round(nosort["trace_ms"] / tt, 3),
                           "anc": round(st["anc"], 4), "distinct_keys": st["distinct"],
                           "warp_efficiency": eff(c), "warp_node_steps_per_32_rays":
                               round(32.0 * c["warp_node_steps"] / n, 2)})
            if cut is not None:
                hcc.hcc_cut_destroy(cut)
    out = {"metric": "key-length sweep: secondary Mrays/s, ANC and warp execution efficiency",
           "unit": "Mrays/s", "config": {"workload": w.name + f" ({n} secondary rays)", "bvh_layout": args.layout,
                                         "hcc_cut_size": "= key bits"},
           "nosort": nosort, "points": points}
    hcc.hcc_bvh_destroy(bvh)
    hcc.hcc_destroy(ctx)
    print(json.dumps(out), flush=True)


def run_methods_sweep(args):
    """Method study (Sec. 6, Tables 1, 2 and 4): every ordering on the same 1080p
    wavefront -- NoSort, TwoPoint, Origin, Origin-Direction, HCC (cut 32), MLHCC16
    (8 + 8), MLHCC32 (16 + 16), regular grid (32 cells) and PPC (an upper bound) --
    for the secondary rays (closest hit) and the shadow rays (any hit); per method
    the encode, sort and trace times, the trace speedup over NoSort, ANC, distinct
    keys and the trace's warp execution efficiency."""
    import torch
    from paper_2305_16652_gb300 import build, hcc
    build()
    dev = torch.device("cuda", 0)
    w = make_workload(1, args.quick, shadow=True, limited=args.viewport == "limited")
    ctx = hcc.hcc_create(0)
    bvh = hcc.hcc_bvh_upload(ctx, w.bvh, layout=args.layout)

    def tm(f, reps=5):
        ts = []
        for _ in range(reps + 2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            f()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts[2:])

    def eff(c):
        return round(c["node_visits"] / (32.0 * max(1, c["warp_node_steps"])), 4)

    cuts = {"hcc": hcc.hcc_select_cut(ctx, bvh, 32, 0.125),
            "mlhcc16": hcc.hcc_select_cut_ml(ctx, bvh, 8, 8, 0.125),
            "mlhcc32": hcc.hcc_select_cut_ml(ctx, bvh, 16, 16, 0.125),
            "grid": hcc.hcc_select_grid(ctx, bvh, 32)}
    methods = [("twopoint", "twopoint", 32, None), ("origin", "origin", 32, None),
               ("origin_dir", "origin_dir", 32, None), ("hcc", "hcc", 32, "hcc"),
               ("mlhcc16", "mlhcc", 16, "mlhcc16"), ("mlhcc32", "mlhcc", 32, "mlhcc32"),
               ("regular_grid", "hcc", 32, "grid")]
    if args.layout == "exact":
        methods.append(("ppc", "ppc", 32, None))
    out = {"metric": "method study: Mrays/s, trace speedup over NoSort, ANC and warp efficiency per ordering",
           "unit": "Mrays/s", "config": {"workload": w.name, "bvh_layout": args.layout}}
    for label, rays, any_hit in (("secondary", w.rays, False), ("shadow", w.shadow, True)):
        if rays is None:
            continue
        n = rays.n
        hcc.hcc_reserve(ctx, n, 32)
        org = torch.from_numpy(rays.org).to(dev)
        dir_ = torch.from_numpy(rays.dir).to(dev)
        perm = torch.empty(n, dtype=torch.int32, device=dev)
        keys = torch.empty(n, dtype=torch.int32, device=dev)
        hits = torch.empty((n, 4), dtype=torch.int32, device=dev)
        c0 = hcc.hcc_trace_counts(ctx, bvh, org, dir_, any_hit=any_hit)
        t0 = tm(lambda: hcc.hcc_trace(ctx, bvh, org, dir_, hits, any_hit=any_hit))
        rows = {"nosort": {"trace_ms": round(t0, 4), "mrays_s": round(n / (t0 * 1e3), 1),
                           "warp_efficiency": eff(c0), "node_visits_per_ray": round(c0["node_visits"] / n, 3)}}
        for name, method, k, cut_name in methods:
            cut = cuts[cut_name] if cut_name else None
            te = tm(lambda: hcc.hcc_encode(ctx, method, bvh, cut, org, dir_, k, keys))
            ts = tm(lambda: hcc.hcc_sort(ctx, keys, k, n, perm))
            tt = tm(lambda: hcc.hcc_trace_sorted(ctx, bvh, org, dir_, perm, hits, any_hit=any_hit))
            st = hcc.hcc_key_stats(ctx, keys, k, perm, n)
            c = hcc.hcc_trace_counts(ctx, bvh, org, dir_, perm=perm, any_hit=any_hit)
            hcc.hcc_sync(ctx)
            tot = te + ts + tt
            rows[name] = {"key_bits": k, "encode_ms": round(te, 4), "sort_ms": round(ts, 4), "trace_ms": round(tt, 4),
                          "total_ms": round(tot, 4), "mrays_s": round(n / (tot * 1e3), 1),
                          "trace_mrays_s": round(n / (tt * 1e3), 1),
                          "trace_speedup_vs_nosort": round(t0 / tt, 3), "speedup_vs_nosort": round(t0 / tot, 3),
                          "overhead_pct_of_trace": round(100 * (te + ts) / tt, 1), "anc": round(st["anc"], 4),
                          "distinct_keys": st["distinct"], "warp_efficiency": eff(c),
                          "node_visits_per_ray": round(c["node_visits"] / n, 3)}
        out[label] = {"rays": n, "any_hit": any_hit, "methods": rows}
        del org, dir_, perm, keys, hits
        torch.cuda.empty_cache()
    for c in cuts.values():
        hcc.hcc_cut_destroy(c)
    hcc.hcc_bvh_destroy(bvh)
    hcc.hcc_destroy(ctx)
    print(json.dumps(out), flush=True)


def run_hyper_sweep(args):
    """Hyperparameter study (App. B): the HAD weight lambda of Eq. 1 for HCC (cut 32,
    32-bit keys) and the TwoPoint estimated ray length as a fraction of the largest
    scene extent, each from 0.1 to 1.0, and the HCC cut size from 32 to 4096 nodes at
    32-bit keys, on the 1080p wavefront; per point the stage times, end-to-end
    Mrays/s, trace speedup over NoSort and ANC."""
    import torch
    from paper_2305_16652_gb300 import build, hcc
    build()
    dev = torch.device("cuda", 0)
    w = make_workload(1, args.quick)
    n = w.rays.n
    ctx = hcc.hcc_create(0)
    bvh = hcc.hcc_bvh_upload(ctx, w.bvh, layout=args.layout)
    hcc.hcc_reserve(ctx, n, 32)
    org = torch.from_numpy(w.rays.org).to(dev)
    dir_ = torch.from_numpy(w.rays.dir).to(dev)
    keys = torch.empty(n, dtype=torch.int32, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    hits = torch.empty((n, 4), dtype=torch.int32, device=dev)

    def tm(f, reps=5):
        ts = []
        for _ in range(reps + 2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            f()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts[2:])

    t0 = tm(lambda: hcc.hcc_trace(ctx, bvh, org, dir_, hits))

    def point(method, cut):
        te = tm(lambda: hcc.hcc_encode(ctx, method, bvh, cut, org, dir_, 32, keys))
        ts = tm(lambda: hcc.hcc_sort(ctx, keys, 32, n, perm))
        tt = tm(lambda: hcc.hcc_trace_sorted(ctx, bvh, org, dir_, perm, hits))
        st = hcc.hcc_key_stats(ctx, keys, 32, perm, n)
        hcc.hcc_sync(ctx)
        return {"encode_ms": round(te, 4), "sort_ms": round(ts, 4), "trace_ms": round(tt, 4),
                "mrays_s": round(n / ((te + ts + tt) * 1e3), 1), "trace_speedup_vs_nosort": round(t0 / tt, 3),
                "anc": round(st["anc"], 4)}

    grid = [round(0.1 * i, 1) for i in range(1, 11)]
    lam_rows, tp_rows = [], []
    for lam in grid:
        cut = hcc.hcc_select_cut(ctx, bvh, 32, lam)
        lam_rows.append({"lambda": lam, **point("hcc", cut)})
        hcc.hcc_cut_destroy(cut)
    for f in grid:
        hcc.hcc_set_twopoint_distance(ctx, f)
        tp_rows.append({"fraction": f, **point("twopoint", None)})
    hcc.hcc_set_twopoint_distance(ctx, 0.25)
    # cut size at 32-bit keys: Algorithm 2 run to C nodes, the key built from
    # the 32 of highest HAD (a larger C reaches deeper, smaller nodes)
    cut_rows = []
    for c in (32, 64, 128, 256, 512, 1024, 2048, 4096):
        cut = hcc.hcc_select_cut(ctx, bvh, c, 0.125)
        cut_rows.append({"cut_size": c, **point("hcc", cut)})
        hcc.hcc_cut_destroy(cut)
    out = {"metric": "hyperparameter study: HCC lambda and cut size, TwoPoint length fraction", "unit": "Mrays/s",
           "config": {"workload": w.name + f" ({n} secondary rays)", "bvh_layout": args.layout, "cut_size": 32,
                      "key_bits": 32},
           "nosort_trace_ms": round(t0, 4), "hcc_lambda": lam_rows, "twopoint_fraction": tp_rows,
           "hcc_cut_size": cut_rows}
    hcc.hcc_bvh_destroy(bvh)
    hcc.hcc_destroy(ctx)
    print(json.dumps(out), flush=True)


def run_batch_sweep(args):
    """Batched wavefronts: 16 rooms (seeds 2-17, 50k-2M triangles) with log-uniform
    wavefronts of 64k-8M rays, two bounces, each bounce one captured CUDA graph
    (fused multi-scene encode, one sort, one fused trace; bounce 2 starts with the
    spawn kernel), autotuned per-scene cut size and shared key length."""
    import torch
    from paper_2305_16652_gb300 import build, gen, hcc, tune
    build()
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    ws = gen.batch_workloads(scale=0.125 if args.quick else 1.0)
    gen_s = time.perf_counter() - t0
    S = len(ws)
    stream = torch.cuda.Stream()
    ctx = hcc.hcc_create(0, stream)
    bvhs = [hcc.hcc_bvh_upload(ctx, w.bvh, layout=args.layout) for w in ws]
    offsets = np.concatenate([[0], np.cumsum([w.rays.n for w in ws])]).astype(np.uint64)
    n = int(offsets[-1])
    with torch.cuda.stream(stream):
        org1 = torch.from_numpy(np.concatenate([w.rays.org for w in ws])).to(dev)
        dir1 = torch.from_numpy(np.concatenate([w.rays.dir for w in ws])).to(dev)
        org2, dir2 = torch.empty_like(org1), torch.empty_like(dir1)
        hits1 = torch.empty((n, 4), dtype=torch.int32, device=dev)
        hits2 = torch.empty_like(hits1)
    stream.synchronize()
    per_scene = [(org1[int(offsets[s]):int(offsets[s + 1])], dir1[int(offsets[s]):int(offsets[s + 1])])
                 for s in range(S)]
    t0 = time.perf_counter()
    tuned = tune.tune_batch(ctx, stream, bvhs, per_scene)
    tune_s = time.perf_counter() - t0
    cuts = [hcc.hcc_select_cut(ctx, b, C, lam) for b, C, lam in zip(bvhs, tuned["cut_sizes"], tuned["lambdas"])]
    batch = hcc.hcc_batch_create(ctx, bvhs, cuts, offsets)
    hcc.hcc_reserve(ctx, n, 64)
    results = {}
    for name, method, k in (("nosort", "nosort", 32), ("twopoint", "twopoint", 30),
                            ("hcc_tuned", "hcc", tuned["key_bits"]), ("hcc_32", "hcc", 32)):
        if name == "hcc_32":
            for c in cuts:
                hcc.hcc_cut_destroy(c)
            cuts = [hcc.hcc_select_cut(ctx, b, 32, 0.125) for b in bvhs]
            hcc.hcc_batch_destroy(batch)
            batch = hcc.hcc_batch_create(ctx, bvhs, cuts, offsets)
        hcc.hcc_graph_begin(ctx)
        hcc.hcc_batch_run(ctx, batch, method, org1, dir1, k, hits1)
        g1 = hcc.hcc_graph_end(ctx)
        hcc.hcc_graph_begin(ctx)
        hcc.hcc_batch_spawn(ctx, batch, org1, dir1, hits1, 1234, 1e-4, org2, dir2)
        hcc.hcc_batch_run(ctx, batch, method, org2, dir2, k, hits2)
        g2 = hcc.hcc_graph_end(ctx)
        times = {}
        for label, g in (("bounce1", g1), ("bounce2_with_spawn", g2)):
            for _ in range(args.warmup):
                hcc.hcc_graph_launch(ctx, g)
            hcc.hcc_sync(ctx)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            for a, b in evs:
                a.record(stream)
                hcc.hcc_graph_launch(ctx, g)
                b.record(stream)
            hcc.hcc_sync(ctx)
            times[label] = statistics.median([a.elapsed_time(b) for a, b in evs])
        # the same bounce issued call by call (no graph), for the launch overhead
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        for a, b in evs:
            a.record(stream)
            hcc.hcc_batch_run(ctx, batch, method, org1, dir1, k, hits1)
            b.record(stream)
        hcc.hcc_sync(ctx)
        times["bounce1_eager"] = statistics.median([a.elapsed_time(b) for a, b in evs])
        hcc.hcc_graph_destroy(g1)
        hcc.hcc_graph_destroy(g2)
        results[name] = {"key_bits": k, **{f"{kk}_ms": round(v, 4) for kk, v in times.items()},
                         "bounce1_mrays_s": round(n / (times["bounce1"] * 1e3), 1),
                         "two_bounces_mrays_s": round(2 * n / ((times["bounce1"] + times["bounce2_with_spawn"]) * 1e3),
                                                      1)}
    out = {"metric": "batched wavefronts: secondary Mrays/s over 2 bounces, one CUDA graph per bounce",
           "unit": "Mrays/s",
           "config": {"workload": f"{S} rooms (seeds 2-17), {sum(w.tris.shape[0] for w in ws)} triangles, "
                                  f"{n} rays per bounce", "bvh_layout": args.layout,
                      "scenes": [{"tris": int(w.tris.shape[0]), "rays": int(w.rays.n)} for w in ws]},
           "autotune": {"key_bits": tuned["key_bits"], "cut_sizes": tuned["cut_sizes"], "lambdas": tuned["lambdas"],
                        "schedule": tuned["schedule"], "shape": list(tuned["shape"]), "shape_ms": tuned["shape_ms"],
                        "totals_ms": tuned["totals_ms"], "seconds": round(tune_s, 1)},
           "generation_s": round(gen_s, 1), "methods": results}
    for c in cuts:
        hcc.hcc_cut_destroy(c)
    hcc.hcc_batch_destroy(batch)
    for b in bvhs:
        hcc.hcc_bvh_destroy(b)
    hcc.hcc_destroy(ctx)
    print(json.dumps(out), flush=True)


class _HitRing:
    """Page-locked hit records handed out to in-flight requests in a ring.

    A region is reused only after every request writing into it has finished:
    take() first collects finished requests and then waits for any unfinished
    one that overlaps the new region (counted as a stall)."""

    def __init__(self, torch, size: int):
        self.buf = torch.empty((size, 4), dtype=torch.int32).pin_memory()
        self.size, self.head = size, 0
        self.live = []  # [ticket, start, end, submit_time]
        self.stalls = 0

    def take(self, n: int, server, done):
        from paper_2305_16652_gb300 import hcc
        if self.head + n > self.size:
            self.head = 0
        a, b = self.head, self.head + n
        self.collect(server, done)
        keep = []
        for item in self.live:
            if item[1] < b and a < item[2]:
                self.stalls += 1
                done.append((item[3], hcc.hcc_server_wait(server, item[0]), item[2] - item[1]))
            else:
                keep.append(item)
        self.live = keep
        self.head = b
        return a, self.buf[a:b]

    def collect(self, server, done, block: bool = False):
        from paper_2305_16652_gb300 import hcc
        keep = []
        for item in self.live:
            if block or hcc.hcc_server_query(server, item[0]):
                done.append((item[3], hcc.hcc_server_wait(server, item[0]), item[2] - item[1]))
            else:
                keep.append(item)
        self.live = keep


def _serve_run(server, ring, pools, reqs, count, rate=None, outstanding=None):
    """Submit requests 0..count-1 of the stream: open loop with Poisson arrivals
    at `rate` requests/s, or closed loop keeping `outstanding` requests queued.
    Returns (completed Mrays/s over the makespan, latencies in ms, stats)."""
    from paper_2305_16652_gb300 import hcc
    done = []
    ring.stalls = 0
    t0 = time.perf_counter()
    arrive = t0 + np.cumsum(reqs["gap"][:count]) / rate if rate else None
    for i in range(count):
        s, n, off = int(reqs["scene"][i]), int(reqs["n"][i]), int(reqs["offset"][i])
        if rate:
            polled = 0.0
            while True:
                now = time.perf_counter()
                if now >= arrive[i]:
                    break
                if now - polled > 2e-4:  # collect finished requests without contending for the server's lock
                    ring.collect(server, done)
                    polled = now
        else:
            while len(ring.live) >= outstanding:
                oldest = ring.live.pop(0)
                done.append((oldest[3], hcc.hcc_server_wait(server, oldest[0]), oldest[2] - oldest[1]))
        a, hits = ring.take(n, server, done)
        org, dir_ = pools[s]
        t = time.perf_counter()
        ticket = hcc.hcc_server_submit(server, s, org[off:off + n], dir_[off:off + n], hits)
        ring.live.append([ticket, a, a + n, t])
    ring.collect(server, done, block=True)
    first = min(d[0] for d in done)
    last = max(d[0] + d[1] / 1e3 for d in done)
    rays = sum(d[2] for d in done)
    lat = np.array([d[1] for d in done])
    return rays / (last - first) / 1e6, lat, hcc.hcc_server_stats_get(server)


def _warm_server(srv, reqs, pools, ring, slots, count):
    """Grow a server's memory pool to the largest request on every slot (so
    that no timed request waits for the driver to map memory), then run a few
    requests through it."""
    import torch
    from paper_2305_16652_gb300 import hcc
    big = int(np.argmax(reqs["n"][:count]))
    s, n, off = int(reqs["scene"][big]), int(reqs["n"][big]), int(reqs["offset"][big])
    hits_w = [torch.empty((n, 4), dtype=torch.int32).pin_memory() for _ in range(slots)]
    tickets = [hcc.hcc_server_submit(srv, s, pools[s][0][off:off + n], pools[s][1][off:off + n], h) for h in hits_w]
    for t in tickets:
        hcc.hcc_server_wait(srv, t)
    _serve_run(srv, ring, pools, reqs, min(24, count), outstanding=2 * slots)


def _serve_summary(mrays, lat, st, ring):
    return {"mrays_s": round(mrays, 1), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
            "max_in_flight": st["max_in_flight"], "ring_stalls": ring.stalls}


def serve_leg(device, bvh, cut, h_org, h_dir, key_bits, count, slots=4, load=0.5, seed=3):
    """Serving on the headline scene: `count` ray-query requests (64k-4M rays,
    log-uniform, windows of the wavefront in page-locked host memory) with
    Poisson arrivals at `load` of the continuous server's closed-loop
    saturation; p50/p99 latency and Mrays/s of continuous admission (`slots`
    requests on the GPU) and of the unbatched path (one at a time)."""
    import torch
    from paper_2305_16652_gb300 import gen, hcc
    pools = [(h_org, h_dir)]
    reqs = gen.serve_requests(seed, count, [int(h_org.shape[0])])
    ring = _HitRing(torch, 24 << 20)

    def server(k):
        srv = hcc.hcc_server_create(device, [bvh], [cut], slots=k, method="hcc", key_bits=key_bits)
        _warm_server(srv, reqs, pools, ring, k, count)
        return srv

    srv = server(slots)
    try:
        sat, lat, st = _serve_run(srv, ring, pools, reqs, count, outstanding=2 * slots)
    finally:
        hcc.hcc_server_destroy(srv)
    mean_rays = float(reqs["n"][:count].mean())
    rate = load * sat * 1e6 / mean_rays
    out = {"requests": count, "rays_per_request": f"64k-4M log-uniform (mean {int(mean_rays)})",
           "saturation": {"slots": slots, **_serve_summary(sat, lat, st, ring)},
           "load": load, "offered_req_s": round(rate, 1), "offered_mrays_s": round(load * sat, 1)}
    for name, k in (("continuous", slots), ("unbatched", 1)):
        srv = server(k)
        try:
            m, lat, st = _serve_run(srv, ring, pools, reqs, count, rate=rate)
        finally:
            hcc.hcc_server_destroy(srv)
        out[name] = _serve_summary(m, lat, st, ring)
    return out


def run_serve_sweep(args):
    """Serving loop: Poisson arrivals of ray queries (64k-4M rays, log-uniform)
    against 8 resident rooms of 0.2-4M triangles; per-request HCC encode, sort
    and trace with host buffers; throughput and p50/p99 latency of the
    continuous-admission server against the unbatched per-request path (one
    request on the GPU at a time) at 25/50/90% of the server's saturation."""
    import torch
    from paper_2305_16652_gb300 import build, gen, hcc
    build()
    scale = 0.125 if args.quick else 1.0
    t0 = time.perf_counter()
    ws = gen.serve_scenes(scale=scale)
    gen_s = time.perf_counter() - t0
    rr = (65_536, 4_194_304) if not args.quick else (8_192, 524_288)
    count = args.serve_requests
    reqs = gen.serve_requests(1, count, [w.rays.n for w in ws], rays_range=rr)
    ctx = hcc.hcc_create(0)
    bvhs = [hcc.hcc_bvh_upload(ctx, w.bvh, layout=args.layout) for w in ws]
    cuts = [hcc.hcc_select_cut(ctx, b, args.cut_size, 0.125) for b in bvhs]
    pools = [(torch.from_numpy(w.rays.org).pin_memory(), torch.from_numpy(w.rays.dir).pin_memory()) for w in ws]
    ring = _HitRing(torch, 64 << 20 if not args.quick else 8 << 20)
    key_bits = args.key_bits

    def server(slots):
        srv = hcc.hcc_server_create(0, bvhs, cuts, slots=slots, method="hcc", key_bits=key_bits)
        _warm_server(srv, reqs, pools, ring, slots, count)
        return srv

    def summary(mrays, lat, st):
        return _serve_summary(mrays, lat, st, ring)

    out = {"metric": "serving: ray-query Mrays/s and p50/p99 latency under Poisson load, continuous admission "
                     "vs the unbatched per-request path", "unit": "Mrays/s",
           "config": {"workload": f"{len(ws)} rooms (seeds 30-37), {sum(w.tris.shape[0] for w in ws)} triangles; "
                                  f"{count} requests of {rr[0]}-{rr[1]} rays (log-uniform, mean "
                                  f"{int(reqs['n'].mean())}), host buffers (page-locked)",
                      "scenes": [{"tris": int(w.tris.shape[0]), "ray_pool": int(w.rays.n)} for w in ws],
                      "method": "hcc", "cut_size": args.cut_size, "key_bits": key_bits, "bvh_layout": args.layout,
                      "slots": args.slots},
           "generation_s": round(gen_s, 1)}
    with ClockSampler(0) as clk:
        # saturation: closed loop, 2 x slots requests outstanding
        sweep = {}
        sat = {}
        for slots in sorted({1, 2, 3, 4, 6, 8, 16, args.slots}):
            srv = server(slots)
            try:
                m, lat, st = _serve_run(srv, ring, pools, reqs, count, outstanding=max(2, 2 * slots))
            finally:
                hcc.hcc_server_destroy(srv)
            sweep[str(slots)] = summary(m, lat, st)
            sat[slots] = m
        out["saturation_by_slots"] = sweep
        mean_rays = float(reqs["n"][:count].mean())
        sat_req_s = sat[args.slots] * 1e6 / mean_rays
        out["saturation"] = {"continuous_mrays_s": round(sat[args.slots], 1), "unbatched_mrays_s": round(sat[1], 1),
                             "continuous_req_s": round(sat_req_s, 1)}
        loads = []
        for load in (0.25, 0.5, 0.9):
            row = {"load": load, "offered_req_s": round(load * sat_req_s, 1),
                   "offered_mrays_s": round(load * sat[args.slots], 1)}
            for name, slots in (("continuous", args.slots), ("unbatched", 1)):
                srv = server(slots)
                try:
                    m, lat, st = _serve_run(srv, ring, pools, reqs, count, rate=load * sat_req_s)
                finally:
                    hcc.hcc_server_destroy(srv)
                row[name] = summary(m, lat, st)
            loads.append(row)
        out["loads"] = loads
    out["clocks"] = clk.summary()
    # each result the same alone and in the mix (GPU vs GPU, full-size requests)
    srv = hcc.hcc_server_create(0, bvhs, cuts, slots=args.slots, method="hcc", key_bits=key_bits)
    k = min(12, count)
    mix = [torch.empty((int(reqs["n"][i]), 4), dtype=torch.int32).pin_memory() for i in range(k)]
    tickets = []
    for i in range(k):
        s, n, off = int(reqs["scene"][i]), int(reqs["n"][i]), int(reqs["offset"][i])
        tickets.append(hcc.hcc_server_submit(srv, s, pools[s][0][off:off + n], pools[s][1][off:off + n], mix[i]))
    for t in tickets:
        hcc.hcc_server_wait(srv, t)
    st = hcc.hcc_server_stats_get(srv)
    hcc.hcc_server_destroy(srv)
    same = True
    for i in range(k):
        s, n, off = int(reqs["scene"][i]), int(reqs["n"][i]), int(reqs["offset"][i])
        alone = torch.empty((n, 4), dtype=torch.int32).pin_memory()
        hcc.hcc_run_host(ctx, "hcc", bvhs[s], cuts[s], pools[s][0][off:off + n], pools[s][1][off:off + n],
                         key_bits, alone)
        same &= bool(torch.equal(alone, mix[i]))
    out["mix_equals_alone"] = {"requests": k, "max_in_flight": st["max_in_flight"], "identical": same}
    for c in cuts:
        hcc.hcc_cut_destroy(c)
    for b in bvhs:
        hcc.hcc_bvh_destroy(b)
    hcc.hcc_destroy(ctx)
    print(json.dumps(out), flush=True)


def profile_case(name: str):
    """Small, fixed workloads for ncu captures (not a benchmark: nothing is timed).

    trace-small: 480x270x8spp room, 200k triangles, exact nodes: HCC encode,
                 sort, trace through the sorted ids, the NoSort trace, then the
                 trace through the sorted ids of the rays as 32-byte records.
    sort-16m:    two sorts of 16,588,800 seeded uniform 32-bit keys.
    sort-hcc:    two sorts of the 16,588,800 HCC keys (cut 32, 32-bit keys) of
                 the 1920x1080x8spp room wavefront.
    gather:      the split gather of that wavefront through its HCC permutation,
                 from and to two float4 arrays, then from and to 32-byte records.
    trace-orders: the 1920x1080x8spp room (16,588,800 rays), exact nodes: the
                 closest-hit trace in NoSort, TwoPoint and HCC order (32-bit
                 keys, cut 32), one launch each, in that order, then in HCC
                 order on the rays as 32-byte records.
    """
    import torch
    from paper_2305_16652_gb300 import build, hcc
    build()
    ctx = hcc.hcc_create(0)
    if name == "sort-16m":
        n = 16_588_800
        k = np.random.default_rng(0).integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
        kt = torch.from_numpy(k.view(np.int32)).cuda()
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        for _ in range(2):
            hcc.hcc_sort(ctx, kt, 32, n, perm)
    elif name == "sort-hcc":
        w = make_workload(1, False)
        n = w.rays.n
        bvh = hcc.hcc_bvh_upload(ctx, w.bvh, layout="exact")
        cut = hcc.hcc_select_cut(ctx, bvh, 32, 0.125)
        org, dir_ = torch.from_numpy(w.rays.org).cuda(), torch.from_numpy(w.rays.dir).cuda()
        keys = torch.empty(n, dtype=torch.int32, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        hcc.hcc_reserve(ctx, n, 32)
        hcc.hcc_encode(ctx, "hcc", bvh, cut, org, dir_, 32, keys)
        for _ in range(2):
            hcc.hcc_sort(ctx, keys, 32, n, perm)
    elif name == "gather":
        w = make_workload(1, False)
        n = w.rays.n
        bvh = hcc.hcc_bvh_upload(ctx, w.bvh, layout="exact")
        cut = hcc.hcc_select_cut(ctx, bvh, 32, 0.125)
        org, dir_ = torch.from_numpy(w.rays.org).cuda(), torch.from_numpy(w.rays.dir).cuda()
        keys = torch.empty(n, dtype=torch.int32, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        hcc.hcc_reserve(ctx, n, 32)
        hcc.hcc_encode(ctx, "hcc", bvh, cut, org, dir_, 32, keys)
        hcc.hcc_sort(ctx, keys, 32, n, perm)
        so, sd = torch.empty_like(org), torch.empty_like(dir_)
        hcc.hcc_gather(ctx, org, dir_, perm, so, sd)
        del so, sd
        rec = torch.cat([org, dir_], 1)
        del org, dir_
        out = torch.empty_like(rec)
        hcc.hcc_gather(ctx, rec[:, :4], rec[:, 4:], perm, out[:, :4], out[:, 4:])
    elif name == "trace-small":
        w = make_workload(1, True)
        n = w.rays.n
        bvh = hcc.hcc_bvh_upload(ctx, w.bvh, layout="exact")
        cut = hcc.hcc_select_cut(ctx, bvh, 32, 0.125)
        org, dir_ = torch.from_numpy(w.rays.org).cuda(), torch.from_numpy(w.rays.dir).cuda()
        keys = torch.empty(n, dtype=torch.int32, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        hits = torch.empty((n, 4), dtype=torch.int32, device="cuda")
        hcc.hcc_encode(ctx, "hcc", bvh, cut, org, dir_, 32, keys)
        hcc.hcc_sort(ctx, keys, 32, n, perm)
        hcc.hcc_trace_sorted(ctx, bvh, org, dir_, perm, hits)
        hcc.hcc_trace(ctx, bvh, org, dir_, hits)
        rec = torch.cat([org, dir_], 1)  # the same rays as 32-byte records, traced in HCC order
        hcc.hcc_trace_sorted(ctx, bvh, rec[:, :4], rec[:, 4:], perm, hits)
    elif name == "trace-orders":
        w = make_workload(1, False)
        n = w.rays.n
        bvh = hcc.hcc_bvh_upload(ctx, w.bvh, layout="exact")
        cut = hcc.hcc_select_cut(ctx, bvh, 32, 0.125)
        org, dir_ = torch.from_numpy(w.rays.org).cuda(), torch.from_numpy(w.rays.dir).cuda()
        keys = torch.empty(n, dtype=torch.int32, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        hits = torch.empty((n, 4), dtype=torch.int32, device="cuda")
        hcc.hcc_reserve(ctx, n, 32)
        hcc.hcc_trace(ctx, bvh, org, dir_, hits)
        for method in ("twopoint", "hcc"):
            hcc.hcc_encode(ctx, method, bvh, cut if method == "hcc" else None, org, dir_, 32, keys)
            hcc.hcc_sort(ctx, keys, 32, n, perm)
            hcc.hcc_trace_sorted(ctx, bvh, org, dir_, perm, hits)
        rec = torch.cat([org, dir_], 1)  # HCC order again, the rays as 32-byte records
        hcc.hcc_trace_sorted(ctx, bvh, rec[:, :4], rec[:, 4:], perm, hits)
    else:
        raise SystemExit(f"unknown case {name}")
    hcc.hcc_sync(ctx)
    hcc.hcc_destroy(ctx)
    print(f"case {name} ok")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cut-size", type=int, default=32)
    ap.add_argument("--key-bits", type=int, default=32)
    ap.add_argument("--layout", choices=["exact", "quantised", "wide"], default="exact")
    ap.add_argument("--quick", action="store_true", help="480x270 image, 200k triangles (development only)")
    ap.add_argument("--cpu-sample", type=int, default=1_500_000)
    ap.add_argument("--ref-sample", type=int, default=300_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", choices=["trace-small", "sort-16m", "sort-hcc", "gather", "trace-orders"], help="run a profiling case and exit")
    ap.add_argument("--sweep", choices=["keylen", "batch", "serve", "methods", "hyper"],
                    help="run a study instead of the headline benchmark")
    ap.add_argument("--slots", type=int, default=4, help="serving: requests on the GPU at once")
    ap.add_argument("--viewport", choices=["full", "limited"], default="full",
                    help="method study: the 60-degree room view or a 10-degree view of the floor (Sec. 6.3)")
    ap.add_argument("--serve-requests", type=int, default=1000, help="serving: requests per run")
    ap.add_argument("--serve-requests-bench", type=int, default=300,
                    help="headline run: requests of its short serving leg (0 = skip)")
    args = ap.parse_args(argv)
    if args.case:
        return profile_case(args.case)
    if args.sweep == "keylen":
        return run_keylen_sweep(args)
    if args.sweep == "batch":
        return run_batch_sweep(args)
    if args.sweep == "serve":
        return run_serve_sweep(args)
    if args.sweep == "methods":
        return run_methods_sweep(args)
    if args.sweep == "hyper":
        return run_hyper_sweep(args)
    args.warmup = max(args.warmup, 3)
    rank, world, local_rank = dist_env()
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if args.impl != "reference":
            import torch
            torch.cuda.set_device(local_rank)
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            out = run_reference(args, rank, world)
        else:
            from paper_2305_16652_gb300 import build
            build()
            out, w, gpu = run_ours(args, rank, world, local_rank)
            if rank == 0 and not args.no_cpu_baseline:
                out["cpu_baseline"], out["parity_sample"] = cpu_baseline(w, args.key_bits, args.cut_size,
                                                                         args.cpu_sample, gpu)
        if rank == 0 and out is not None:
            print(json.dumps(out), flush=True)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
