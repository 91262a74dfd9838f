"""Benchmark: beam segments/s of the hybrid beam/ray tracer on one GB300.

Workload (default): the district configuration -- a synthetic 2 km x 2 km
city of 5,000 extruded buildings (201,381 triangles), 1,000 point sources at
0.5 m on lane centres, 20,480 beams per source (icosahedron level 5),
reflection orders 0..6, 250,000 microphones on a 4 m grid at 1.5 m.

One step = the whole hot path on one batch: scene ingest and BVH build,
microphone binning, beam generation, axis-ray traversal, reflection,
microphone test and energy scatter, level readout.

  value   device-resident inputs (torch CUDA tensors) -> segments/s
  e2e     the same calls with pinned host buffers, host->device copies and the
          device->host read of the levels inside the timed region

The district configuration splits the city plane into 4 x 4 sub-domains
linked by hand-off queues (the default --tiles); the line also carries the
same workload timed without the split (`untiled`).

`--impl reference` times the FP64 CPU oracle instead, on a bounded sample of
the same workload (a seeded subset of the sources per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "beam segments/s"
UNIT = "segments/s"


# The arithmetic type each precision variant computes in: "mixed" is float32
# traversal with a float-pair (double-float) image-source chain and float64
# energy accumulation.
DTYPE = {"fp32": "f32", "mixed": "mixed", "fp64": "f64", "mixed64": "mixed64"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="district", choices=["district", "tiny", "batch", "serve", "volume"],
                    help="batch: 64 cities of uneven size traced as one batch (CUDA graph); "
                         "volume: the district with 13.75 M microphones on a 4 m 3D grid; "
                         "serve: Poisson query streams against 8 resident cities")
    ap.add_argument("--rates", default="50,200,1000,2000", help="serve: arrival rates, queries/s")
    ap.add_argument("--queries", type=int, default=200, help="serve: queries per rate")
    ap.add_argument("--step-lineages", type=int, default=1 << 22, help="serve: lineages per server step")
    ap.add_argument("--oldest-share", type=float, default=1.0,
                    help="serve: share of a step's lineages that goes to the oldest query first")
    ap.add_argument("--small-lineages", type=int, default=0,
                    help="serve: queries with at most this many lineages left go first")
    ap.add_argument("--fill", default="work", choices=["work", "arrival"],
                    help="serve: what is left of a step after the oldest query goes to the others "
                         "shortest remaining work first (work) or in arrival order (arrival)")
    ap.add_argument("--mix-ratio", type=float, default=1.0,
                    help="serve: a step over several queries holds at most this many times the oldest "
                         "query's lineages, at least --mix-floor (0 = the whole step budget)")
    ap.add_argument("--mix-floor", type=int, default=1 << 18,
                    help="serve: with --mix-ratio, a shared step may always hold this many lineages")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the short served-latency measurement in the default line")
    ap.add_argument("--autotune", action="store_true",
                    help="batch: tune blocks per SM and lineages per launch on 16 of the cities first")
    ap.add_argument("--tune-cache", default=None,
                    help="batch --autotune: JSON file of tuned knobs per (cities, GPU model), reused when present")
    ap.add_argument("--sources", type=int, default=None, help="override the source count")
    ap.add_argument("--split-sources", action="store_true",
                    help="trace one district with its sources split over the ranks (one sum all-reduce of "
                         "the partial results per step); the default under torchrun with more than one GPU")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--tiles", default="4x4",
                    help="sub-domain grid; the district configuration splits the plane 4x4")
    ap.add_argument("--no-untiled", action="store_true",
                    help="skip the secondary timing of the same workload without sub-domains")
    ap.add_argument("--leaf-size", type=int, default=0, help="most triangles per BVH leaf (0 = library default)")
    ap.add_argument("--beams-per-warp", type=int, default=0,
                    help="lineages a warp reserves at a time (0 = library default)")
    ap.add_argument("--queue-depth", type=int, default=0, help="hand-off queue slots per sub-domain (0 = automatic)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32", "fp64", "mixed64"],
                    help="mixed: float-pair image-source chain (the parity-checked default)")
    return ap.parse_args()


def make_workload(name, rank=0, n_sources=None):
    from paper_1912_03998_gb300 import synth
    if name == "tiny":
        w = synth.tiny_city(seed=1 + rank)
    elif name == "volume":
        w = synth.district(seed=2, n_sources=1000)
        w = synth.Workload("district-volume", w.scene, w.src, w.power, synth.volume_mics(), w.level,
                           w.max_order, w.tiles, dict(w.info))
    else:
        w = synth.district(seed=2, n_sources=1000)
        if rank:  # independent traffic snapshot per rank, same city
            rng = np.random.Generator(np.random.PCG64(1000 + rank))
            w.src[:, :2] = w.src[rng.permutation(len(w.src)), :2]
    if n_sources is not None:
        w = w.subset_sources(np.arange(min(n_sources, len(w.src))))
    return w


def describe(w, tiles):
    return {"workload": f"{w.name}: {w.scene.info.get('n_buildings', 64)} buildings, "
                        f"{w.scene.n_tris} triangles, {len(w.src)} sources, L={w.level} "
                        f"({20 * 4 ** w.level} beams/source), K={w.max_order}, "
                        f"{len(w.mics)} microphones",
            "triangles": w.scene.n_tris, "sources": len(w.src), "icosa_level": w.level,
            "max_order": w.max_order, "microphones": len(w.mics), "bands": 8,
            "tiles": f"{tiles[0]}x{tiles[1]}"}


# ------------------------------------------------------------------ clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def kernel_hash():
    """Hash of the traversal kernels' source with comments and blank space
    removed, so that a comment edit does not orphan a committed capture."""
    import re
    h = hashlib.sha256()
    for f in ("trace.cu", "bt_internal.cuh"):
        src = open(os.path.join(ROOT, "paper_1912_03998_gb300", "csrc", f)).read()
        # the header's host launcher declarations do not change device code
        src = src.split("// ------------------------------------------------------------ host launchers")[0]
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def trace_kernel_name(tiles):
    return "k_trace" if tuple(tiles) == (1, 1) else "k_trace_tiled"


def ncu_counters(kernel, args, tiles):
    """DRAM and L2 bytes of one launch of `kernel` as a function of its units
    of work, from the committed ncu summary of two small cases of the same
    workload (the district's geometry with 16 and 64 of its sources, MIXED,
    split 4x4 or unsplit), only if it was taken on the current kernel source:
    {"dram": (a, b), "l2": (a, b), "unit": "segment" or "emitted segment"},
    bytes = a + b * units, or None.  The committed summaries set a = 0 and b =
    the bytes per unit of the larger case: traffic grows in proportion to the
    segments a launch traces (for the scatter, emits)."""
    if (args.workload != "district" or args.precision != "mixed"
            or tuple(tiles) not in ((4, 4), (1, 1))):
        return None
    split = "4x4" if tuple(tiles) == (4, 4) else "1x1"
    p = os.path.join(ROOT, "profiles", f"{kernel}_district_{split}_counters.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if kernel != "k_scatter" and d.get("kernel_hash") != kernel_hash():
        return None
    return {"dram": tuple(d["fit"]["dram"]), "l2": tuple(d["fit"]["lts"]), "unit": d["unit"],
            "file": os.path.relpath(p, ROOT)}


def l2_peak(ctx):
    """Measured L2 read bandwidth of this GPU, GB/s: the library's probe reads
    a 48 MB buffer (resident in the 126 MB L2) 200 times over in one kernel
    with L2-only loads; the best of a few grid sizes and 3 runs each."""
    from paper_1912_03998_gb300 import btrace
    return max(btrace.bt_l2_bandwidth(ctx, 48 << 20, 200, b) for b in (2, 4, 8) for _ in range(3))


def flush_l2(buf):
    buf.zero_()


# ------------------------------------------------------------------ our arm
def trial_table(table):
    """An autotuner's trials as rows of knob values and ms, fastest first."""
    names = sorted({k for knobs, _ in table for k in knobs})
    return {"knobs": names, "rows": [[knobs.get(n) for n in names] + [round(ms, 3)] for knobs, ms in table]}


def source_shard_result(trace_block, n_sources, rank, world, reduce):
    """One step of the sources split over the ranks (beams of different
    sources never interact, so the result for all sources is the sum of the
    ranks' partial results): this rank traces its contiguous block of the
    sources with trace_block(lo, hi) -> (intensity, path counts) as tensors on
    its device, and the partial results are summed over the ranks in place by
    reduce(intensity, counts) (one all-reduce; nothing to sum on one rank)."""
    from paper_1912_03998_gb300 import shard
    lo, hi = shard.source_block(n_sources, rank, world)
    I, cnt = trace_block(lo, hi)
    if world > 1:
        reduce(I, cnt)
    return I, cnt


def run_ours(args, rank, world):
    import torch
    from paper_1912_03998_gb300 import btrace, shard
    dev = torch.device("cuda", rank % max(1, torch.cuda.device_count()))
    torch.cuda.set_device(dev)
    split = args.split_sources
    # split: every rank holds the same district and traces a block of its
    # sources; replicas: every rank traces its own traffic snapshot
    w = make_workload(args.workload, 0 if split else rank, args.sources)
    tiles = tuple(int(v) for v in args.tiles.lower().split("x"))
    stream = torch.cuda.current_stream(dev)
    ctx = btrace.bt_create(dev.index, stream.cuda_stream)
    D = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    d_in = dict(verts=D(w.scene.verts), tris=D(w.scene.tris), mat=D(w.scene.mat),
                refl=D(w.scene.refl), src=D(w.src), power=D(w.power), mics=D(w.mics))
    n_m, nb = len(w.mics), w.scene.refl.shape[1]
    d_level = torch.empty((n_m, nb), dtype=torch.float64, device=dev)
    params = btrace.bt_params_default()
    params.max_order = w.max_order
    params.tiles_x, params.tiles_y = tiles
    params.precision = {"mixed": btrace.BT_PREC_MIXED, "fp32": btrace.BT_PREC_FP32,
                        "fp64": btrace.BT_PREC_FP64, "mixed64": btrace.BT_PREC_MIXED64}[args.precision]
    params.leaf_size, params.beams_per_warp, params.queue_depth = args.leaf_size, args.beams_per_warp, args.queue_depth
    tuned = None
    if args.autotune:
        # knobs picked by measurement on this workload (cached per GPU model)
        from paper_1912_03998_gb300 import autotune
        tr = btrace.Tracer(ctx=ctx)
        sid = tr.load(w)
        key, gpu = autotune.workload_key(w, params), torch.cuda.get_device_name(dev)
        cache = autotune.TuneCache(args.tune_cache) if args.tune_cache else None
        knobs, table = (cache.get(key, gpu) if cache else None), None
        if knobs is None:
            knobs, table = autotune.tune_trace(tr, sid, params)
            if cache:
                cache.put(key, gpu, knobs, table)
        btrace.bt_unload_scene(ctx, sid)
        autotune.apply(params, knobs)
        tuned = {"chosen": knobs, "cached": table is None, "tuned_on": "the whole workload"}
        if table is not None:
            tuned["trials_ms"] = trial_table(table)
    l2_flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    d_I = torch.empty((n_m, nb), dtype=torch.float64, device=dev)
    d_cnt = torch.empty(n_m, dtype=torch.int32, device=dev)

    def step(inp, level_out):
        sid = btrace.bt_load_scene(ctx, inp["verts"], inp["tris"], inp["mat"], inp["refl"])
        btrace.bt_set_microphones(ctx, sid, inp["mics"])
        if split:
            def trace_block(lo, hi):
                btrace.bt_set_sources(ctx, sid, inp["src"][lo:hi], inp["power"][lo:hi], w.level)
                btrace.bt_trace(ctx, sid, params)
                btrace.bt_read_levels(ctx, sid, None, d_I, d_cnt)
                return d_I, d_cnt
            I, cnt = source_shard_result(trace_block, len(w.src), rank, world, shard.allreduce_result)
            st = btrace.bt_read_levels(ctx, sid)  # this rank's trace
            btrace.bt_set_result(ctx, sid, I, cnt)
            btrace.bt_read_levels(ctx, sid, level_out, None, None)
        else:
            btrace.bt_set_sources(ctx, sid, inp["src"], inp["power"], w.level)
            btrace.bt_trace(ctx, sid, params)
            st = btrace.bt_read_levels(ctx, sid, level_out, None, None)
        btrace.bt_unload_scene(ctx, sid)
        return st

    def timed(inp, level_out, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        stats = []
        barrier(world)
        torch.cuda.synchronize(dev)
        n0 = btrace.bt_kernel_launches()
        for i in range(steps):
            flush_l2(l2_flush)
            ev[i][0].record(stream)
            stats.append(step(inp, level_out))
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        launches = btrace.bt_kernel_launches() - n0
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms, stats, launches

    for _ in range(args.warmup):
        step(d_in, d_level)
    with Clocks(dev.index) as clk:
        ms, stats, launches = timed(d_in, d_level, args.steps)
    untiled = None
    if tiles != (1, 1) and not args.no_untiled and world == 1:
        # the same workload without the sub-domain split, for comparison
        params.tiles_x, params.tiles_y = 1, 1
        for _ in range(args.warmup):
            step(d_in, d_level)
        u_ms, u_stats, _ = timed(d_in, d_level, args.steps)
        untiled = {"value": sum(s["segments"] for s in u_stats) / (sum(u_ms) * 1e-3),
                   "ms_per_step": sum(u_ms) / len(u_ms),
                   "kernel_ms_per_step": sum(s["trace_kernel_ms"] for s in u_stats) / len(u_stats),
                   "launches_per_step": sum(s["trace_launches"] for s in u_stats) / len(u_stats)}
        params.tiles_x, params.tiles_y = tiles
    segs = sum(s["segments"] for s in stats)
    contrib = sum(s["contributions"] for s in stats)
    total_ms = sum(ms)
    # roofline of the dominant kernel: its algorithmic bytes per launch over
    # its mean launch time; for the traversal, node + triangle bytes counted
    # in one extra, untimed trace
    tk = sum(s["trace_kernel_ms"] for s in stats)
    sk = sum(s["scatter_kernel_ms"] for s in stats)
    tl = sum(s["trace_launches"] for s in stats)
    params.count_work = 1
    cst = step(d_in, d_level)
    params.count_work = 0
    peak, peak_kind = measured_peaks()
    if sk > tk:
        # the scatter dominates (a volume of microphones): per launch, the
        # segment records read (192 B each), a 16 B microphone position per
        # candidate, and per contribution the 8 float64 accumulators and the
        # int32 count read and written (136 B)
        kernel = "k_scatter"
        sl = sum(s["scatter_launches"] for s in stats)
        last = stats[-1]
        alg_bytes = 192.0 * last["emitted"] + 16.0 * last["candidates"] + 136.0 * last["contributions"]
        bytes_per_launch = alg_bytes / max(1, last["scatter_launches"])
        achieved = bytes_per_launch / (sk / max(1, sl) * 1e-3) / 1e9
        counters = ncu_counters(kernel, args, tiles)
        units, kms = float(stats[-1]["emitted"]) / max(1, sl // args.steps), sk / max(1, sl)
        # its other roof: the L2's float64 atomic additions (8 per
        # contribution), against the library's probe of the same pattern
        adds = 8.0 * last["contributions"] / max(1, last["scatter_launches"])
        a_pk = max(btrace.bt_l2_atomics(ctx, 32 << 20, 64, b) for b in (2, 4, 8))
        atomics = {"achieved": adds / (kms * 1e-3), "peak": a_pk, "unit": "float64 atomic additions/s",
                   "frac": adds / (kms * 1e-3) / a_pk, "additions_per_launch": adds,
                   "peak_kind": "measured in this run: 8 float64 atomic additions to scattered 64-byte slots "
                                "of a 32 MB L2-resident buffer (bt_l2_atomics)"}
    else:
        kernel = trace_kernel_name(tiles)
        # a wide node visit reads four child boxes and four child codes (112 B),
        # a triangle test the triangle's three vertices (48 B)
        alg_bytes = 112.0 * cst["nodes_visited"] + 48.0 * cst["tris_tested"]
        bytes_per_launch = alg_bytes / max(1, cst["trace_launches"])
        achieved = bytes_per_launch / (tk / max(1, tl) * 1e-3) / 1e9
        counters = ncu_counters(kernel, args, tiles)
        units, kms = float(stats[-1]["segments"]) / max(1, tl // args.steps), tk / max(1, tl)
    traffic, l2 = None, None
    if kernel != "k_scatter":
        atomics = None
    if counters:
        traffic = counters["dram"][0] + counters["dram"][1] * units
        l2_bytes = counters["l2"][0] + counters["l2"][1] * units
        l2_pk = l2_peak(ctx)
        l2 = {"achieved": l2_bytes / (kms * 1e-3) / 1e9, "peak": l2_pk, "unit": "GB/s",
              "frac": l2_bytes / (kms * 1e-3) / 1e9 / l2_pk, "bytes_per_launch": l2_bytes,
              "peak_kind": "measured in this run: L2-only reads of a 48 MB resident buffer (bt_l2_bandwidth)",
              "counters": counters["file"] + f" (ncu lts__t_bytes of two small cases, linear in the {counters['unit']}s of a launch)"}
    res = dict(segs=segs, contrib=contrib, total_ms=total_ms, ms=ms, launches=launches,
               stats=stats[-1], tk=tk, sk=sk, tl=tl, alg_bytes=alg_bytes, kernel=kernel,
               bytes_per_launch=bytes_per_launch, achieved=achieved, peak=peak,
               peak_kind=peak_kind, traffic=traffic, clocks=clk.summary(), work=cst, w=w,
               tiles=tiles, untiled=untiled, autotune=tuned, l2=l2, atomics=atomics)
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        h_in = {k: pin(v.cpu().numpy()) for k, v in d_in.items()}
        h_level = torch.empty((n_m, nb), dtype=torch.float64).pin_memory()
        step(h_in, h_level)
        e_ms, e_stats, _ = timed(h_in, h_level, args.steps)
        h2d = sum(int(v.numel() * v.element_size()) for v in h_in.values())
        d2h = int(h_level.numel() * h_level.element_size())
        res["e2e"] = {"value": sum(s["segments"] for s in e_stats) / (sum(e_ms) * 1e-3),
                      "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                      "ms_per_step": sum(e_ms) / len(e_ms)}
    btrace.bt_destroy(ctx)
    return res


# ------------------------------------------------------------------ batches
def run_batch(args):
    """64 cities of uneven size: one batch run (persistent launches replayed
    from a CUDA graph) against the same cities traced one at a time."""
    import torch
    from paper_1912_03998_gb300 import autotune, btrace, synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ws = synth.batch_cities(seed=4, n=64)
    stream = torch.cuda.Stream(dev)
    tr = btrace.Tracer(0, stream.cuda_stream)
    prec = {"mixed": btrace.BT_PREC_MIXED, "fp32": btrace.BT_PREC_FP32, "fp64": btrace.BT_PREC_FP64, "mixed64": btrace.BT_PREC_MIXED64}[args.precision]
    sids = [tr.load(w) for w in ws]
    params = [tr.params(w.max_order, precision=prec) for w in ws]
    tuned = None
    if args.autotune:
        cache = autotune.TuneCache(args.tune_cache) if args.tune_cache else None
        key, gpu = autotune.batch_key(ws[:16], params[:16]), torch.cuda.get_device_name(dev)
        knobs, table = (cache.get(key, gpu) if cache else None), None
        if knobs is None:
            knobs, table = autotune.tune_batch(tr, sids[:16], params[:16])
            if cache:
                cache.put(key, gpu, knobs, table)
        for p in params:
            autotune.apply(p, knobs)
        tuned = {"chosen": knobs, "cached": table is None, "tuned_on": "the first 16 cities"}
        if table is not None:
            tuned["trials_ms"] = trial_table(table)
    l2_flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def span(fn):
        with torch.cuda.stream(stream):
            flush_l2(l2_flush)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b)

    b = btrace.bt_batch_create(tr.ctx, sids, params)
    for _ in range(args.warmup):
        btrace.bt_batch_run(tr.ctx, b)
    n0 = btrace.bt_kernel_launches()
    with Clocks(0) as clk:
        ms = [span(lambda: btrace.bt_batch_run(tr.ctx, b)) for _ in range(args.steps)]
    launches = btrace.bt_kernel_launches() - n0
    st = btrace.bt_batch_stats(b)
    segs = st["segments"]

    def one_at_a_time():
        for sid, p in zip(sids, params):
            btrace.bt_trace(tr.ctx, sid, p)

    one_at_a_time()
    ms1 = [span(one_at_a_time) for _ in range(max(1, min(args.steps, 2)))]
    btrace.bt_batch_destroy(b)
    tr.close()
    value = segs / (np.mean(ms) * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(ms)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": "batch: 64 cities of 100-5,000 buildings, 1-1,000 sources, L 3-6, "
                                   "K 2-8, 1k-250k microphones (seeded), traced as one batch",
                       "cities": len(ws), "triangles": int(sum(w.scene.n_tris for w in ws)),
                       "sources": int(sum(len(w.src) for w in ws)),
                       "lineages": int(sum(len(w.src) * 20 * 4 ** w.level for w in ws)),
                       "microphones": int(sum(len(w.mics) for w in ws)), "precision": args.precision,
                       "l2": "flushed before every step (256 MB write, outside the events)",
                       "parallelism": "1 GPU"},
            "clocks": clk.summary(), "gpu_launches": launches,
            "segments_per_step": segs,
            "one_at_a_time": {"value": segs / (np.mean(ms1) * 1e-3), "ms_per_step": float(np.mean(ms1))},
            "speedup_vs_one_at_a_time": float(np.mean(ms1) / np.mean(ms))}
    if tuned:
        line["autotune"] = tuned
    print(json.dumps(line))


# ------------------------------------------------------------------ serving
def serve_once(tr, cities, rate, n_queries, seed, prec, step_lineages, oldest_share=1.0, small_lineages=0,
               **server_kw):
    """One Poisson stream served by the loop and, on the same stream, one
    query at a time; latency summaries of both."""
    from paper_1912_03998_gb300 import btrace, serve, synth
    qs = synth.serving_queries(seed=seed, n_queries=n_queries, n_cities=len(cities), rate_qps=rate)
    srv = serve.Server(tr, cities, step_lineages=step_lineages, precision=prec, oldest_share=oldest_share,
                       small_lineages=small_lineages, **server_kw)
    try:
        srv.run(qs[:4], realtime=False)  # warm-up through both paths
        serve.run_plain(tr, srv.city_ids, qs[:4], precision=prec, realtime=False)
        n0 = btrace.bt_kernel_launches()
        t0 = time.perf_counter()
        done = srv.run(qs, realtime=True)
        wall = time.perf_counter() - t0
        launches = btrace.bt_kernel_launches() - n0
        t0 = time.perf_counter()
        plain = serve.run_plain(tr, srv.city_ids, qs, precision=prec, realtime=True)
        wall_p = time.perf_counter() - t0
    finally:
        srv.close()
    return {"rate_qps": rate, "served": serve.latency_summary(done, wall),
            "plain": serve.latency_summary(plain, wall_p), "steps": srv.steps,
            "segments_per_s": srv.segments / wall, "gpu_launches": launches,
            "server_time_s": {k: round(v, 4) for k, v in srv.host_s.items()}, "wall_s": round(wall, 4),
            "sources_mean": float(np.mean([len(q.src) for q in qs])),
            "microphones_mean": float(np.mean([len(q.mics) for q in qs]))}


def run_serve(args):
    """Poisson streams of traffic-noise queries against 8 resident cities,
    served by the continuous-batching loop and, on the same stream, one query
    at a time (plain whole-query traces)."""
    import torch
    from paper_1912_03998_gb300 import btrace, serve, synth
    torch.cuda.set_device(0)
    prec = {"mixed": btrace.BT_PREC_MIXED, "fp32": btrace.BT_PREC_FP32, "fp64": btrace.BT_PREC_FP64, "mixed64": btrace.BT_PREC_MIXED64}[args.precision]
    cities = synth.serving_cities(seed=5, n=8)
    tr = btrace.Tracer(0)
    rows = []
    with Clocks(0) as clk:
        for k, rate in enumerate(float(r) for r in args.rates.split(",")):
            rows.append(serve_once(tr, cities, rate, args.queries, 100 + k, prec, args.step_lineages,
                                   args.oldest_share, args.small_lineages, fill=args.fill,
                                   mix_ratio=args.mix_ratio, mix_floor=args.mix_floor))
    tr.close()
    head = rows[-1]
    line = {"metric": "served p50/p99 latency and queries/s", "value": head["served"]["queries_per_s"],
            "unit": "queries/s", "n_gpus": 1, "steps": len(rows), "warmup": 4,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": "serve: Poisson streams against 8 resident cities of 500-5,000 buildings; "
                                   "queries of 1-2,000 sources (0.001-1 W per band), 1k-250k microphones, "
                                   "L=4, K 3-6", "queries_per_rate": args.queries,
                       "step_lineages": args.step_lineages, "oldest_share": args.oldest_share,
                       "small_lineages": args.small_lineages, "fill": args.fill, "mix_ratio": args.mix_ratio, "mix_floor": args.mix_floor,
                       "precision": args.precision, "parallelism": "1 GPU"},
            "clocks": clk.summary(), "rates": rows}
    print(json.dumps(line))


# ------------------------------------------------------------------ oracle
def oracle_sample(w, seconds, threads, rng_seed=5):
    """Time the oracle on a seeded subset of sources sized to ~`seconds`."""
    from oracle import oracle as O
    sc = O.Scene(w.scene)
    rng = np.random.Generator(np.random.PCG64(rng_seed))
    order = rng.permutation(len(w.src))
    n = min(len(w.src), threads)
    t0 = time.perf_counter()
    O.trace(sc, w.src[order[:n]], w.power[order[:n]], w.level, w.mics, w.max_order,
            n_threads=threads)
    pilot = time.perf_counter() - t0
    n2 = int(min(len(w.src), max(n, n * seconds / max(pilot, 1e-3))))
    n2 = max(threads, (n2 // threads) * threads) if n2 >= threads else n2
    sel = order[:n2]
    t0 = time.perf_counter()
    r = O.trace(sc, w.src[sel], w.power[sel], w.level, w.mics, w.max_order, n_threads=threads)
    dt = time.perf_counter() - t0
    return dict(value=r["stats"]["segments"] / dt, seconds=dt, n_sources=n2, stats=r["stats"])


def run_reference(args, rank, world):
    w = make_workload(args.workload, 0, args.sources)
    threads = os.cpu_count() or 1
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    from oracle import oracle as O
    sc = O.Scene(w.scene)
    probe = oracle_sample(w, per_step, threads)
    n = probe["n_sources"]
    rng = np.random.Generator(np.random.PCG64(77))
    segs = 0.0
    total = 0.0
    for i in range(args.warmup + args.steps):
        sel = rng.choice(len(w.src), n, replace=False)
        t0 = time.perf_counter()
        r = O.trace(sc, w.src[sel], w.power[sel], w.level, w.mics, w.max_order, n_threads=threads)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            segs += r["stats"]["segments"]
            total += dt
    value = segs / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**describe(w, tuple(int(v) for v in args.tiles.lower().split("x"))),
                       "sample": f"{n} of {len(w.src)} sources per step (seeded), all microphones"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{n} of {len(w.src)} sources per step, {threads} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ main
def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, rank, world)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "batch":
        if rank == 0:
            run_batch(args)
        return
    if args.workload == "serve":
        if rank == 0:
            run_serve(args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", int(os.environ.get("LOCAL_RANK", rank))))
        # several GPUs trace one district with its sources split between them
        args.split_sources = args.workload == "district"
    res = run_ours(args, int(os.environ.get("LOCAL_RANK", rank)), world)
    # whole-job value: segments of all ranks over the slowest rank's time
    segs, total_ms = float(res["segs"]), float(res["total_ms"])
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([segs, total_ms], dtype=torch.float64, device="cuda")
        s = t.clone()
        dist.all_reduce(s[:1], op=dist.ReduceOp.SUM)
        dist.all_reduce(t[1:], op=dist.ReduceOp.MAX)
        segs, total_ms = float(s[0]), float(t[1])
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    w = res["w"]
    value = segs / (total_ms * 1e-3)
    cfg = describe(w, res["tiles"])
    cfg.update({"l2": "flushed before every step (256 MB write, outside the events)",
                "precision": ("MIXED: image-source chain in float pairs (double-float, about 48 "
                              "bits) on the FP32 pipe, FP32 watertight traversal with an FP64 "
                              "re-test of ambiguous hits, FP32 microphone tests with a float-pair "
                              "re-test near cone and end planes, FP64 energy accumulation")
                             if args.precision == "mixed" else
                             ("FP64 image-source chain, triangle tests, microphone tests and "
                              "contributions; FP32 BVH boxes and band powers; FP64 accumulation")
                             if args.precision == "fp64" else
                             ("MIXED64: FP32 watertight traversal with FP64 settling of ambiguous hits "
                              "and near ties, FP64 image-source chain, FP32 microphone tests with a "
                              "float-pair re-test, FP64 energy accumulation")
                             if args.precision == "mixed64" else
                             "FP32 chain, traversal and microphone tests, FP64 energy accumulation",
                "parallelism": (f"sources split over {world} GPU(s), one float64 sum all-reduce of the "
                                f"partial intensities and path counts per step" if args.split_sources else
                                f"replicas x{world}" if world > 1 else "1 GPU")})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "strong" if args.split_sources else "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision],
            "data": "synthetic", "config": cfg, "clocks": res["clocks"],
            "gpu_launches": res["launches"],
            "contributions_per_s": res["contrib"] * world / (total_ms * 1e-3),
            "roofline": {"kernel": res["kernel"], "bound": "hbm",
                         "achieved": res["achieved"],
                         "peak": res["peak"], "unit": "GB/s",
                         "frac": res["achieved"] / res["peak"], "traffic": res["traffic"],
                         "peak_kind": res["peak_kind"],
                         "algorithmic_bytes_per_launch": res["bytes_per_launch"],
                         "launches_per_step": res["tl"] / args.steps,
                         "kernel_ms_per_step": (res["sk"] if res["kernel"] == "k_scatter" else res["tk"]) / args.steps,
                         "trace_kernel_ms_per_step": res["tk"] / args.steps,
                         "scatter_kernel_ms_per_step": res["sk"] / args.steps,
                         "l2": res["l2"],
                         "atomics": res["atomics"],
                         "nodes_per_segment": res["work"]["nodes_visited"] / max(1, res["work"]["segments"]),
                         "tris_per_segment": res["work"]["tris_tested"] / max(1, res["work"]["segments"])},
            "stats": {k: res["stats"][k] for k in ("segments", "hits", "escapes", "emitted",
                                                   "candidates", "contributions", "handoffs",
                                                   "steals", "rounds")}}
    if "e2e" in res:
        line["e2e"] = res["e2e"]
    if res["untiled"]:
        line["untiled"] = res["untiled"]
    if res.get("autotune"):
        line["autotune"] = res["autotune"]
    if not args.no_serve and world == 1 and args.workload == "district":
        # the metric's second half: served p50/p99 latency on a short stream
        import torch
        from paper_1912_03998_gb300 import btrace, synth
        torch.cuda.set_device(0)
        prec = {"mixed": btrace.BT_PREC_MIXED, "fp32": btrace.BT_PREC_FP32,
                "fp64": btrace.BT_PREC_FP64, "mixed64": btrace.BT_PREC_MIXED64}[args.precision]
        tr = btrace.Tracer(0)
        try:
            # 300 queries, so that the 99th percentile rests on three of them
            line["serving"] = serve_once(tr, synth.serving_cities(seed=5, n=8), 200.0, 300, 100, prec,
                                         args.step_lineages, args.oldest_share, args.small_lineages,
                                         fill=args.fill, mix_ratio=args.mix_ratio, mix_floor=args.mix_floor)
        finally:
            tr.close()
    if not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        cb = oracle_sample(w, args.cpu_seconds, threads)
        line["cpu_baseline"] = {"value": cb["value"], "unit": UNIT, "cores": threads,
                                "kind": "oracle",
                                "sample": f"{cb['n_sources']} of {len(w.src)} sources (seeded), "
                                          f"all {len(w.mics)} microphones, {cb['seconds']:.1f} s"}
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
