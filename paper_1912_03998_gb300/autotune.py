"""Autotuner for the trace's launch knobs, by measurement.

Knobs searched:
  blocks_per_sm  resident 128-thread blocks per SM of the persistent trace
                 kernels (more warps hide more latency; fewer leave more
                 registers and L1 to each), 0 = as many as fit
  chunk_beams    lineages per persistent launch (fewer, larger launches have
                 fewer tails; smaller ones keep the segment buffer small)
  queue_depth    hand-off queue slots per sub-domain (split traces only)

The tracer itself fixes one lineage per lane (32 beams per warp) and one
triangle per BVH leaf (the LBVH's leaves), so those are not searched.  Every
candidate runs the real workload (or a caller-chosen part of it) through the
C ABI and is timed on the device (bt_stats.trace_ms); the fastest wins.
`TuneCache` keeps the winners on disk per (workload, GPU model), so that a
workload is measured once per GPU model (`tuned`).
"""
from __future__ import annotations

import itertools

from . import btrace


def _chunk_candidates(max_order: int):
    # 0: the library's default, segment records in a quarter of the free
    # device memory (1..32 GiB) per launch
    per = max_order + 1
    return [0, (1 << 22) // per, (1 << 24) // per]


def tune_batch(tracer, scene_ids, params, blocks=(0, 4, 5), chunks=None, repeats=2):
    """Tune blocks_per_sm and chunk_beams for a batch of loaded scenes with
    per-scene `params` (bt_trace_params).  Returns (best knobs dict, list of
    (knobs, ms) for every candidate)."""
    kmax = max(p.max_order for p in params)
    chunks = chunks if chunks is not None else _chunk_candidates(kmax)
    results = []
    for bps, chunk in itertools.product(blocks, chunks):
        ps = []
        for p in params:
            q = btrace.bt_trace_params.from_buffer_copy(p)
            q.blocks_per_sm = bps
            q.chunk_beams = chunk
            ps.append(q)
        b = btrace.bt_batch_create(tracer.ctx, scene_ids, ps)
        try:
            btrace.bt_batch_run(tracer.ctx, b)  # captures the graph
            best = None
            for _ in range(repeats):
                btrace.bt_batch_run(tracer.ctx, b)
                ms = btrace.bt_batch_stats(b)["trace_ms"]
                best = ms if best is None else min(best, ms)
        finally:
            btrace.bt_batch_destroy(b)
        results.append((dict(blocks_per_sm=bps, chunk_beams=chunk), best))
    results.sort(key=lambda r: r[1])
    return results[0][0], results


def tune_trace(tracer, scene_id, params, blocks=(0, 4, 5), depths=(0, 1 << 16, 1 << 18), repeats=2):
    """Tune blocks_per_sm and, for a split trace, queue_depth for one scene.
    Returns (best knobs dict, list of (knobs, ms))."""
    split = params.tiles_x * params.tiles_y > 1
    results = []
    for bps, depth in itertools.product(blocks, depths if split else (0,)):
        q = btrace.bt_trace_params.from_buffer_copy(params)
        q.blocks_per_sm = bps
        q.queue_depth = depth
        best = None
        for _ in range(repeats + 1):
            btrace.bt_trace(tracer.ctx, scene_id, q)
            ms = btrace.bt_read_levels(tracer.ctx, scene_id)["trace_ms"]
            best = ms if best is None else min(best, ms)
        results.append((dict(blocks_per_sm=bps, queue_depth=depth), best))
    results.sort(key=lambda r: r[1])
    return results[0][0], results


# ------------------------------------------------------------------ cache
def workload_key(w, params) -> str:
    """Key of a tuning result: the scene's geometry and materials, the
    source and microphone counts, the beam level and the trace parameters
    that shape the work (order, sub-domain grid, precision).  Two workloads
    with the same key run the same launches."""
    import hashlib

    import numpy as np
    h = hashlib.sha256()
    for a in (w.scene.verts, w.scene.tris, w.scene.mat, w.scene.refl):
        a = np.ascontiguousarray(a)
        h.update(str((a.dtype.str, a.shape)).encode())
        h.update(a.tobytes())
    h.update(str((len(w.src), len(w.mics), int(w.level), int(params.max_order), int(params.tiles_x),
                  int(params.tiles_y), int(params.precision))).encode())
    return h.hexdigest()[:32]


def batch_key(workloads, params) -> str:
    """Key of a batch's tuning result: its workloads' keys in order."""
    import hashlib
    h = hashlib.sha256()
    for w, p in zip(workloads, params):
        h.update(workload_key(w, p).encode())
    return h.hexdigest()[:32]


class TuneCache:
    """Tuned knobs kept in a JSON file, per (workload key, device name), so a
    workload is tuned once per GPU model.  A missing or unreadable file is an
    empty cache; writes replace the file atomically."""

    def __init__(self, path: str):
        import json
        import os
        self.path = path
        self.entries = {}
        if os.path.exists(path):
            try:
                with open(path) as f:
                    d = json.load(f)
                if isinstance(d, dict):
                    self.entries = d
            except (OSError, ValueError):
                self.entries = {}

    @staticmethod
    def _slot(key: str, device: str) -> str:
        return f"{device}|{key}"

    def get(self, key: str, device: str):
        e = self.entries.get(self._slot(key, device))
        return dict(e["knobs"]) if e else None

    def put(self, key: str, device: str, knobs: dict, table=None):
        import json
        import os
        self.entries[self._slot(key, device)] = {
            "knobs": dict(knobs),
            "table": [[dict(k), float(ms)] for k, ms in (table or [])],
        }
        tmp = f"{self.path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def tuned(cache: TuneCache, key: str, device: str, tune):
    """The cached knobs of (key, device), else run `tune()` (returning
    (knobs, table) like tune_batch and tune_trace), store and return its
    knobs."""
    knobs = cache.get(key, device)
    if knobs is None:
        knobs, table = tune()
        cache.put(key, device, knobs, table)
    return knobs
