"""Autotuner for the trace's knobs, by measurement.

Knobs searched (each changes only the speed of a trace, never its result):
  queue_depth     hand-off queue slots per sub-domain, also the most lineages
                  in flight at once (split traces only); 0 = automatic
  leaf_size       most triangles per BVH leaf (1..4): fewer node visits
                  against more triangle tests per leaf
  beams_per_warp  beam lineages a warp of the persistent trace reserves at a
                  time (0 = as many as its lanes need): fewer draws on the
                  launch's lineage counter against a coarser launch tail
  blocks_per_sm   resident 128-thread blocks per SM of the persistent trace
                  kernels, 0 = as many as fit
  chunk_beams     lineages per persistent launch (batches)

The search is coordinate descent from the library's defaults: one knob at a
time over its candidates, the others held at the best so far, repeated until
a pass changes nothing (at most `passes` passes).  Every candidate runs the
real workload (or a caller-chosen part of it) through the C ABI and is timed
on the device (bt_stats.trace_ms, the best of `repeats` runs after one
warm-up); the fastest wins.  `TuneCache` keeps the winners on disk per
(workload, GPU model), so that a workload is measured once per GPU model
(`tuned`).
"""
from __future__ import annotations

from . import btrace

TRACE_SPACE = {
    "queue_depth": (0, 1 << 16, 1 << 17),
    "leaf_size": (1, 2, 4),
    "beams_per_warp": (0, 64, 256),
    "blocks_per_sm": (0, 5),
}
DEFAULTS = {"queue_depth": 0, "leaf_size": 1, "beams_per_warp": 0, "blocks_per_sm": 0, "chunk_beams": 0}


def _chunk_candidates(max_order: int):
    # 0: the library's default, segment records in a quarter of the free
    # device memory (1..32 GiB) per launch
    per = max_order + 1
    return (0, (1 << 22) // per, (1 << 24) // per)


def coordinate_search(measure, space: dict, start: dict | None = None, passes: int = 2):
    """Minimise measure(knobs) -> ms over the product of `space`'s candidate
    lists by coordinate descent from `start` (default: each knob's first
    candidate).  Returns (best knobs, [(knobs, ms), ...] for every distinct
    setting measured, fastest first)."""
    best = {k: (start or {}).get(k, v[0]) for k, v in space.items()}
    seen = {}

    def run(knobs):
        key = tuple(sorted(knobs.items()))
        if key not in seen:
            seen[key] = float(measure(dict(knobs)))
        return seen[key]

    best_ms = run(best)
    for _ in range(passes):
        changed = False
        for name, cands in space.items():
            for v in cands:
                if v == best[name]:
                    continue
                trial = dict(best, **{name: v})
                ms = run(trial)
                if ms < best_ms:
                    best, best_ms, changed = trial, ms, True
        if not changed:
            break
    table = sorted(((dict(k), ms) for k, ms in seen.items()), key=lambda r: r[1])
    return best, table


def _with(params, knobs):
    q = btrace.bt_trace_params.from_buffer_copy(params)
    for k, v in knobs.items():
        setattr(q, k, int(v))
    return q


def tune_trace(tracer, scene_id, params, space=None, repeats=2, passes=2):
    """Tune one scene's trace: queue depth (split traces), leaf size, beams
    per warp and blocks per SM.  Returns (best knobs dict, trial table)."""
    space = dict(space or TRACE_SPACE)
    if params.tiles_x * params.tiles_y <= 1:
        space.pop("queue_depth", None)

    def measure(knobs):
        q = _with(params, knobs)
        btrace.bt_trace(tracer.ctx, scene_id, q)  # warm-up (and any leaf re-collapse)
        best = None
        for _ in range(repeats):
            btrace.bt_trace(tracer.ctx, scene_id, q)
            ms = btrace.bt_read_levels(tracer.ctx, scene_id)["trace_ms"]
            best = ms if best is None else min(best, ms)
        return best

    return coordinate_search(measure, space, DEFAULTS, passes)


def tune_batch(tracer, scene_ids, params, space=None, repeats=2, passes=2):
    """Tune a batch of loaded scenes with per-scene `params`: leaf size, beams
    per warp, blocks per SM and lineages per launch (a batch traces its scenes
    unsplit, so there is no queue).  Returns (best knobs dict, trial table)."""
    kmax = max(p.max_order for p in params)
    space = dict(space or {"leaf_size": TRACE_SPACE["leaf_size"],
                           "beams_per_warp": TRACE_SPACE["beams_per_warp"],
                           "blocks_per_sm": (0, 4, 5),
                           "chunk_beams": _chunk_candidates(kmax)})

    def measure(knobs):
        b = btrace.bt_batch_create(tracer.ctx, scene_ids, [_with(p, knobs) for p in params])
        try:
            btrace.bt_batch_run(tracer.ctx, b)  # captures the graph
            best = None
            for _ in range(repeats):
                btrace.bt_batch_run(tracer.ctx, b)
                ms = btrace.bt_batch_stats(b)["trace_ms"]
                best = ms if best is None else min(best, ms)
        finally:
            btrace.bt_batch_destroy(b)
        return best

    return coordinate_search(measure, space, DEFAULTS, passes)


def apply(params, knobs):
    """Set the tuned knobs on bt_trace_params `params` in place."""
    for k, v in knobs.items():
        setattr(params, k, int(v))
    return params


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
