"""Continuous-batching server for traffic-noise queries against resident
cities.

The cities' geometry and BVHs stay on the device; every query (a set of car
sources with band powers, a microphone set, a reflection order) gets a scene
that shares its city's geometry (bt_scene_share) for its own sources,
microphones and result.  The server runs in steps.  Before a step it admits
waiting queries in arrival order while a scene slot is free and their device
memory fits the budget; a step then traces the next lineages of the admitted
queries -- the step's lineage budget first to the oldest query, the rest to
the others shortest remaining work first -- in the same persistent launches
(bt_trace_ranges, accumulating), so queries that arrive while others are on
the GPU join at the next step and their work overlaps on the device.  A query
whose lineages are all traced is read back (levels to the host), its scene
freed, and its latency (completion - arrival) recorded.

Optionally (`admit_ahead`) admission is just in time: a query's set-up
(scene share, sources, microphone binning) waits while the admitted
queries already hold a given number of untraced lineages, so that a burst
of arrivals does not put every set-up ahead of the oldest query's trace.
Measured, it left the 99th percentile at 200 q/s where it was and gave up
the overload lead (less batching), so it is off by default.

A query is traced whole by one synchronous bt_trace, as plain serving
would, when it is the only query to trace and none is waiting, or when it
is the oldest and bigger than a step: there is nothing to overlap it with,
and one launch over all its lineages pays one launch tail and no per-step
host round trips (`whole`, on by default).  Steps over several queries
keep the continuous batching, each capped at `mix_ratio` times the
oldest query's own lineages (at least `mix_floor`): by default a step
holds the oldest query's lineages and, while those are fewer than
mix_floor (2^18), the others' up to that many, so that small queries share
launches (less per-query launch overhead) without a big one holding the
oldest back (measured on Poisson streams: at 200 q/s the 99th percentile
of uncapped steps was 1.4x plain serving's, capped it is within 4 %; under
overload the cap also raised throughput).  The others join a step only
whole (`partial_fill` off): a big query given part of a step would lose
its whole trace and go on in step-sized launches with their tails, and the
queries behind it would wait through all of them.

With `submit_alone`, a query that is the only one to trace and fits one
step is traced whole with the asynchronous call (bt_submit), behind a
submitted trace still running if there is one: while the GPU traces, the
loop goes on admitting arrivals and polls the submitted traces (bt_poll) to
retire them, so that read-back and admission overlap the traces; a step over
several queries waits until no submitted trace is running.  Measured on
Poisson streams at 200 q/s it raised the median latency by about 2 ms
against the synchronous steps (the poll loop notices completions later than
a blocking wait does), so it is off by default.  Admission also checks the
device's free memory, not only the budget.

`run_plain` serves the same stream one query at a time with whole-query
traces (bt_trace), the baseline the server is compared with.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import btrace

# device bytes of a query's own state: sources (xyz + 8 powers), microphones
# (sorted positions, cell ids, grid), accumulators (8 float64 + count) and the
# read-back buffers (levels, intensity, count)
BYTES_PER_SOURCE = 16 + 4 * 8
BYTES_PER_MIC = 16 + 8 + 8 * 8 + 4 + 8 * 8 * 2 + 4


def query_bytes(q) -> int:
    n = len(q.src) * BYTES_PER_SOURCE + len(q.mics) * BYTES_PER_MIC + (1 << 16)
    d = getattr(q, "directivity", None)
    if d is not None:
        # gains (float32 per pattern and beam) and each source's pattern index
        n += 4 * len(d.patterns) * 20 * 4 ** q.level + 4 * len(q.src)
    return n


def set_query_directivity(ctx, sid, q):
    """A query's directional sources, if it has any, sampled at the beams."""
    d = getattr(q, "directivity", None)
    if d is not None:
        btrace.bt_set_directivity(ctx, sid, d.gains(btrace.bt_beam_axes(ctx, q.level)), d.pattern_of)


def step_shares(left, work, budget: int, oldest_share: float = 1.0, quantum: int = 0, small: int = 0,
                fill: str = "work", partial: bool = True):
    """Lineages each active query traces in the next step.

    left[i]: the query's lineages still to trace; work[i]: its remaining
    work (lineages times segments per lineage); queries in admission order
    (index 0 the oldest).  Queries with at most `small` lineages left are
    served first, shortest remaining work first, so that they finish in this
    step.  Then the oldest query takes up to `oldest_share` of the step's
    lineage budget (all of it by default: first come, first served, so a big
    query is not held back by the stream behind it); what is left goes to
    the queries shortest remaining work first (`fill="work"`) or in
    admission order (`fill="arrival"`); with `partial` False a query other
    than the oldest joins only if all its remaining lineages fit, so that
    none is left part-traced (a part-traced query can no longer be traced
    whole).  With a nonzero `quantum`
    every query the budget did not reach still gets that many lineages (the
    step then exceeds the budget by up to len(left) quanta).
    """
    n = len(left)
    share = [0] * n
    if n == 0:
        return share
    b = int(budget)
    if small > 0:
        for i in sorted(range(n), key=lambda i: work[i]):
            if left[i] > small or left[i] > b:
                continue
            share[i] = left[i]
            b -= left[i]
    if oldest_share > 0.0 and share[0] < left[0] and b > 0:
        g = min(left[0] - share[0], int(budget * oldest_share), b)
        share[0] += g
        b -= g
    for i in (sorted(range(n), key=lambda i: work[i]) if fill == "work" else range(n)):
        if b <= 0:
            break
        if not partial and i > 0 and left[i] - share[i] > b:
            continue
        g = min(left[i] - share[i], b)
        share[i] += g
        b -= g
    if b <= 0 and quantum > 0:
        q = max(1, min(int(quantum), int(budget) // n))
        for i in range(n):
            if share[i] == 0 and left[i] > 0:
                share[i] = min(left[i], q)
    return share


@dataclass
class Done:
    index: int
    arrival_s: float
    admitted_s: float
    done_s: float
    level: np.ndarray = field(repr=False)
    count: np.ndarray = field(repr=False)

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


def device_free_bytes():
    """Free memory of the current CUDA device, or None without one."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.mem_get_info()[0])
    except Exception:
        pass
    return None


class Server:
    def __init__(self, tracer, cities, step_lineages: int = 1 << 22, quantum: int = 0,
                 mem_budget: int = 4 << 30, max_active: int = 48, precision: int = btrace.BT_PREC_MIXED,
                 oldest_share: float = 1.0, small_lineages: int = 0, mem_reserve: int = 1 << 30,
                 submit_alone: bool = False, check_free: bool = True, whole: bool = True,
                 fill: str = "work", mix_ratio: float = 1.0, mix_floor: int = 1 << 18,
                 admit_ahead: int = 0, partial_fill: bool = False):
        self.tr = tracer
        self.quantum = int(quantum)
        self.oldest_share = float(oldest_share)
        self.small_lineages = int(small_lineages)
        self.city_ids = [tracer.load_geometry(w) for w in cities]
        self.step_lineages = int(step_lineages)
        self.mem_budget = int(mem_budget)
        self.max_active = int(max_active)
        self.precision = precision
        self.mem_reserve = int(mem_reserve)
        self.submit_alone = bool(submit_alone)
        self.whole = bool(whole)
        if fill not in ("work", "arrival"):
            raise ValueError(f"fill must be 'work' or 'arrival', not {fill!r}")
        self.fill = fill
        self.mix_ratio = float(mix_ratio)
        self.partial_fill = bool(partial_fill)
        self.mix_floor = int(mix_floor)
        # optional admission just in time: set up (scene share, sources,
        # microphone binning) only while the admitted queries hold fewer
        # untraced lineages than this; -1: what one shared step takes, 0 (the
        # default): no limit
        self.admit_ahead = (self.mix_floor if self.mix_ratio > 0.0 else self.step_lineages) \
            if admit_ahead < 0 else int(admit_ahead)
        self.check_free = bool(check_free)
        self.waiting = collections.deque()
        self.active = []
        self.mem_used = 0
        self.done = []
        self.steps = 0
        self.segments = 0
        self.host_s = dict(admit=0.0, step=0.0, gpu_trace=0.0, retire=0.0)
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, index: int, q, arrival_s: float):
        self.waiting.append((index, q, arrival_s))

    def _admit(self):
        free = device_free_bytes() if self.waiting and self.check_free else None
        while self.waiting and len(self.active) < self.max_active:
            if (self.active and self.admit_ahead > 0 and
                    sum(a["total"] - a["next"] for a in self.active) >= self.admit_ahead):
                break  # enough queued work for the next step: the rest waits for its set-up
            index, q, arrival = self.waiting[0]
            need = query_bytes(q)
            if self.active and (self.mem_used + need > self.mem_budget or
                                (free is not None and need + self.mem_reserve > free)):
                break  # wait for memory; a lone query is always admitted
            if free is not None:
                free -= need
            self.waiting.popleft()
            ctx = self.tr.ctx
            sid = btrace.bt_scene_share(ctx, self.city_ids[q.city])
            btrace.bt_set_sources(ctx, sid, q.src, q.power, q.level)
            set_query_directivity(ctx, sid, q)
            btrace.bt_set_microphones(ctx, sid, q.mics)
            p = self.tr.params(q.max_order, precision=self.precision)
            total = len(q.src) * 20 * 4 ** q.level
            self.active.append(dict(index=index, q=q, sid=sid, p=p, next=0, total=total, mem=need,
                                    arrival=arrival, admitted=self.now(), inflight=False))
            self.mem_used += need

    def _poll(self) -> bool:
        """Poll the submitted whole-query trace, if any; True while it runs."""
        busy = False
        for a in self.active:
            if a["inflight"]:
                if btrace.bt_poll(self.tr.ctx, a["sid"]):
                    a["inflight"] = False
                else:
                    busy = True
        return busy

    def step(self) -> bool:
        """Admit, trace one step, retire finished queries.  False when idle."""
        t0 = time.perf_counter()
        self._admit()
        busy = self._poll()
        t1 = time.perf_counter()
        self.host_s["admit"] += t1 - t0
        if not self.active:
            return False
        pending = [a for a in self.active if a["next"] < a["total"]]
        if (self.submit_alone and len(pending) == 1 and not self.waiting
                and pending[0]["next"] == 0 and pending[0]["total"] <= self.step_lineages):
            # the only query to trace, and small: the whole query in one
            # asynchronous trace (behind a submitted one still running, if
            # any, on the same stream), so that the loop stays free to admit
            # arrivals and retire queries while the GPU traces
            a = pending[0]
            btrace.bt_submit(self.tr.ctx, a["sid"], a["p"])
            a["inflight"] = a["submitted"] = True
            a["next"] = a["total"]
            self.steps += 1
            self.host_s["step"] += time.perf_counter() - t1
            return True
        if busy:
            # a submitted trace is running: retire it before a (synchronous)
            # step of the others, so that its latency does not include theirs
            return True
        if self.whole and pending and self._trace_whole(pending):
            self.steps += 1
            t2 = time.perf_counter()
            self.host_s["step"] += t2 - t1
            self._retire(t2)
            return True
        left = [a["total"] - a["next"] for a in self.active]
        work = [l * (a["q"].max_order + 1) for l, a in zip(left, self.active)]
        budget = self.step_lineages
        if self.mix_ratio > 0.0:
            # the others may delay the oldest query's step by at most
            # mix_ratio - 1 times its own lineages (at least mix_floor in all)
            budget = min(budget, max(int(self.mix_ratio * left[0]), self.mix_floor))
        share = step_shares(left, work, budget, self.oldest_share, self.quantum, self.small_lineages,
                            self.fill, self.partial_fill)
        ids, begins, ends, params = [], [], [], []
        for a, s in zip(self.active, share):
            if s > 0 and not a["inflight"]:
                ids.append(a["sid"])
                begins.append(a["next"])
                ends.append(a["next"] + s)
                params.append(a["p"])
                a["next"] += s
        if ids:
            btrace.bt_trace_ranges(self.tr.ctx, ids, begins, ends, params, accumulate=True)
            st = btrace.bt_ranges_stats(self.tr.ctx)
            self.segments += st["segments"]
            self.host_s["gpu_trace"] += st["trace_ms"] * 1e-3
        self.steps += 1
        t2 = time.perf_counter()
        self.host_s["step"] += t2 - t1
        self._retire(t2)
        return True

    def _trace_whole(self, pending) -> bool:
        """Trace the oldest pending query whole (one bt_trace) if it is the
        only one to trace with nothing waiting, or bigger than a step; True
        if it did."""
        a = pending[0]
        if a["next"] != 0 or a["inflight"]:
            return False
        if not ((len(pending) == 1 and not self.waiting) or a["total"] > self.step_lineages):
            return False
        btrace.bt_trace(self.tr.ctx, a["sid"], a["p"])
        a["next"] = a["total"]
        a["whole"] = True
        return True

    def _retire(self, t2):
        """Read back every query whose lineages are all traced."""
        still = []
        for a in self.active:
            if a["next"] < a["total"] or a["inflight"]:
                still.append(a)
                continue
            q = a["q"]
            n, nb = len(q.mics), q.power.shape[1]
            level = np.empty((n, nb), np.float64)
            count = np.empty(n, np.int32)
            st = btrace.bt_read_levels(self.tr.ctx, a["sid"], level, None, count)
            if a.get("submitted") or a.get("whole"):
                self.segments += st["segments"]
                self.host_s["gpu_trace"] += st["trace_ms"] * 1e-3
            btrace.bt_unload_scene(self.tr.ctx, a["sid"])
            self.mem_used -= a["mem"]
            self.done.append(Done(a["index"], a["arrival"], a["admitted"], self.now(), level, count))
        self.active = still
        self.host_s["retire"] += time.perf_counter() - t2

    def run(self, queries, realtime: bool = True):
        """Serve `queries` (arrival_s from the start of the run).  With
        realtime, a query is submitted once its arrival time has passed;
        otherwise all are submitted at once.  Returns the Done records in
        query order."""
        self.t0 = time.perf_counter()
        self.done, self.steps, self.segments = [], 0, 0
        self.host_s = dict(admit=0.0, step=0.0, gpu_trace=0.0, retire=0.0)
        i = 0
        while i < len(queries) or self.waiting or self.active:
            now = self.now()
            while i < len(queries) and (not realtime or queries[i].arrival_s <= now):
                self.submit(i, queries[i], queries[i].arrival_s if realtime else 0.0)
                i += 1
            if not self.step() and i < len(queries):
                time.sleep(max(0.0, min(1e-3, queries[i].arrival_s - self.now())))
            elif any(a["inflight"] for a in self.active) and not self.waiting and (
                    i >= len(queries) or queries[i].arrival_s > self.now()):
                time.sleep(50e-6)  # the GPU is tracing a submitted query; nothing else to do yet
        return sorted(self.done, key=lambda d: d.index)

    def close(self):
        for cid in self.city_ids:
            btrace.bt_unload_scene(self.tr.ctx, cid)
        self.city_ids = []


def run_plain(tracer, city_ids, queries, precision: int = btrace.BT_PREC_MIXED, realtime: bool = True,
              gpu_s=None):
    """The same stream served one query at a time, each traced whole.  With
    `gpu_s` (a one-element list) the device time of the traces is added to
    gpu_s[0] in seconds."""
    ctx = tracer.ctx
    t0 = time.perf_counter()
    done = []
    for i, q in enumerate(queries):
        if realtime:
            wait = q.arrival_s - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        start = time.perf_counter() - t0
        sid = btrace.bt_scene_share(ctx, city_ids[q.city])
        btrace.bt_set_sources(ctx, sid, q.src, q.power, q.level)
        set_query_directivity(ctx, sid, q)
        btrace.bt_set_microphones(ctx, sid, q.mics)
        btrace.bt_trace(ctx, sid, tracer.params(q.max_order, precision=precision))
        n, nb = len(q.mics), q.power.shape[1]
        level = np.empty((n, nb), np.float64)
        count = np.empty(n, np.int32)
        st = btrace.bt_read_levels(ctx, sid, level, None, count)
        if gpu_s is not None:
            gpu_s[0] += st["trace_ms"] * 1e-3
        btrace.bt_unload_scene(ctx, sid)
        done.append(Done(i, q.arrival_s if realtime else 0.0, start, time.perf_counter() - t0, level, count))
    return done


def latency_summary(done, wall_s: float) -> dict:
    lat = np.array([d.latency_s for d in done])
    return {"queries": len(done), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "queries_per_s": len(done) / wall_s}
