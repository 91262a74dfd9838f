"""Host-side logic that needs no GPU: the server's step allocation, the
volumetric microphone grid and the autotuner's cache."""
import numpy as np

from paper_1912_03998_gb300 import serve, synth


def test_step_shares_oldest_first_then_shortest_remaining():
    left = [5000, 300, 40, 2000]
    work = [5000 * 7, 300 * 4, 40 * 7, 2000 * 4]
    # the oldest query takes the whole budget when it can use it
    assert serve.step_shares(left, work, 4096) == [4096, 0, 0, 0]
    # what it leaves goes shortest remaining work first
    s = serve.step_shares([100] + left[1:], [700] + work[1:], 1000)
    assert s == [100, 300, 40, 560]
    # pure shortest remaining first
    s = serve.step_shares(left, work, 1000, oldest_share=0.0)
    assert s == [0, 300, 40, 660]
    # a share of the budget for the oldest query
    s = serve.step_shares(left, work, 1000, oldest_share=0.5)
    assert s == [500, 300, 40, 160]


def test_step_shares_fill_in_arrival_order():
    # after the oldest query, what is left of the budget goes to the others
    # in admission order instead of shortest remaining work first
    left = [300, 5000, 200, 100]
    work = [l * 5 for l in left]
    assert serve.step_shares(left, work, 1000) == [300, 400, 200, 100]
    assert serve.step_shares(left, work, 1000, fill="arrival") == [300, 700, 0, 0]
    assert serve.step_shares(left, work, 10000, fill="arrival") == left


def test_step_shares_without_partial_fill():
    # other queries join only whole: one that does not fit what is left of
    # the budget is skipped, a smaller one after it still joins
    left = [300, 5000, 600, 200]
    work = [l * 5 for l in left]
    assert serve.step_shares(left, work, 1000) == [300, 0, 500, 200]
    assert serve.step_shares(left, work, 1000, partial=False) == [300, 0, 0, 200]
    assert serve.step_shares(left, work, 1100, partial=False) == [300, 0, 600, 200]


def test_step_shares_invariants():
    rng = np.random.Generator(np.random.PCG64(3))
    for _ in range(500):
        n = int(rng.integers(1, 20))
        left = [int(x) for x in rng.integers(0, 10000, n)]
        work = [l * int(k) for l, k in zip(left, rng.integers(4, 8, n))]
        budget = int(rng.integers(1, 30000))
        frac = float(rng.choice([0.0, 0.25, 0.5, 1.0]))
        q = int(rng.choice([0, 64]))
        s = serve.step_shares(left, work, budget, frac, q)
        assert all(0 <= a <= l for a, l in zip(s, left))
        if q == 0:
            assert sum(s) <= budget
            # the budget is used up unless every query got all it has left
            assert sum(s) == min(budget, sum(left))
        else:
            assert sum(s) <= budget + n * q
        # without partial fill every query but the oldest gets all it has
        # left or nothing, within the budget
        fill = str(rng.choice(["work", "arrival"]))
        s = serve.step_shares(left, work, budget, frac, 0, 0, fill, partial=False)
        assert sum(s) <= budget and 0 <= s[0] <= left[0]
        assert all(a == 0 or a == l for a, l in zip(s[1:], left[1:]))


def test_volume_microphone_grid():
    m = synth.volume_mics(n_side=20, n_heights=5)
    assert m.shape == (20 * 20 * 5, 3) and m.dtype == np.float32
    zs = np.unique(m[:, 2])
    assert np.allclose(zs, 1.5 + 4.0 * np.arange(5))
    xs = np.unique(m[:, 0])
    assert len(xs) == 20 and np.allclose(np.diff(xs), synth.DIST_MIC_SIDE / 20)
    full = synth.volume_mics()
    assert full.shape == (13_750_000, 3) and float(full[:, 2].max()) == 217.5


def test_step_shares_small_queries_first():
    left = [5_000_000, 200_000, 40_000, 3_000_000]
    work = [l * 5 for l in left]
    # without the small-query rule the oldest takes the whole step
    assert serve.step_shares(left, work, 1 << 22) == [1 << 22, 0, 0, 0]
    # with it the two small queries finish in this step, the oldest takes the rest
    s = serve.step_shares(left, work, 1 << 22, small=1 << 18)
    assert s[1:3] == [200_000, 40_000] and s[0] == (1 << 22) - 240_000 and s[3] == 0
    assert sum(s) == 1 << 22


def test_tune_cache_per_workload_and_device(tmp_path):
    # a workload is tuned once per device model; the cache survives a reload,
    # a different scene or device misses, and an unreadable file is empty
    from paper_1912_03998_gb300 import autotune, btrace, synth
    w1 = synth.tiny_city(seed=1, level=3, max_order=3)
    w2 = synth.tiny_city(seed=2, level=3, max_order=3)
    p = btrace.bt_trace_params()
    p.max_order, p.tiles_x, p.tiles_y, p.precision = 3, 1, 1, btrace.BT_PREC_MIXED
    k1, k2 = autotune.workload_key(w1, p), autotune.workload_key(w2, p)
    assert k1 != k2 and k1 == autotune.workload_key(synth.tiny_city(seed=1, level=3, max_order=3), p)
    q = btrace.bt_trace_params.from_buffer_copy(p)
    q.tiles_x = q.tiles_y = 4
    assert autotune.workload_key(w1, q) != k1
    assert autotune.batch_key([w1, w2], [p, p]) != autotune.batch_key([w2, w1], [p, p])
    calls = []

    def tune():
        calls.append(1)
        return {"blocks_per_sm": 4, "chunk_beams": 0}, [({"blocks_per_sm": 4, "chunk_beams": 0}, 1.5)]

    path = str(tmp_path / "tune.json")
    c = autotune.TuneCache(path)
    assert autotune.tuned(c, k1, "GB300", tune) == {"blocks_per_sm": 4, "chunk_beams": 0}
    assert autotune.tuned(c, k1, "GB300", tune) == {"blocks_per_sm": 4, "chunk_beams": 0}
    assert len(calls) == 1
    c2 = autotune.TuneCache(path)
    assert c2.get(k1, "GB300") == {"blocks_per_sm": 4, "chunk_beams": 0}
    assert c2.get(k2, "GB300") is None and c2.get(k1, "B200") is None
    autotune.tuned(c2, k1, "B200", tune)
    assert len(calls) == 2
    with open(path, "w") as f:
        f.write("{not json")
    assert autotune.TuneCache(path).get(k1, "GB300") is None


def test_generators_are_deterministic_per_seed():
    # every synthetic input is a function of its seed alone
    def arrays(w):
        return [w.scene.verts, w.scene.tris, w.scene.mat, w.scene.refl, w.src, w.power, w.mics]

    for make in (lambda s: synth.tiny_city(seed=s, n_sources=3),
                 lambda s: synth.district(seed=s, n_buildings=200, n_sources=20, n_mic_side=40)):
        a, b, c = make(7), make(7), make(8)
        assert all(np.array_equal(x, y) for x, y in zip(arrays(a), arrays(b)))
        assert not all(np.array_equal(x, y) if x.shape == y.shape else False
                       for x, y in zip(arrays(a), arrays(c)))
    q1 = synth.serving_queries(seed=3, n_queries=5, n_cities=2, rate_qps=100.0, max_sources=20, max_mics=2000)
    q2 = synth.serving_queries(seed=3, n_queries=5, n_cities=2, rate_qps=100.0, max_sources=20, max_mics=2000)
    assert all(x.arrival_s == y.arrival_s and np.array_equal(x.src, y.src) and np.array_equal(x.mics, y.mics)
               for x, y in zip(q1, q2))


def test_query_bytes_count_directivity():
    q = synth.serving_queries(seed=1, n_queries=1, n_cities=1, rate_qps=10.0, max_sources=10, max_mics=2000)[0]
    base = serve.query_bytes(q)
    import dataclasses
    d = synth.Directivity([synth.cardioid((1, 0, 0))], np.zeros(len(q.src), np.int32))
    assert serve.query_bytes(dataclasses.replace(q, directivity=d)) == base + 4 * 20 * 4 ** q.level + 4 * len(q.src)


class _FakeLib:
    """Stands in for the library calls the server makes: records every
    lineage range it is asked to trace (no GPU)."""

    def __init__(self):
        self.next_sid = 100
        self.live = set()
        self.ranges = {}      # sid -> list of (begin, end)
        self.calls = []       # per bt_trace_ranges call: list of sids
        self.totals = []      # per bt_trace_ranges call: lineages traced
        self.directivity = {}
        self.submitted, self.polls, self.total = [], {}, {}
        self.whole = []       # per bt_trace call (a whole query): its sid

    def bt_scene_share(self, ctx, base):
        self.next_sid += 1
        self.live.add(self.next_sid)
        self.ranges[self.next_sid] = []
        return self.next_sid

    def bt_set_sources(self, ctx, sid, src, power, level):
        assert sid in self.live
        self.total[sid] = len(src) * 20 * 4 ** level

    def bt_set_microphones(self, ctx, sid, mics):
        assert sid in self.live

    def bt_beam_axes(self, ctx, level):
        return np.zeros((20 * 4 ** level, 3), np.float32)

    def bt_set_directivity(self, ctx, sid, gains, of):
        self.directivity[sid] = (gains.shape, len(of))

    def bt_trace_ranges(self, ctx, ids, begins, ends, params, accumulate=False):
        assert accumulate
        self.calls.append(list(ids))
        self.totals.append(sum(e - b for b, e in zip(begins, ends)))
        for sid, b, e in zip(ids, begins, ends):
            assert sid in self.live and 0 <= b < e
            self.ranges[sid].append((b, e))

    def bt_ranges_stats(self, ctx):
        return {"segments": 0, "trace_ms": 0.0}

    def bt_trace(self, ctx, sid, params):
        # a whole-query trace, synchronous
        assert sid in self.live and not self.ranges[sid]
        self.whole.append(sid)
        self.ranges[sid].append((0, self.total[sid]))

    def bt_submit(self, ctx, sid, params):
        # a whole-query trace: every lineage of the scene in one range
        assert sid in self.live and not self.ranges[sid]
        self.submitted.append(sid)
        self.ranges[sid].append((0, self.total[sid]))
        self.polls[sid] = 2  # finishes on the second poll

    def bt_poll(self, ctx, sid):
        self.polls[sid] -= 1
        return self.polls[sid] <= 0

    def bt_read_levels(self, ctx, sid, level=None, intensity=None, count=None):
        if level is not None:
            level[:] = sid
        if count is not None:
            count[:] = 1
        return {"segments": 0, "trace_ms": 0.0}

    def bt_unload_scene(self, ctx, sid):
        self.live.discard(sid)


class _FakeTracer:
    ctx = None

    def load_geometry(self, w):
        return 0

    def params(self, max_order, **kw):
        return ("params", max_order)


def test_server_traces_every_lineage_once_in_order(monkeypatch):
    # each query's lineages are traced exactly once, as consecutive ranges,
    # its scene is freed after its last range, results come back in query
    # order, and no step holds more than max_active queries
    lib = _FakeLib()
    for name in ("bt_scene_share", "bt_set_sources", "bt_set_microphones", "bt_beam_axes", "bt_set_directivity",
                 "bt_trace_ranges", "bt_ranges_stats", "bt_read_levels", "bt_unload_scene", "bt_submit", "bt_poll",
                 "bt_trace"):
        monkeypatch.setattr(serve.btrace, name, getattr(lib, name))
    qs = synth.serving_queries(seed=2, n_queries=12, n_cities=2, rate_qps=1e4, level=3, max_sources=40,
                               max_mics=3000)
    srv = serve.Server(_FakeTracer(), [None, None], step_lineages=1500, max_active=4, whole=False)
    done = srv.run(qs, realtime=False)
    assert [d.index for d in done] == list(range(len(qs)))
    assert not lib.live  # every query's scene was freed
    assert max(len(c) for c in lib.calls) <= 4
    assert max(lib.totals) <= 1500 and srv.steps == len(lib.calls) + len(lib.submitted)
    assert not lib.whole
    for d, q in zip(done, qs):
        sid = int(d.level[0, 0])
        rs = lib.ranges[sid]
        assert rs[0][0] == 0 and rs[-1][1] == len(q.src) * 20 * 4 ** q.level
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))  # consecutive, no gap or overlap


def test_coordinate_search_finds_the_separable_minimum_with_few_trials():
    """The autotuner's search on a made-up cost with a known best setting: it
    must reach it, report every measured setting once, fastest first, and
    measure far fewer settings than the whole product."""
    from paper_1912_03998_gb300 import autotune
    space = {"queue_depth": (0, 1 << 16, 1 << 17), "leaf_size": (1, 2, 4), "beams_per_warp": (0, 64, 256),
             "blocks_per_sm": (0, 5)}
    best = {"queue_depth": 1 << 16, "leaf_size": 2, "beams_per_warp": 0, "blocks_per_sm": 5}
    calls = []

    def cost(k):
        calls.append(dict(k))
        return 10.0 + sum((space[n].index(k[n]) - space[n].index(best[n])) ** 2 for n in space)

    knobs, table = autotune.coordinate_search(cost, space, autotune.DEFAULTS)
    assert knobs == best
    assert table[0][0] == best and table[0][1] == 10.0
    assert [ms for _, ms in table] == sorted(ms for _, ms in table)
    assert len(table) == len(calls) == len({tuple(sorted(c.items())) for c in calls})
    assert len(calls) < 3 * 3 * 3 * 2


def test_coordinate_search_keeps_defaults_when_nothing_is_faster():
    from paper_1912_03998_gb300 import autotune
    space = {"leaf_size": (1, 2, 4), "beams_per_warp": (0, 64, 256)}
    knobs, table = autotune.coordinate_search(lambda k: 5.0 + k["leaf_size"] + k["beams_per_warp"] / 64,
                                              space, autotune.DEFAULTS)
    assert knobs == {"leaf_size": 1, "beams_per_warp": 0}
    assert len(table) == 5  # the defaults and the four single-knob changes, one pass


def test_server_submits_a_lone_small_query_whole_and_polls_it(monkeypatch):
    # a query arriving to an idle server that fits one step is traced whole
    # by one asynchronous submission, polled until it finishes, then read back
    lib = _FakeLib()
    for name in ("bt_scene_share", "bt_set_sources", "bt_set_microphones", "bt_beam_axes", "bt_set_directivity",
                 "bt_trace_ranges", "bt_ranges_stats", "bt_read_levels", "bt_unload_scene", "bt_submit", "bt_poll",
                 "bt_trace"):
        monkeypatch.setattr(serve.btrace, name, getattr(lib, name))
    qs = synth.serving_queries(seed=3, n_queries=3, n_cities=1, rate_qps=1.0, level=2, max_sources=3,
                               max_mics=1000)
    srv = serve.Server(_FakeTracer(), [None], step_lineages=1 << 20, submit_alone=True)
    for i, q in enumerate(qs):  # one at a time: the server is idle at every arrival
        srv.submit(i, q, 0.0)
        while srv.waiting or srv.active:
            srv.step()
    assert len(lib.submitted) == 3 and not lib.calls and not lib.live
    assert [d.index for d in srv.done] == [0, 1, 2]
    for d, q in zip(srv.done, qs):
        assert lib.ranges[int(d.level[0, 0])] == [(0, len(q.src) * 20 * 4 ** q.level)]


def test_server_traces_lone_and_oversized_queries_whole(monkeypatch):
    # With the whole-query policy (the default) a query that is the only one
    # to trace with none waiting, or the oldest and bigger than a step, is
    # traced by one bt_trace over all its lineages; queries that overlap
    # otherwise share steps; every lineage is still traced exactly once.
    lib = _FakeLib()
    for name in ("bt_scene_share", "bt_set_sources", "bt_set_microphones", "bt_beam_axes", "bt_set_directivity",
                 "bt_trace_ranges", "bt_ranges_stats", "bt_read_levels", "bt_unload_scene", "bt_submit", "bt_poll",
                 "bt_trace"):
        monkeypatch.setattr(serve.btrace, name, getattr(lib, name))
    qs = synth.serving_queries(seed=2, n_queries=12, n_cities=2, rate_qps=1e4, level=3, max_sources=40,
                               max_mics=3000)
    step = 1500
    srv = serve.Server(_FakeTracer(), [None, None], step_lineages=step, max_active=4)
    done = srv.run(qs, realtime=False)
    assert [d.index for d in done] == list(range(len(qs)))
    assert not lib.live
    assert srv.steps == len(lib.calls) + len(lib.whole)
    totals = {d.index: len(q.src) * 20 * 4 ** q.level for d, q in zip(done, qs)}
    for d, q in zip(done, qs):
        sid = int(d.level[0, 0])
        rs = lib.ranges[sid]
        assert rs[0][0] == 0 and rs[-1][1] == totals[d.index]
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        if sid in lib.whole:
            assert rs == [(0, totals[d.index])]
    # the first query (the oldest, bigger than a step) is traced whole; a big
    # query that already took part in a shared step goes on in steps; the
    # shared steps keep to the budget
    assert totals[0] > step and int(done[0].level[0, 0]) in lib.whole
    assert lib.calls and max(lib.totals) <= step
    # a lone query to an idle server: one whole trace
    lib2 = _FakeLib()
    for name in ("bt_scene_share", "bt_set_sources", "bt_set_microphones", "bt_trace", "bt_read_levels",
                 "bt_unload_scene", "bt_trace_ranges"):
        monkeypatch.setattr(serve.btrace, name, getattr(lib2, name))
    srv2 = serve.Server(_FakeTracer(), [None], step_lineages=1 << 20)
    srv2.submit(0, qs[0], 0.0)
    while srv2.waiting or srv2.active:
        srv2.step()
    assert len(lib2.whole) == 1 and not lib2.calls


def test_district_matches_its_configuration():
    # the district configuration: 5,000 buildings of 4-12-gon footprints with
    # areas lognormal around a 400 m^2 median and heights lognormal around
    # 20 m with a tail to 200 m, about 200k triangles, 1,000 sources with
    # 0.01-1 W per band, 250k microphones on a 4 m grid at 1.5 m
    w = synth.district(seed=2)
    info = w.info
    assert info["n_buildings"] == 5000
    q10, q50, q90 = info["area_quantiles"]
    assert 360.0 <= q50 <= 440.0 and q10 < 0.6 * q50 and q90 > 1.5 * q50
    assert 18.0 <= info["height_quantiles"][1] <= 22.0 and info["height_max"] <= 200.0
    assert 4.0 < info["ngon_mean"] < 12.0
    assert 190_000 <= w.scene.n_tris <= 210_000
    assert len(w.src) == 1000 and np.all((w.power >= 0.01 - 1e-6) & (w.power <= 1.0 + 1e-6))
    assert len(w.mics) == 250_000 and np.all(w.mics[:, 2] == np.float32(1.5))
    d = np.diff(np.unique(w.mics[:, 0]))
    assert np.allclose(d, 4.0, atol=1e-3)


def test_server_admits_just_in_time(monkeypatch):
    # with admit_ahead, a waiting query is set up only while the admitted
    # queries hold fewer untraced lineages than that: with 1, one query at a
    # time; every query is still traced exactly once and answered in order
    lib = _FakeLib()
    for name in ("bt_scene_share", "bt_set_sources", "bt_set_microphones", "bt_beam_axes", "bt_set_directivity",
                 "bt_trace_ranges", "bt_ranges_stats", "bt_read_levels", "bt_unload_scene", "bt_submit", "bt_poll",
                 "bt_trace"):
        monkeypatch.setattr(serve.btrace, name, getattr(lib, name))
    qs = synth.serving_queries(seed=2, n_queries=8, n_cities=2, rate_qps=1e4, level=3, max_sources=40,
                               max_mics=3000)
    srv = serve.Server(_FakeTracer(), [None, None], step_lineages=1500, admit_ahead=1)
    seen = []
    orig = srv._admit

    def admit():
        orig()
        seen.append(len(srv.active))

    srv._admit = admit
    done = srv.run(qs, realtime=False)
    assert [d.index for d in done] == list(range(len(qs)))
    assert not lib.live and max(seen) == 1
    # -1 holds back once a shared step's worth of lineages is admitted; the
    # default (0) admits every waiting query that fits
    assert serve.Server(_FakeTracer(), [None], step_lineages=1 << 22, admit_ahead=-1).admit_ahead == 1 << 18
    assert serve.Server(_FakeTracer(), [None], step_lineages=1 << 22, mix_ratio=0.0,
                        admit_ahead=-1).admit_ahead == 1 << 22
    assert serve.Server(_FakeTracer(), [None]).admit_ahead == 0
