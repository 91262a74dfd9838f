"""The continuous-batching server: every query's result is the same alone
(one whole-query trace) and in the mix (traced step by step together with the
other admitted queries); admission respects the memory budget."""
import numpy as np
import pytest

from paper_1912_03998_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tracer():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03998_gb300 import btrace
    t = btrace.Tracer(0)
    yield t
    t.close()


@pytest.fixture(scope="module")
def setting():
    cities = synth.serving_cities(seed=5, n=2)
    queries = synth.serving_queries(seed=9, n_queries=10, n_cities=2, rate_qps=1000.0,
                                    max_sources=24, max_mics=6000)
    return cities, queries


def same(a, b):
    assert (a.count == b.count).all()
    assert (np.isneginf(a.level) == np.isneginf(b.level)).all()
    fin = np.isfinite(b.level)
    assert np.abs(a.level[fin] - b.level[fin]).max(initial=0.0) < 1e-6


@pytest.mark.parametrize("step_lineages,whole,mix_ratio",
                         [(1 << 12, False, 0.0), (1 << 12, False, 2.0), (1 << 12, True, 0.0), (1 << 20, True, 0.0)])
def test_results_same_alone_and_in_the_mix(tracer, setting, step_lineages, whole, mix_ratio):
    # whole=False: every query goes through steps shared with the others;
    # whole=True (the default): lone or oversized queries are traced whole
    from paper_1912_03998_gb300 import serve
    cities, queries = setting
    srv = serve.Server(tracer, cities, step_lineages=step_lineages, whole=whole, mix_ratio=mix_ratio,
                       mix_floor=1 << 10)
    try:
        mixed = srv.run(queries, realtime=False)
        alone = serve.run_plain(tracer, srv.city_ids, queries, realtime=False)
    finally:
        srv.close()
    assert len(mixed) == len(alone) == len(queries)
    if step_lineages == 1 << 12 and not whole:
        assert srv.steps > len(queries)  # queries spanned several steps and overlapped
    for a, b in zip(mixed, alone):
        same(a, b)
    # a query far from its microphones may hear nothing; most hear something
    assert np.mean([a.count.max() > 0 for a in mixed]) >= 0.5


def test_admission_by_memory(tracer, setting):
    from paper_1912_03998_gb300 import serve
    cities, queries = setting
    srv = serve.Server(tracer, cities, step_lineages=1 << 14, mem_budget=1)
    seen = []
    orig = srv.step

    def step():
        r = orig()
        seen.append(len(srv.active))
        return r

    srv.step = step
    try:
        done = srv.run(queries[:4], realtime=False)
    finally:
        srv.close()
    assert len(done) == 4 and max(seen) <= 1  # one query at a time fits a 1-byte budget


def test_shared_geometry_scenes(tracer):
    # a scene sharing a resident city's geometry traces like a scene of its
    # own, split or not; the city cannot be unloaded while shared
    from paper_1912_03998_gb300 import btrace
    w = synth.tiny_city(seed=4, level=4, max_order=4, n_sources=2)
    own = tracer.run(w)
    btrace.bt_unload_scene(tracer.ctx, own["scene_id"])
    city = tracer.load_geometry(w)
    sid = btrace.bt_scene_share(tracer.ctx, city)
    try:
        btrace.bt_set_sources(tracer.ctx, sid, w.src, w.power, w.level)
        btrace.bt_set_microphones(tracer.ctx, sid, w.mics)
        for tiles in ((1, 1), (4, 4)):
            btrace.bt_trace(tracer.ctx, sid, tracer.params(w.max_order, tiles_x=tiles[0], tiles_y=tiles[1]))
            n = len(w.mics)
            I = np.empty((n, 8))
            c = np.empty(n, np.int32)
            btrace.bt_read_levels(tracer.ctx, sid, None, I, c)
            assert (c == own["cnt"]).all() and np.allclose(I, own["I"], rtol=1e-9, atol=0)
        with pytest.raises(btrace.BtError) as e:
            btrace.bt_unload_scene(tracer.ctx, city)
        assert e.value.code == btrace.BT_E_STATE
    finally:
        btrace.bt_unload_scene(tracer.ctx, sid)
        btrace.bt_unload_scene(tracer.ctx, city)


def test_directional_queries_same_alone_and_in_the_mix(tracer, setting):
    # queries whose sources are cardioids (every other source omnidirectional)
    # trace the same in the server's steps as alone, and the patterns reach
    # the levels (they differ from the all-omnidirectional queries)
    import dataclasses
    from paper_1912_03998_gb300 import serve
    cities, queries = setting
    qs = []
    for k, q in enumerate(queries[:6]):
        of = np.where(np.arange(len(q.src)) % 2 == 0, k % 2, -1).astype(np.int32)
        d = synth.Directivity([synth.cardioid((1.0, 0.0, 0.0)), synth.cardioid((0.0, 1.0, 0.3), 0.8)], of)
        qs.append(dataclasses.replace(q, directivity=d))
    srv = serve.Server(tracer, cities, step_lineages=1 << 12)
    try:
        mixed = srv.run(qs, realtime=False)
        alone = serve.run_plain(tracer, srv.city_ids, qs, realtime=False)
        omni = serve.run_plain(tracer, srv.city_ids, queries[:6], realtime=False)
    finally:
        srv.close()
    for a, b in zip(mixed, alone):
        same(a, b)
    differs = 0
    for a, o in zip(alone, omni):
        assert (a.count == o.count).all()  # gains scale energy, not which beams hit
        fin = np.isfinite(o.level)
        differs += int(np.abs(a.level[fin] - o.level[fin]).max(initial=0.0) > 1e-3)
    assert differs >= 1
