"""Batches: several scenes of uneven size traced together in one persistent
launch per group of lineages, replayed from a CUDA graph.  Every scene's
result must equal its own single-scene trace (the oracle for one of them)."""
import numpy as np
import pytest

from paper_1912_03998_gb300 import synth
from tests.parity import assert_parity, level_db

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


def uneven_workloads():
    ws = [synth.tiny_city(seed=11, level=3, max_order=2, n_grid=16),
          synth.tiny_city(seed=12, level=4, max_order=5, n_sources=3, n_grid=40),
          synth.boxes(3, seed=5, level=5, max_order=4, n_grid=24),
          synth.ground_only(seed=2, level=4),
          synth.tiny_city(seed=13, level=2, max_order=8, n_sources=2, n_grid=9)]
    return ws


def read(tracer, sid, w):
    from paper_1912_03998_gb300 import btrace
    n, nb = len(w.mics), w.scene.refl.shape[1]
    L = np.empty((n, nb), np.float64)
    I = np.empty((n, nb), np.float64)
    c = np.empty(n, np.int32)
    btrace.bt_read_levels(tracer.ctx, sid, L, I, c)
    return dict(level=L, I=I, cnt=c)


@pytest.mark.parametrize("precision", ["mixed", "fp32", "fp64"])
def test_batch_equals_single_scene_traces(tracer, oracle_mod, precision):
    from paper_1912_03998_gb300 import btrace
    prec = {"mixed": btrace.BT_PREC_MIXED, "fp32": btrace.BT_PREC_FP32, "fp64": btrace.BT_PREC_FP64}[precision]
    ws = uneven_workloads()
    singles = []
    for w in ws:
        r = tracer.run(w, precision=prec)
        singles.append(r)
        btrace.bt_unload_scene(tracer.ctx, r["scene_id"])
    sids = [tracer.load(w) for w in ws]
    params = [tracer.params(w.max_order, precision=prec) for w in ws]
    b = btrace.bt_batch_create(tracer.ctx, sids, params)
    try:
        btrace.bt_batch_run(tracer.ctx, b)
        first = [read(tracer, sid, w) for sid, w in zip(sids, ws)]
        st = btrace.bt_batch_stats(b)
        assert st["segments"] == sum(r["stats"]["segments"] for r in singles)
        for g, r in zip(first, singles):
            assert (g["cnt"] == r["cnt"]).all()
            assert np.allclose(g["I"], r["I"], rtol=1e-9, atol=0)
        # the graph replays: same results again
        btrace.bt_batch_run(tracer.ctx, b)
        for sid, w, g in zip(sids, ws, first):
            g2 = read(tracer, sid, w)
            assert (g2["cnt"] == g["cnt"]).all()
            assert np.allclose(g2["I"], g["I"], rtol=1e-12, atol=0)
        if precision == "mixed":
            # one scene against the oracle as well
            r = oracle_mod.trace_workload(ws[1])
            assert_parity(first[1]["level"], level_db(r["I"]), "batched tiny city")
        # a scene that changes invalidates the batch
        btrace.bt_set_sources(tracer.ctx, sids[2], ws[2].src, ws[2].power, ws[2].level)
        with pytest.raises(btrace.BtError) as e:
            btrace.bt_batch_run(tracer.ctx, b)
        assert e.value.code == btrace.BT_E_STATE
    finally:
        btrace.bt_batch_destroy(b)
        for sid in sids:
            btrace.bt_unload_scene(tracer.ctx, sid)


def test_batch_rejects_bad_requests(tracer):
    from paper_1912_03998_gb300 import btrace
    ws = uneven_workloads()[:2]
    sids = [tracer.load(w) for w in ws]
    try:
        p = [tracer.params(w.max_order) for w in ws]
        p[1].tiles_x = 2
        with pytest.raises(btrace.BtError) as e:
            btrace.bt_batch_create(tracer.ctx, sids, p)
        assert e.value.code == btrace.BT_E_INVALID
        p = [tracer.params(w.max_order) for w in ws]
        p[1].precision = btrace.BT_PREC_FP32
        with pytest.raises(btrace.BtError):
            btrace.bt_batch_create(tracer.ctx, sids, p)
        with pytest.raises(btrace.BtError):
            btrace.bt_batch_create(tracer.ctx, [sids[0], sids[0]], [p[0], p[0]])
        # a batch left alive is freed with its context
        b = btrace.bt_batch_create(tracer.ctx, sids, [tracer.params(w.max_order) for w in ws])
        btrace.bt_batch_run(tracer.ctx, b)
    finally:
        for sid in sids:
            btrace.bt_unload_scene(tracer.ctx, sid)


def test_batch_and_ranges_carry_directional_sources(tracer):
    # a scene with directional sources traced alone, in a batch with another
    # scene, and through the serving step (ranges of lineages, accumulated)
    # gives the same result every way; the directivity calls check their
    # state and arguments
    from paper_1912_03998_gb300 import btrace
    ws = uneven_workloads()[:2]
    w = ws[1]
    n_b = 20 * 4 ** w.level
    axes = btrace.bt_beam_axes(tracer.ctx, w.level)
    patterns = np.stack([0.5 + axes[:, 2] ** 2, np.linspace(0.0, 2.0, n_b)]).astype(np.float32)
    pattern_of = np.array([1, -1, 0][:len(w.src)], np.int32)
    sids = [tracer.load(x) for x in ws]
    try:
        btrace.bt_set_directivity(tracer.ctx, sids[1], patterns, pattern_of)
        p = [tracer.params(x.max_order) for x in ws]
        btrace.bt_trace(tracer.ctx, sids[1], p[1])
        alone = read(tracer, sids[1], w)
        b = btrace.bt_batch_create(tracer.ctx, sids, p)
        try:
            btrace.bt_batch_run(tracer.ctx, b)
            batched = read(tracer, sids[1], w)
        finally:
            btrace.bt_batch_destroy(b)
        assert (batched["cnt"] == alone["cnt"]).all()
        assert np.allclose(batched["I"], alone["I"], rtol=1e-9, atol=0)
        # in two ranges, accumulated
        n_lin = len(w.src) * n_b
        btrace.bt_set_microphones(tracer.ctx, sids[1], w.mics)  # zero the accumulators
        for lo, hi in ((0, n_lin // 3), (n_lin // 3, n_lin)):
            btrace.bt_trace_ranges(tracer.ctx, [sids[1], sids[0]], [lo, 0], [hi, 1], [p[1], p[0]], accumulate=True)
        ranged = read(tracer, sids[1], w)
        assert (ranged["cnt"] == alone["cnt"]).all()
        assert np.allclose(ranged["I"], alone["I"], rtol=1e-9, atol=0)
        # the patterns change the result, and clearing them restores the
        # omnidirectional trace
        btrace.bt_set_directivity(tracer.ctx, sids[1], None, None)
        btrace.bt_trace(tracer.ctx, sids[1], p[1])
        omni = read(tracer, sids[1], w)
        assert not np.allclose(omni["I"], alone["I"])
        r = tracer.run(w)
        assert np.allclose(omni["I"], r["I"], rtol=1e-9, atol=0)
        btrace.bt_unload_scene(tracer.ctx, r["scene_id"])
        # errors: a negative gain, a level out of range, an unloaded scene
        bad = patterns.copy()
        bad[0, 5] = -1.0
        with pytest.raises(btrace.BtError) as e:
            btrace.bt_set_directivity(tracer.ctx, sids[1], bad, pattern_of)
        assert e.value.code == btrace.BT_E_INVALID
        with pytest.raises(btrace.BtError):
            btrace.bt_beam_axes(tracer.ctx, 9)
    finally:
        for sid in sids:
            btrace.bt_unload_scene(tracer.ctx, sid)
    with pytest.raises(btrace.BtError) as e:
        btrace.bt_set_directivity(tracer.ctx, sids[1], patterns, pattern_of)
