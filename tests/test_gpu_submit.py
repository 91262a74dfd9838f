"""Asynchronous traces (bt_submit / bt_poll / bt_wait): a submitted trace
gives the synchronous trace's result; several scenes can be in flight at
once; a call naming a scene whose trace is in flight waits for it."""
import time

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


def read(tracer, w, sid):
    from paper_1912_03998_gb300 import btrace
    n, nb = len(w.mics), int(w.scene.refl.shape[1])
    I = np.empty((n, nb))
    cnt = np.empty(n, np.int32)
    st = btrace.bt_read_levels(tracer.ctx, sid, None, I, cnt)
    return I, cnt, st


def same(a, ref):
    I, cnt, st = a
    assert (cnt == ref["cnt"]).all()
    assert np.allclose(I, ref["I"], rtol=1e-9, atol=0)
    assert st["segments"] == ref["stats"]["segments"] and st["contributions"] == ref["stats"]["contributions"]


def test_submitted_traces_match_synchronous_ones(tracer):
    from paper_1912_03998_gb300 import btrace
    ws = [synth.tiny_city(seed=3, level=4, max_order=4, n_sources=2),
          synth.tiny_city(seed=6, level=5, max_order=3),
          synth.tiny_city(seed=8, level=4, max_order=5)]
    kws = [{}, {}, dict(tiles_x=4, tiles_y=4)]  # the sub-domain path too
    refs = [tracer.run(w, **kw) for w, kw in zip(ws, kws)]
    ids = [r["scene_id"] for r in refs]
    try:
        params = [tracer.params(w.max_order, **kw) for w, kw in zip(ws, kws)]
        for sid, p in zip(ids, params):
            btrace.bt_submit(tracer.ctx, sid, p)
        done = [False] * len(ids)
        t0 = time.monotonic()
        while not all(done) and time.monotonic() - t0 < 120.0:
            done = [d or btrace.bt_poll(tracer.ctx, sid) for d, sid in zip(done, ids)]
        assert all(done)
        for w, sid, ref in zip(ws, ids, refs):
            same(read(tracer, w, sid), ref)
            assert btrace.bt_poll(tracer.ctx, sid)  # a finished trace stays finished
        # bt_wait, and a read that names a scene still in flight waits for it
        btrace.bt_submit(tracer.ctx, ids[1], params[1])
        btrace.bt_wait(tracer.ctx, ids[1])
        same(read(tracer, ws[1], ids[1]), refs[1])
        btrace.bt_submit(tracer.ctx, ids[0], params[0])
        same(read(tracer, ws[0], ids[0]), refs[0])
        # submitting again before polling: the earlier trace finishes first
        btrace.bt_submit(tracer.ctx, ids[2], params[2])
        btrace.bt_submit(tracer.ctx, ids[2], params[2])
        btrace.bt_wait(tracer.ctx, ids[2])
        same(read(tracer, ws[2], ids[2]), refs[2])
    finally:
        for sid in ids:
            btrace.bt_unload_scene(tracer.ctx, sid)


def test_poll_without_a_trace_is_a_state_error(tracer):
    from paper_1912_03998_gb300 import btrace
    w = synth.tiny_city(seed=2, level=3, max_order=2)
    sid = tracer.load(w)
    try:
        for f in (btrace.bt_poll, btrace.bt_wait):
            with pytest.raises(btrace.BtError) as e:
                f(tracer.ctx, sid)
            assert e.value.code == btrace.BT_E_STATE
        bad = tracer.params(w.max_order)
        bad.max_order = -1
        with pytest.raises(btrace.BtError) as e:
            btrace.bt_submit(tracer.ctx, sid, bad)
        assert e.value.code == btrace.BT_E_INVALID
        with pytest.raises(btrace.BtError) as e:
            btrace.bt_poll(tracer.ctx, sid)  # nothing was enqueued
        assert e.value.code == btrace.BT_E_STATE
        with pytest.raises(btrace.BtError) as e:
            btrace.bt_poll(tracer.ctx, 63 if sid != 63 else 62)
        assert e.value.code == btrace.BT_E_INVALID
    finally:
        btrace.bt_unload_scene(tracer.ctx, sid)
