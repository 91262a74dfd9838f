"""The device-side failure paths, triggered on purpose through the trace's test
hook (bt_trace_params.fault_test), with nothing that faults or hangs the GPU:

* BT_FAULT_WITHHOLD: the sub-domain trace never publishes its first hand-off,
  so the consumer that took it waits on the queue slot until the watchdog
  (watchdog_ms, here 50 ms) runs out; the trace returns BT_E_TIMEOUT.
* BT_FAULT_SEGMENTS: the segment buffer has room for one record, so the
  warp-aggregated append overflows; the trace returns BT_E_QUEUE_FULL.

After each failure the same context and scene trace normally again and match
the FP64 oracle.
"""
import time

import pytest

from paper_1912_03998_gb300 import synth
from tests.parity import assert_parity, level_db

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03998_gb300 import btrace
    t = btrace.Tracer(0)
    yield btrace, t
    t.close()


def recover(btrace, t, oracle_mod, w, sid, **kw):
    g = t.run(w, sid=sid, **kw)
    r = oracle_mod.trace_workload(w)
    assert_parity(g["level"], level_db(r["I"]), "trace after a failure")
    assert g["stats"]["segments"] == r["stats"]["segments"]
    return g


def test_withheld_handoff_times_out_and_context_recovers(env, oracle_mod):
    btrace, t = env
    w = synth.tiny_city(seed=3, level=4, max_order=4)
    sid = t.load(w)
    ok = t.run(w, sid=sid, tiles_x=3, tiles_y=3)
    assert ok["stats"]["handoffs"] > 0  # the hook needs a hand-off to withhold
    t0 = time.perf_counter()
    with pytest.raises(btrace.BtError) as e:
        btrace.bt_trace(t.ctx, sid, t.params(w.max_order, tiles_x=3, tiles_y=3, watchdog_ms=50,
                                             fault_test=btrace.BT_FAULT_WITHHOLD))
    assert e.value.code == btrace.BT_E_TIMEOUT, e.value
    assert time.perf_counter() - t0 < 20.0  # bounded by the watchdog, not a hang
    # the scene reports the failed trace until it is traced again
    with pytest.raises(btrace.BtError) as e2:
        btrace.bt_read_levels(t.ctx, sid)
    assert e2.value.code == btrace.BT_E_TIMEOUT
    recover(btrace, t, oracle_mod, w, sid, tiles_x=3, tiles_y=3)
    recover(btrace, t, oracle_mod, w, sid)
    btrace.bt_unload_scene(t.ctx, sid)


@pytest.mark.parametrize("tiles", [(1, 1), (2, 2)])
def test_segment_overflow_reports_queue_full_and_context_recovers(env, oracle_mod, tiles):
    btrace, t = env
    w = synth.tiny_city(seed=6, level=3, max_order=3)
    sid = t.load(w)
    with pytest.raises(btrace.BtError) as e:
        btrace.bt_trace(t.ctx, sid, t.params(w.max_order, tiles_x=tiles[0], tiles_y=tiles[1],
                                             fault_test=btrace.BT_FAULT_SEGMENTS))
    assert e.value.code == btrace.BT_E_QUEUE_FULL, e.value
    recover(btrace, t, oracle_mod, w, sid, tiles_x=tiles[0], tiles_y=tiles[1])
    btrace.bt_unload_scene(t.ctx, sid)
