"""bt_trace_noalloc: the trace for callers that must not allocate device memory
(a service under a device-memory budget fixed up front, a per-frame loop where
cudaMalloc/cudaFree would synchronise the device), checked against the regular
bt_trace + bt_read_levels path on two calls in a row.

This file is collected last on purpose: it also runs on its own, in a fresh
process, because it sets up everything it uses.
"""
import numpy as np
import pytest

from paper_1912_03998_gb300 import synth
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03998_gb300 import btrace
    t = btrace.Tracer(0)
    yield torch, btrace, t
    t.close()


@pytest.mark.parametrize("case", ["tiny_city", "tiny_city_3_sources_fp32"])
def test_noalloc_matches_regular_trace_twice(env, case):
    torch, btrace, t = env
    if case == "tiny_city":
        w, extra = synth.tiny_city(seed=2), {}
    else:
        w = synth.tiny_city(seed=5, level=3, max_order=5, n_sources=3)
        extra = {"precision": btrace.BT_PREC_FP32}
    ref = t.run(w, **extra)  # the regular entry points
    sid = ref["scene_id"]
    params = t.params(w.max_order, **extra)
    n, nb = len(w.mics), w.scene.refl.shape[1]
    free = []
    for call in range(2):
        # stale contents must be overwritten by every call
        L = torch.full((n, nb), 7.0, dtype=torch.float64, device="cuda")
        cnt = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        btrace.bt_trace_noalloc(t.ctx, sid, params, L, cnt)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert_parity(L.cpu().numpy(), ref["level"], f"{case}, no-allocation call {call + 1}")
        assert (cnt.cpu().numpy() == ref["cnt"]).all()
        st = btrace.bt_read_levels(t.ctx, sid)
        assert st["segments"] == ref["stats"]["segments"]
        assert st["contributions"] == ref["stats"]["contributions"]
    # the second call leaves free device memory exactly as it found it
    assert free[3] == free[2], free
    btrace.bt_unload_scene(t.ctx, sid)


def test_noalloc_rejects_levels_beyond_its_scratch(env):
    torch, btrace, t = env
    w = synth.free_field(seed=1, level=7)  # one above the limit of 6
    sid = t.load(w)
    L = torch.empty((len(w.mics), 8), dtype=torch.float64, device="cuda")
    with pytest.raises(btrace.BtError) as e:
        btrace.bt_trace_noalloc(t.ctx, sid, t.params(w.max_order), L)
    assert e.value.code == btrace.BT_E_INVALID
    assert "level 7" in e.value.message and "limit" in e.value.message
    btrace.bt_unload_scene(t.ctx, sid)
