"""bt_trace_noalloc: the trace for callers that must not allocate device memory
(a service under a device-memory budget fixed up front, a per-frame loop where
cudaMalloc/cudaFree would synchronise the device), checked against the regular
bt_trace + bt_read_levels path on two calls in a row, and against the FP64
oracle at the parity bar.

The two paths run the same kernels; only the lineages per launch differ, so
the float64 sums differ at most in their rounding order: intensities agree to
1e-9 relative and path counts exactly.

This file is collected last on purpose: it also runs on its own, in a fresh
process, because it sets up everything it uses.
"""
import numpy as np
import pytest

from paper_1912_03998_gb300 import synth
from tests.parity import assert_parity, level_db

pytestmark = pytest.mark.gpu

REL_TOL = 1e-9


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03998_gb300 import btrace
    t = btrace.Tracer(0)
    yield torch, btrace, t
    t.close()


def _case(name):
    """(workload, extra params, whether the scratch forces several launches)."""
    if name == "tiny_city":
        return synth.tiny_city(seed=2), {}, False
    if name == "tiny_city_3_sources_fp32":
        w = synth.tiny_city(seed=5, level=3, max_order=5, n_sources=3)
        return w, {"precision": 1}, False  # BT_PREC_FP32
    # Level 6 (81,920 beams a source) at order 6: the 32 MiB scratch holds the
    # MIXED beam table and about 19k lineages of segment records, so the 3
    # sources' 245,760 lineages take a dozen launches.
    return synth.tiny_city(seed=7, level=6, max_order=6, n_sources=3), {}, True


@pytest.mark.parametrize("case", ["tiny_city", "tiny_city_3_sources_fp32", "level6_many_launches"])
def test_noalloc_matches_regular_trace_twice(env, oracle_mod, case):
    torch, btrace, t = env
    w, extra, many = _case(case)
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
        # the call replaces the scene's result: read its intensities back
        I = np.empty((n, nb), np.float64)
        st = btrace.bt_read_levels(t.ctx, sid, None, I, None)
        reached = ref["I"] > 0
        assert ((I > 0) == reached).all(), f"{case}, call {call + 1}: microphones reached differ"
        rel = np.abs(I[reached] - ref["I"][reached]) / ref["I"][reached]
        assert rel.max(initial=0.0) <= REL_TOL, f"{case}, call {call + 1}: intensity rel. error {rel.max()}"
        Lh = L.cpu().numpy()
        both = np.isneginf(Lh) & np.isneginf(ref["level"])
        with np.errstate(invalid="ignore"):
            dl = np.where(both, 0.0, np.abs(Lh - ref["level"]))
        assert dl.max() <= 1e-7, f"{case}, call {call + 1}: level error {dl.max()} dB"
        assert (cnt.cpu().numpy() == ref["cnt"]).all()
        assert st["segments"] == ref["stats"]["segments"]
        assert st["emitted"] == ref["stats"]["emitted"]
        assert st["contributions"] == ref["stats"]["contributions"]
        assert st["candidates"] == ref["stats"]["candidates"]
        if many:
            assert st["trace_launches"] > 1 and st["scatter_launches"] == st["trace_launches"], st
    # the second call leaves free device memory exactly as it found it
    assert free[3] == free[2], free
    # and both paths meet the parity bar against the FP64 oracle
    r = oracle_mod.trace_workload(w)
    assert_parity(Lh, level_db(r["I"]), f"{case}: no-allocation trace vs oracle")
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


def test_noalloc_rejects_what_bt_trace_rejects_and_subdomains(env):
    torch, btrace, t = env
    w = synth.tiny_city(seed=2, level=2, max_order=2)
    sid = t.load(w)
    L = torch.empty((len(w.mics), 8), dtype=torch.float64, device="cuda")
    bad = t.params(w.max_order)
    bad.blocks_per_sm = 99  # bt_trace rejects this too
    with pytest.raises(btrace.BtError) as e:
        btrace.bt_trace_noalloc(t.ctx, sid, bad, L)
    assert e.value.code == btrace.BT_E_INVALID and "blocks_per_sm" in e.value.message
    tiled = t.params(w.max_order, tiles_x=2, tiles_y=2)
    with pytest.raises(btrace.BtError) as e:
        btrace.bt_trace_noalloc(t.ctx, sid, tiled, L)
    assert e.value.code == btrace.BT_E_INVALID and "1x1" in e.value.message
    btrace.bt_unload_scene(t.ctx, sid)
