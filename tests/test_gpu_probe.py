"""The L2 probes (measurement aids of the bench): the read bandwidth, a
positive figure above the HBM copy bandwidth for an L2-resident buffer; the
float64 atomic-addition rate, whose every addition the library checks it
finds in the buffer; and their argument checks."""
import json
import os

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_l2_probe_beats_hbm_and_checks_arguments():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03998_gb300 import btrace
    with btrace.Tracer(0) as t:
        gbs = max(btrace.bt_l2_bandwidth(t.ctx, 48 << 20, 100, b) for b in (2, 4))
        assert gbs > 0
        peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(peaks):
            assert gbs > json.load(open(peaks))["hbm_gbs"], gbs
        for args in ((1 << 20, 10, 4), (48 << 20, 0, 4), (48 << 20, 10, 9), ((48 << 20) + 4, 10, 4)):
            with pytest.raises(btrace.BtError) as e:
                btrace.bt_l2_bandwidth(t.ctx, *args)
            assert e.value.code == btrace.BT_E_INVALID


def test_l2_atomics_probe_and_its_argument_checks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_03998_gb300 import btrace
    with btrace.Tracer(0) as t:
        # the library sums the buffer after the timed kernel and fails unless
        # it holds every addition
        ops = max(btrace.bt_l2_atomics(t.ctx, 32 << 20, 16, b) for b in (2, 4))
        assert 1e9 < ops < 1e13, ops
        for args in ((1 << 20, 10, 4), (32 << 20, 0, 4), (32 << 20, 10, 9), ((32 << 20) + 16, 10, 4)):
            with pytest.raises(btrace.BtError) as e:
                btrace.bt_l2_atomics(t.ctx, *args)
            assert e.value.code == btrace.BT_E_INVALID
