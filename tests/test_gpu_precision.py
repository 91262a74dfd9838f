"""Precision variants of the GPU trace against the FP64 oracle.

BT_PREC_MIXED (the default), BT_PREC_MIXED64 (float32 traversal, float64
image-source chain) and BT_PREC_FP64 are held to the parity bar (0.1 dB for
>= 99.9 % of microphones, 1 dB for all).  BT_PREC_FP32 is measured: the
district-scale matrix records its error beside the others, and the fraction
of hit/miss decisions that flip against the oracle's, from per-segment hit
logs of both.
"""
import json
import os

import numpy as np
import pytest

from paper_1912_03998_gb300 import synth
from tests.parity import assert_parity, level_db, summary

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


def gpu_run(tracer, w, **kw):
    from paper_1912_03998_gb300 import btrace
    r = tracer.run(w, **kw)
    btrace.bt_unload_scene(tracer.ctx, r["scene_id"])
    return r


def prec(name):
    from paper_1912_03998_gb300 import btrace
    return {"fp32": btrace.BT_PREC_FP32, "mixed": btrace.BT_PREC_MIXED, "fp64": btrace.BT_PREC_FP64,
            "mixed64": btrace.BT_PREC_MIXED64}[name]


def beam_map(tracer, oracle_mod, level):
    """The oracle's beam index of each of the library's beams, matched by axis
    (the two number the beams independently)."""
    from scipy.spatial import cKDTree

    from paper_1912_03998_gb300 import btrace
    ga = btrace.bt_beam_axes(tracer.ctx, level).reshape(-1, 3).astype(np.float64)
    oa = oracle_mod.beam_axes(level)
    d, idx = cKDTree(oa).query(ga)
    assert d.max() < 1e-6 and len(np.unique(idx)) == len(idx)
    return idx


def hit_flips(tracer, oracle_mod, w, oracle_hits, **kw):
    """Trace w on the GPU with a hit log; compare every segment both traces
    reached: (flipped decisions, common segments, segments one side only)."""
    import torch

    from paper_1912_03998_gb300 import btrace
    n_beams = 20 * 4 ** w.level
    sid = tracer.load(w)
    hits = torch.full((len(w.src) * n_beams, w.max_order + 1), -2, dtype=torch.int32, device="cuda")
    btrace.bt_set_hit_log(tracer.ctx, sid, hits)
    tracer.run(w, sid=sid, **kw)
    btrace.bt_set_hit_log(tracer.ctx, sid, None)
    btrace.bt_unload_scene(tracer.ctx, sid)
    g = hits.cpu().numpy()
    bm = beam_map(tracer, oracle_mod, w.level)
    lin_o = (np.arange(len(w.src))[:, None] * n_beams + bm[None, :]).reshape(-1)
    o = oracle_hits[lin_o]
    both = (g >= -1) & (o >= -1)
    flips = int((both & (g != o)).sum())
    return flips, int(both.sum()), int(((g >= -1) != (o >= -1)).sum())


def test_fp64_free_field_closed_form(tracer):
    w = synth.free_field(seed=3, level=3, n_mics=777)
    g = gpu_run(tracer, w, precision=prec("fp64"))
    rr = np.linalg.norm(w.mics.astype(np.float64) - w.src[0].astype(np.float64), axis=1)
    expect = w.power[0].astype(np.float64)[None, :] / (4 * np.pi * rr[:, None] ** 2)
    assert (g["cnt"] == 1).all()
    # band powers are float32, the rest float64
    assert np.abs(g["I"] / expect - 1).max() < 1e-6


@pytest.mark.parametrize("n_boxes,max_order", [(1, 2), (2, 3), (4, 4)])
def test_fp64_box_path_counts_exact(tracer, oracle_mod, n_boxes, max_order):
    w = synth.boxes(n_boxes, seed=5, level=5, max_order=max_order, n_grid=24)
    g = gpu_run(tracer, w, precision=prec("fp64"))
    r = oracle_mod.trace_workload(w)
    assert (g["cnt"] == r["cnt"]).all(), np.nonzero(g["cnt"] != r["cnt"])
    assert_parity(g["level"], level_db(r["I"]), f"boxes{n_boxes}, FP64")


@pytest.mark.parametrize("seed", [1, 2])
def test_fp64_tiny_city(tracer, oracle_mod, seed):
    w = synth.tiny_city(seed=seed)
    g = gpu_run(tracer, w, precision=prec("fp64"))
    r = oracle_mod.trace_workload(w)
    s = assert_parity(g["level"], level_db(r["I"]), f"tiny city seed {seed}, FP64")
    assert (g["cnt"] == r["cnt"]).mean() >= 0.999, s
    assert g["stats"]["segments"] == r["stats"]["segments"]


def test_fp64_sub_domains_match_unsplit(tracer):
    w = synth.tiny_city(seed=3, level=4, max_order=4, n_sources=2)
    base = gpu_run(tracer, w, precision=prec("fp64"))
    g = gpu_run(tracer, w, precision=prec("fp64"), tiles_x=4, tiles_y=4)
    assert g["stats"]["handoffs"] > 0
    assert (g["cnt"] == base["cnt"]).all()
    assert np.allclose(g["I"], base["I"], rtol=1e-12, atol=0)


@pytest.mark.parametrize("name", ["mixed64", "mixed", "fp32", "fp64"])
def test_hit_logs_against_the_oracle_tiny_city(tracer, oracle_mod, name):
    """Per-segment hit logs: on the tiny city every variant takes the oracle's
    hit decisions on (nearly) every segment, and the log holds exactly the
    trace's hits and escapes."""
    w = synth.tiny_city(seed=2, level=4, max_order=4, n_sources=2)
    r = oracle_mod.trace_workload(w, hit_log=True)
    assert (r["hits"] >= 0).sum() == r["stats"]["hits"] and (r["hits"] == -1).sum() == r["stats"]["escapes"]
    flips, common, one_side = hit_flips(tracer, oracle_mod, w, r["hits"], precision=prec(name), tiles_x=2, tiles_y=2)
    assert common >= 0.999 * r["stats"]["segments"]
    assert flips <= (1e-3 if name == "fp32" else 1e-4) * common, (name, flips, common, one_side)


def test_mixed64_parity(tracer, oracle_mod):
    for seed in (1, 2):
        w = synth.tiny_city(seed=seed)
        g = gpu_run(tracer, w, precision=prec("mixed64"))
        r = oracle_mod.trace_workload(w)
        assert_parity(g["level"], level_db(r["I"]), f"tiny city seed {seed}, MIXED64")
        assert g["stats"]["segments"] == r["stats"]["segments"]
    w = synth.boxes(2, seed=5, level=5, max_order=3, n_grid=24)
    g = gpu_run(tracer, w, precision=prec("mixed64"), tiles_x=2, tiles_y=2)
    r = oracle_mod.trace_workload(w)
    assert (g["cnt"] == r["cnt"]).all()


def test_precision_matrix_district(tracer, oracle_mod):
    # The district configuration (all 1,000 sources, 250,000 microphones,
    # 4x4 sub-domains) in each precision; the oracle computes a seeded sample
    # of 10,000 microphones from all sources.  Per variant: max and 99.9th
    # percentile dB error over microphones and bands, the fraction within
    # 0.1 dB, microphones whose path count differs from the oracle's (the
    # visible trace of flipped hit or in-beam decisions), segment and hit
    # counts against the oracle's, and the trace's device time.
    w = synth.district(seed=2)
    pick = np.sort(np.random.Generator(np.random.PCG64(33)).choice(len(w.mics), 10000, replace=False))
    r = oracle_mod.trace_workload(w.with_mics(w.mics[pick]), n_threads=max(1, os.cpu_count() or 1))
    L_ref = level_db(r["I"])
    rows = {}
    # hit/miss decisions: per-segment hit logs on the first 16 sources (all
    # their segments), against the oracle's
    w16 = w.subset_sources(np.arange(16)).with_mics(w.mics[pick[:64]])
    r16 = oracle_mod.trace_workload(w16, n_threads=max(1, os.cpu_count() or 1), hit_log=True)
    for name in ("fp32", "mixed", "mixed64", "fp64"):
        g = gpu_run(tracer, w, precision=prec(name), tiles_x=4, tiles_y=4)
        s = summary(g["level"][pick], L_ref)
        st = g["stats"]
        rows[name] = dict(max_db=s["max_db"], p999_db=s["p999_db"], frac_within_0p1=s["frac_within_0p1"],
                          path_count_mismatch=float((g["cnt"][pick] != r["cnt"]).mean()),
                          segments=st["segments"], oracle_segments=int(r["stats"]["segments"]),
                          hits=st["hits"], oracle_hits=int(r["stats"]["hits"]),
                          trace_ms=st["trace_ms"],
                          segments_per_s=st["segments"] / (st["trace_ms"] * 1e-3))
        flips, common, one_side = hit_flips(tracer, oracle_mod, w16, r16["hits"], precision=prec(name),
                                            tiles_x=4, tiles_y=4)
        rows[name].update(hit_flip_fraction=flips / common, segments_compared=common,
                          segments_one_side_only=one_side)
    print("PRECISION_MATRIX " + json.dumps(rows))
    for name in ("mixed", "mixed64", "fp64"):
        assert rows[name]["frac_within_0p1"] >= 0.999 and rows[name]["max_db"] <= 1.0, (name, rows[name])
