"""GPU parity: libbtrace (called through its C ABI) against the FP64 oracle.

Bar: per microphone and band, level within 0.1 dB for >= 99.9% of
microphones and within 1 dB for all; microphones no beam reached are -inf on
both sides; path counts exact on the small brute-force scenes.
"""
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


def oracle_levels(oracle_mod, w, **kw):
    r = oracle_mod.trace_workload(w, **kw)
    return r, level_db(r["I"])


def gpu_run(tracer, w, **kw):
    r = tracer.run(w, **kw)
    tracer_sid = r["scene_id"]
    from paper_1912_03998_gb300 import btrace
    btrace.bt_unload_scene(tracer.ctx, tracer_sid)
    return r


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("level", [0, 2, 4])
def test_free_field(tracer, oracle_mod, level):
    w = synth.free_field(seed=3, level=level, n_mics=777)
    g = gpu_run(tracer, w)
    rr = np.linalg.norm(w.mics.astype(np.float64) - w.src[0].astype(np.float64), axis=1)
    expect = w.power[0].astype(np.float64)[None, :] / (4 * np.pi * rr[:, None] ** 2)
    assert (g["cnt"] == 1).all()
    assert np.abs(g["I"] / expect - 1).max() < 1e-5
    assert g["stats"]["segments"] == 20 * 4 ** level and g["stats"]["hits"] == 0


def test_ground_plane(tracer, oracle_mod):
    w = synth.ground_only(seed=1, level=5)
    g = gpu_run(tracer, w)
    r, L = oracle_levels(oracle_mod, w)
    assert_parity(g["level"], L, "ground plane")
    assert (g["cnt"] == r["cnt"]).mean() >= 0.99


def test_single_wall(tracer, oracle_mod):
    w = synth.single_wall(seed=2, level=4)
    g = gpu_run(tracer, w)
    r, L = oracle_levels(oracle_mod, w)
    assert_parity(g["level"], L, "single wall")
    assert (g["cnt"] == 2).all()


# ------------------------------------------------------------- tiny scenes
@pytest.mark.parametrize("n_boxes,max_order", [(1, 4), (2, 4), (4, 3)])
def test_boxes_path_counts_exact(tracer, oracle_mod, n_boxes, max_order):
    w = synth.boxes(n_boxes, seed=5, level=5, max_order=max_order, n_grid=24)
    g = gpu_run(tracer, w)
    r, L = oracle_levels(oracle_mod, w)
    assert (g["cnt"] == r["cnt"]).all(), np.nonzero(g["cnt"] != r["cnt"])
    assert_parity(g["level"], L, f"boxes{n_boxes}")


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tiny_city(tracer, oracle_mod, seed):
    w = synth.tiny_city(seed=seed)  # 8x8 boxes, L = 4, K = 4, 32x32 microphones
    g = gpu_run(tracer, w)
    r, L = oracle_levels(oracle_mod, w)
    s = assert_parity(g["level"], L, f"tiny city seed {seed}")
    assert (g["cnt"] == r["cnt"]).mean() >= 0.999, s
    assert g["stats"]["segments"] == r["stats"]["segments"]


def test_tiny_city_many_sources_air_damping(tracer, oracle_mod):
    w = synth.tiny_city(seed=7, level=4, max_order=5, n_sources=9, n_grid=48)
    w.power[:] = np.random.Generator(np.random.PCG64(3)).uniform(0.01, 1.0, w.power.shape)
    alpha = np.linspace(0.0, 0.04, synth.N_BANDS)
    g = gpu_run(tracer, w, air_atten_db_per_m=alpha)
    r, L = oracle_levels(oracle_mod, w, alpha=alpha, n_threads=4)
    assert_parity(g["level"], L, "tiny city, 9 sources, air damping")


def test_energy_threshold(tracer, oracle_mod):
    w = synth.tiny_city(seed=3, level=3, max_order=6)
    g = gpu_run(tracer, w, energy_threshold_w=0.75)
    r, L = oracle_levels(oracle_mod, w, energy_threshold=0.75)
    assert_parity(g["level"], L, "threshold")
    assert g["stats"]["segments"] == r["stats"]["segments"]


# ------------------------------------------------------------- edge cases
def test_ragged_and_degenerate_sizes(tracer, oracle_mod):
    # ragged microphone counts, microphones outside the city and at many heights,
    # K = 0, level 0, a single triangle scene
    base = synth.tiny_city(seed=4, level=3, max_order=3)
    rng = np.random.Generator(np.random.PCG64(9))
    mics = np.column_stack([rng.uniform(-300, 900, 4999), rng.uniform(-300, 900, 4999),
                            rng.uniform(0.0, 90.0, 4999)]).astype(np.float32)
    for w in (base.with_mics(mics), base.with_mics(mics[:1]), base.with_mics(mics[:33])):
        g = gpu_run(tracer, w)
        _, L = oracle_levels(oracle_mod, w)
        assert_parity(g["level"], L, f"{len(w.mics)} mics")
    for level, K in ((0, 0), (0, 2), (2, 0)):
        w = synth.tiny_city(seed=4, level=level, max_order=K)
        g = gpu_run(tracer, w)
        r, L = oracle_levels(oracle_mod, w)
        assert_parity(g["level"], L, f"L={level} K={K}")
        assert g["stats"]["segments"] == r["stats"]["segments"]
    one = synth.Scene(np.array([[-50, -50, 0], [50, -50, 0], [0, 80, 0]], np.float32),
                      np.array([[0, 1, 2]], np.int32), np.zeros(1, np.uint8), synth.refl_table())
    w = synth.Workload("one", one, np.array([[1, 2, 3]], np.float32), np.ones((1, 8), np.float32),
                       synth.mic_grid(-40, -40, 40, 40, 9, 9, 1.0), 4, 2)
    g = gpu_run(tracer, w)
    r, L = oracle_levels(oracle_mod, w)
    assert_parity(g["level"], L, "single triangle")
    assert (g["cnt"] == r["cnt"]).all()


def test_empty_inputs(tracer):
    from paper_1912_03998_gb300 import btrace
    w = synth.free_field(seed=1, level=1)
    # no sources: zero intensity everywhere
    w0 = synth.Workload("nosrc", w.scene, np.zeros((0, 3), np.float32), np.zeros((0, 8), np.float32),
                        w.mics, 1, 2)
    g = gpu_run(tracer, w0)
    assert (g["I"] == 0).all() and np.isneginf(g["level"]).all() and (g["cnt"] == 0).all()
    # no microphones
    w1 = w.with_mics(np.zeros((0, 3), np.float32))
    g = gpu_run(tracer, w1)
    assert g["level"].shape == (0, 8) and g["stats"]["segments"] == 20 * 4


def test_invalid_inputs_rejected(tracer):
    from paper_1912_03998_gb300 import btrace
    ctx = tracer.ctx
    w = synth.tiny_city(seed=1, level=1, max_order=1)
    bad_v = w.scene.verts.copy()
    bad_v[5, 2] = np.nan
    with pytest.raises(btrace.BtError) as e:
        btrace.bt_load_scene(ctx, bad_v, w.scene.tris, w.scene.mat, w.scene.refl)
    assert e.value.code == btrace.BT_E_INVALID
    bad_t = w.scene.tris.copy()
    bad_t[3, 1] = len(w.scene.verts)
    with pytest.raises(btrace.BtError) as e:
        btrace.bt_load_scene(ctx, w.scene.verts, bad_t, w.scene.mat, w.scene.refl)
    assert e.value.code == btrace.BT_E_INVALID
    bad_m = w.scene.mat.copy()
    bad_m[0] = 7
    with pytest.raises(btrace.BtError):
        btrace.bt_load_scene(ctx, w.scene.verts, w.scene.tris, bad_m, w.scene.refl)
    with pytest.raises(btrace.BtError):
        btrace.bt_load_scene(ctx, w.scene.verts, w.scene.tris, w.scene.mat, w.scene.refl * 2)
    sid = btrace.bt_load_scene(ctx, w.scene.verts, w.scene.tris, w.scene.mat, w.scene.refl)
    p = btrace.bt_params_default()
    with pytest.raises(btrace.BtError) as e:
        btrace.bt_trace(ctx, sid, p)  # no sources yet
    assert e.value.code == btrace.BT_E_STATE
    with pytest.raises(btrace.BtError):
        btrace.bt_set_sources(ctx, sid, w.src, -w.power, 1)
    with pytest.raises(btrace.BtError):
        btrace.bt_set_sources(ctx, sid, w.src, w.power, 9)
    btrace.bt_set_sources(ctx, sid, w.src, w.power, 1)
    m = w.mics.copy()
    m[3, 0] = np.inf
    with pytest.raises(btrace.BtError):
        btrace.bt_set_microphones(ctx, sid, m)
    btrace.bt_set_microphones(ctx, sid, w.mics)
    p.max_order = 33
    with pytest.raises(btrace.BtError):
        btrace.bt_trace(ctx, sid, p)
    p.max_order = 1
    for depth in (16, 48, 1 << 23):
        p.queue_depth = depth
        with pytest.raises(btrace.BtError) as e:
            btrace.bt_trace(ctx, sid, p)
        assert e.value.code == btrace.BT_E_INVALID
    p.queue_depth = 0
    btrace.bt_trace(ctx, sid, p)  # the context still works after the errors
    btrace.bt_unload_scene(ctx, sid)


def test_device_pointer_inputs_match_host(tracer):
    torch = pytest.importorskip("torch")
    from paper_1912_03998_gb300 import btrace
    ctx = tracer.ctx
    w = synth.tiny_city(seed=6, level=3, max_order=3)
    host = gpu_run(tracer, w)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sid = btrace.bt_load_scene(ctx, dev(w.scene.verts), dev(w.scene.tris), dev(w.scene.mat),
                               dev(w.scene.refl))
    btrace.bt_set_sources(ctx, sid, dev(w.src), dev(w.power), w.level)
    btrace.bt_set_microphones(ctx, sid, dev(w.mics))
    p = btrace.bt_params_default()
    p.max_order = w.max_order
    btrace.bt_trace(ctx, sid, p)
    L = torch.empty((len(w.mics), 8), dtype=torch.float64, device="cuda")
    cnt = torch.empty(len(w.mics), dtype=torch.int32, device="cuda")
    btrace.bt_read_levels(ctx, sid, L, None, cnt)
    torch.cuda.synchronize()
    assert (cnt.cpu().numpy() == host["cnt"]).all()
    Lh = L.cpu().numpy()
    assert np.allclose(Lh[np.isfinite(Lh)], host["level"][np.isfinite(host["level"])], rtol=0, atol=1e-9)
    btrace.bt_unload_scene(ctx, sid)


def test_repeat_trace_is_reproducible(tracer):
    w = synth.tiny_city(seed=2, level=4, max_order=4, n_sources=3)
    a = tracer.run(w)
    from paper_1912_03998_gb300 import btrace
    b = tracer.run(w, sid=a["scene_id"])
    assert (a["cnt"] == b["cnt"]).all()
    assert np.allclose(a["I"], b["I"], rtol=1e-12, atol=0)
    btrace.bt_unload_scene(tracer.ctx, a["scene_id"])


def test_source_linearity(tracer):
    # beams of different sources never interact: tracing A u B equals A + B
    w = synth.tiny_city(seed=8, level=3, max_order=4, n_sources=6)
    ab = gpu_run(tracer, w)
    a = gpu_run(tracer, w.subset_sources(np.arange(0, 3)))
    b = gpu_run(tracer, w.subset_sources(np.arange(3, 6)))
    assert (ab["cnt"] == a["cnt"] + b["cnt"]).all()
    assert np.allclose(ab["I"], a["I"] + b["I"], rtol=1e-9, atol=0)


# ------------------------------------------------------- volumetric microphones
def test_volumetric_microphones(tracer, oracle_mod):
    # microphones through the whole height of the city (Section 4's receivers
    # fill a volume): binned in xy cells and height layers
    base = synth.tiny_city(seed=7, level=4, max_order=4, n_sources=2)
    layers = [synth.mic_grid(10.0, 10.0, 550.0, 550.0, 20, 20, z) for z in np.linspace(1.5, 71.5, 8)]
    w = base.with_mics(np.concatenate(layers).astype(np.float32))
    g = gpu_run(tracer, w)
    r, L = oracle_levels(oracle_mod, w)
    s = assert_parity(g["level"], L, "volumetric microphones")
    assert (g["cnt"] == r["cnt"]).mean() >= 0.999, s
    assert g["stats"]["segments"] == r["stats"]["segments"]
    assert (r["cnt"] > 0).mean() > 0.3  # many microphones sit inside buildings
    # split 4x4 as well
    g4 = gpu_run(tracer, w, tiles_x=4, tiles_y=4)
    assert (g4["cnt"] == g["cnt"]).all() and np.allclose(g4["I"], g["I"], rtol=1e-9, atol=0)



def test_scatter_in_order_of_place(tracer, oracle_mod):
    # More than 2^20 microphones: the trace scatters its segments in order of
    # the grid cell under each one.  The result must be the one the
    # trace-order scatter gives: here the same microphones traced in two
    # blocks below that size, whose scatters keep the trace order.
    from paper_1912_03998_gb300 import shard
    base = synth.tiny_city(seed=11, level=4, max_order=4, n_sources=3)
    layers = [synth.mic_grid(5.0, 5.0, 555.0, 555.0, 380, 380, z) for z in np.linspace(1.5, 50.0, 8)]
    mics = np.concatenate(layers).astype(np.float32)
    assert len(mics) > (1 << 20)
    w = base.with_mics(mics)
    full = gpu_run(tracer, w)
    parts = []
    for r in range(2):
        lo, hi = shard.mic_block(len(mics), r, 2)
        assert hi - lo <= (1 << 20)
        parts.append(gpu_run(tracer, w.with_mics(mics[lo:hi])))
    cnt = np.concatenate([g["cnt"] for g in parts])
    I = np.concatenate([g["I"] for g in parts])
    assert (cnt == full["cnt"]).all()
    assert np.allclose(I, full["I"], rtol=1e-9, atol=0)
    assert full["stats"]["contributions"] == sum(g["stats"]["contributions"] for g in parts)
    # sub-domains and order of place together
    g4 = gpu_run(tracer, w, tiles_x=2, tiles_y=2)
    assert (g4["cnt"] == full["cnt"]).all() and np.allclose(g4["I"], full["I"], rtol=1e-9, atol=0)
    # and the oracle on a sample of the microphones
    idx = np.random.default_rng(3).choice(len(mics), 3000, replace=False)
    r, L = oracle_levels(oracle_mod, w.with_mics(mics[idx]))
    assert_parity(full["level"][idx], L, "order of place, sampled microphones")
    assert (full["cnt"][idx] == r["cnt"]).mean() >= 0.999

# ------------------------------------------------------------- district scale
@pytest.fixture(scope="module")
def district():
    return synth.district(seed=2)


def test_district_source_subset(tracer, oracle_mod, district):
    # full-size district (about 200k triangles, 250k microphones, L = 5,
    # K = 6) on a seeded subset of 16 of its 1,000 sources
    import os
    idx = np.random.Generator(np.random.PCG64(21)).choice(len(district.src), 16, replace=False)
    w = district.subset_sources(np.sort(idx))
    g = gpu_run(tracer, w)
    r, L = oracle_levels(oracle_mod, w, n_threads=max(1, os.cpu_count() or 1))
    s = assert_parity(g["level"], L, "district, 16 sources")
    reached = r["cnt"] > 0
    assert reached.sum() > 10000
    assert abs(g["stats"]["segments"] / r["stats"]["segments"] - 1) < 1e-3, (g["stats"], r["stats"])
    print("district 16 sources:", s)


# ------------------------------------------------------------- hit queries
@pytest.mark.parametrize("scene_name", ["tiny", "district"])
def test_cast_rays_match_oracle(tracer, oracle_mod, scene_name, district):
    # a4 on its own: the closest hit of seeded random rays, GPU vs oracle on
    # the same float32 rays; the triangle index must agree exactly
    from paper_1912_03998_gb300 import btrace
    w = synth.tiny_city(seed=4) if scene_name == "tiny" else district
    lo, hi = w.scene.verts.min(0), w.scene.verts.max(0)
    rng = np.random.Generator(np.random.PCG64(12))
    n = 200_000
    o = np.column_stack([rng.uniform(lo[0] + 500, hi[0] - 500, n), rng.uniform(lo[1] + 500, hi[1] - 500, n),
                         rng.uniform(0.1, 60.0, n)]).astype(np.float32)
    d = rng.normal(size=(n, 3)).astype(np.float32)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    sid = btrace.bt_load_scene(tracer.ctx, w.scene.verts, w.scene.tris, w.scene.mat, w.scene.refl)
    tg, ig = btrace.bt_cast_rays(tracer.ctx, sid, o, d)
    btrace.bt_unload_scene(tracer.ctx, sid)
    dd = d.astype(np.float64)
    dd /= np.linalg.norm(dd, axis=1, keepdims=True)
    to, io = oracle_mod.cast_rays(oracle_mod.Scene(w.scene), o.astype(np.float64), dd,
                                  mode=oracle_mod.HIT_BVH)
    assert (io >= 0).mean() > 0.3
    mism = np.nonzero(ig != io)[0]
    assert len(mism) <= n * 1e-5, [(int(i), int(ig[i]), float(tg[i]), int(io[i]), float(to[i])) for i in mism[:10]]
    hit = (io >= 0) & (ig == io)
    # both sides take the same float32 origins and directions; the library
    # reports the float64 distance to the hit triangle's plane rounded to
    # float32 (half an ulp: 6e-8 relative), the oracle its float64 one
    assert np.allclose(tg[hit], to[hit], rtol=2e-7, atol=1e-6)


def test_fp32_precision_mode(tracer, oracle_mod):
    from paper_1912_03998_gb300 import btrace
    w = synth.tiny_city(seed=2)
    g = gpu_run(tracer, w, precision=btrace.BT_PREC_FP32)
    _, L = oracle_levels(oracle_mod, w)
    assert_parity(g["level"], L, "tiny city, FP32 chain")


def test_district_full_size_sampled_microphones(tracer, oracle_mod, district):
    # the bench configuration itself: all 1,000 sources and all 250,000
    # microphones on the GPU; the oracle computes a seeded sample of 10,000
    # microphones from all sources (the 99.9 % bar then allows 10 outliers) (a microphone's result does not depend on
    # the other microphones)
    import os
    g = gpu_run(tracer, district)
    pick = np.sort(np.random.Generator(np.random.PCG64(33)).choice(len(district.mics), 10000, replace=False))
    r, L = oracle_levels(oracle_mod, district.with_mics(district.mics[pick]),
                         n_threads=max(1, os.cpu_count() or 1))
    s = assert_parity(g["level"][pick], L, "district, 1000 sources, sampled microphones")
    assert (g["cnt"][pick] == r["cnt"]).mean() >= 0.999
    assert (r["cnt"] > 0).mean() > 0.5
    assert abs(g["stats"]["segments"] / r["stats"]["segments"] - 1) < 1e-4
    print("district full size, 10000 sampled microphones:", s)


# ------------------------------------------------------------- sub-domains
@pytest.mark.parametrize("tiles", [(2, 2), (4, 4), (3, 5)])
def test_tiles_match_oracle_and_unsplit(tracer, oracle_mod, tiles):
    # Section 3: splitting the geometry into sub-domains with beam hand-off
    # must not change any result
    w = synth.tiny_city(seed=3, level=4, max_order=4, n_sources=2)
    base = gpu_run(tracer, w)
    g = gpu_run(tracer, w, tiles_x=tiles[0], tiles_y=tiles[1])
    r, L = oracle_levels(oracle_mod, w)
    assert_parity(g["level"], L, f"tiles {tiles}")
    assert (g["cnt"] == base["cnt"]).all()
    assert np.allclose(g["I"], base["I"], rtol=1e-9, atol=0)
    assert g["stats"]["segments"] == base["stats"]["segments"] == r["stats"]["segments"]
    assert g["stats"]["handoffs"] > 0 and g["stats"]["rounds"] >= 1


def test_tiles_tiny_queues(tracer, oracle_mod):
    # 32-slot hand-off queues: at most 32 lineages in flight and rings that
    # wrap many times; neither may change a result
    w = synth.tiny_city(seed=5, level=4, max_order=4, n_sources=3)
    base = gpu_run(tracer, w)
    g = gpu_run(tracer, w, tiles_x=4, tiles_y=4, queue_depth=32)
    assert g["stats"]["handoffs"] > 32 * 16
    assert (g["cnt"] == base["cnt"]).all()
    assert np.allclose(g["I"], base["I"], rtol=1e-9, atol=0)
    assert g["stats"]["segments"] == base["stats"]["segments"]
    g2 = gpu_run(tracer, w, tiles_x=4, tiles_y=4, queue_depth=32, chunk_beams=777)
    assert (g2["cnt"] == base["cnt"]).all() and g2["stats"]["rounds"] > 1
    assert np.allclose(g2["I"], base["I"], rtol=1e-9, atol=0)


def test_tiles_district_source_subset(tracer, oracle_mod, district):
    import os
    idx = np.random.Generator(np.random.PCG64(21)).choice(len(district.src), 16, replace=False)
    w = district.subset_sources(np.sort(idx))
    g = gpu_run(tracer, w, tiles_x=4, tiles_y=4)
    r, L = oracle_levels(oracle_mod, w, n_threads=max(1, os.cpu_count() or 1))
    assert_parity(g["level"], L, "district, 16 sources, 4x4 tiles")
    assert abs(g["stats"]["segments"] / r["stats"]["segments"] - 1) < 1e-4
    assert g["stats"]["handoffs"] > 0 and g["stats"]["steals"] >= 0


# ------------------------------------------------------------- source shards
def test_source_shards_sum_to_the_full_trace(tracer):
    # Section 3: results of disjoint source sets are gathered by summation;
    # three shards traced separately, summed on the host and installed with
    # bt_set_result give the one-trace result
    from paper_1912_03998_gb300 import btrace, shard
    w = synth.tiny_city(seed=8, level=4, max_order=4, n_sources=7)
    full = gpu_run(tracer, w)
    I = np.zeros_like(full["I"])
    cnt = np.zeros_like(full["cnt"])
    for r in range(3):
        lo, hi = shard.source_block(len(w.src), r, 3)
        g = gpu_run(tracer, w.subset_sources(np.arange(lo, hi)))
        I += g["I"]
        cnt += g["cnt"]
    sid = tracer.load(w)
    btrace.bt_set_result(tracer.ctx, sid, I, cnt)
    L = np.empty_like(full["level"])
    I2 = np.empty_like(full["I"])
    c2 = np.empty_like(full["cnt"])
    btrace.bt_read_levels(tracer.ctx, sid, L, I2, c2)
    assert (c2 == full["cnt"]).all() and (I2 == I).all()
    assert np.allclose(I2, full["I"], rtol=1e-12, atol=0)
    assert (np.isneginf(L) == np.isneginf(full["level"])).all()
    fin = np.isfinite(full["level"])
    assert np.abs(L[fin] - full["level"][fin]).max() < 1e-9
    # device-resident arrays work the same way; NULL counts install zeros
    torch = pytest.importorskip("torch")
    btrace.bt_set_result(tracer.ctx, sid, torch.from_numpy(I).cuda(), None)
    btrace.bt_read_levels(tracer.ctx, sid, L, I2, c2)
    assert (I2 == I).all() and (c2 == 0).all()
    btrace.bt_unload_scene(tracer.ctx, sid)


def test_microphone_blocks_gather_to_the_full_trace(tracer):
    # Section 3's microphone partitioning: three blocks of the microphones,
    # each traced against every source, concatenate to the one-trace result
    from paper_1912_03998_gb300 import shard
    w = synth.tiny_city(seed=9, level=4, max_order=4, n_sources=3)
    full = gpu_run(tracer, w)
    parts = []
    for r in range(3):
        lo, hi = shard.mic_block(len(w.mics), r, 3)
        parts.append(gpu_run(tracer, w.with_mics(w.mics[lo:hi])))
    cnt = np.concatenate([g["cnt"] for g in parts])
    I = np.concatenate([g["I"] for g in parts])
    assert (cnt == full["cnt"]).all()
    assert np.allclose(I, full["I"], rtol=1e-9, atol=0)


def test_cast_rays_through_shared_vertices_and_edges(tracer):
    # Rays straight down onto the shared vertices and edges of coplanar
    # triangle fans: every float32 test there is ambiguous, so the MIXED
    # search leaves the triangles to float64 after the traversal (up to 8 per
    # ray; a 12-triangle fan overflows that list and the rest are decided in
    # float32).  Every ray must still hit the plane at the right distance,
    # on a triangle of the fan that contains the point.
    from paper_1912_03998_gb300 import btrace
    verts, tris = [], []

    def fan(cx, cy, k, r):
        c = len(verts)
        verts.append((cx, cy, 10.0))
        for i in range(k):
            a = 2.0 * np.pi * i / k
            verts.append((cx + r * np.cos(a), cy + r * np.sin(a), 10.0))
        for i in range(k):
            tris.append((c, c + 1 + i, c + 1 + (i + 1) % k))
        return c

    centres = [fan(0.0, 0.0, 12, 5.0), fan(20.0, 0.0, 6, 5.0), fan(40.0, 0.0, 3, 5.0), fan(60.0, 0.0, 8, 5.0)]
    verts = np.asarray(verts, np.float32)
    tris = np.asarray(tris, np.int32)
    mat = np.zeros(len(tris), np.uint8)
    refl = np.full((1, 8), 0.9, np.float32)
    # targets: the fan centres (every triangle of the fan contains them) and
    # the midpoints of the spokes (the edges two triangles share); points on
    # the rim, the union's boundary, may round outside it and are left out
    pts = [verts[c, :2] for c in centres]
    for a, b, c in tris:
        pts.append(0.5 * (verts[a, :2] + verts[b, :2]))
    pts = np.asarray(pts, np.float32)
    o = np.column_stack([pts, np.full(len(pts), 50.0, np.float32)]).astype(np.float32)
    d = np.tile(np.asarray([[0.0, 0.0, -1.0]], np.float32), (len(pts), 1))
    sid = btrace.bt_load_scene(tracer.ctx, verts, tris, mat, refl)
    try:
        t, ids = btrace.bt_cast_rays(tracer.ctx, sid, o, d)
    finally:
        btrace.bt_unload_scene(tracer.ctx, sid)
    assert (ids >= 0).all(), np.nonzero(ids < 0)[0][:10]
    assert np.allclose(t, 40.0, atol=1e-4), t[np.abs(t - 40.0) > 1e-4][:10]
    # a centre is a tie of the whole fan, which goes to the lowest triangle
    # index wherever the fan fits the float64 list (3, 6 and 8 triangles)
    first = [0, 12, 18, 21]
    assert [int(i) for i in ids[1:4]] == first[1:4], ids[:4]
    assert 0 <= ids[0] < 12
    # the hit triangle contains the target point (edges inclusive, 1e-5 m)
    for p, i in zip(pts.astype(np.float64), ids):
        a, b, c = verts[tris[i]].astype(np.float64)[:, :2]
        def side(u, v, w):
            return (v[0] - u[0]) * (w[1] - u[1]) - (v[1] - u[1]) * (w[0] - u[0])
        s = [side(a, b, p), side(b, c, p), side(c, a, p)]
        assert min(s) >= -1e-5 * 5.0 or max(s) <= 1e-5 * 5.0, (p, i, s)


def test_cast_rays_through_coincident_stacks(tracer):
    # Two stacks of 2,048 identical triangles, one 5 m above the other: every
    # triangle of a stack has the same Morton code, so the LBVH splits them by
    # index alone, every box of the stack overlaps every ray, and the search
    # must visit the whole stack (the deepest hierarchies and longest stacks
    # a scene can give).  Rays from above hit the upper stack at exactly 40 m:
    # a tie of the whole stack, which MIXED decides in float64 up to the
    # length of its list and then in float32, so the hit is some triangle of
    # the upper stack.  Rays from below hit the lower stack.
    from paper_1912_03998_gb300 import btrace
    k = 2048
    tri = np.asarray([(-5.0, -5.0, 0.0), (5.0, -5.0, 0.0), (0.0, 6.0, 0.0)], np.float32)
    verts = np.concatenate([tri + np.float32([0.0, 0.0, 10.0])] * k + [tri + np.float32([0.0, 0.0, 5.0])] * k)
    tris = np.arange(len(verts), dtype=np.int32).reshape(-1, 3)
    mat = np.zeros(len(tris), np.uint8)
    refl = np.full((1, 8), 0.9, np.float32)
    rng = np.random.Generator(np.random.PCG64(31))
    n = 4096
    xy = np.column_stack([rng.uniform(-2.0, 2.0, n), rng.uniform(-3.0, 1.0, n)]).astype(np.float32)
    up = np.arange(n) % 2 == 0
    o = np.column_stack([xy, np.where(up, 50.0, -35.0)]).astype(np.float32)
    d = np.zeros((n, 3), np.float32)
    d[:, 2] = np.where(up, -1.0, 1.0)
    sid = btrace.bt_load_scene(tracer.ctx, verts, tris, mat, refl)
    try:
        t, ids = btrace.bt_cast_rays(tracer.ctx, sid, o, d)
    finally:
        btrace.bt_unload_scene(tracer.ctx, sid)
    assert (ids >= 0).all()
    assert np.allclose(t, 40.0, atol=1e-4), t[np.abs(t - 40.0) > 1e-4][:10]
    assert (ids[up] < k).all() and (ids[~up] >= k).all()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_directional_sources_match_oracle(tracer, oracle_mod, precision):
    # Section 2: a source's energy is split between the beams by its power in
    # each direction.  Three sources of the tiny city: two with seeded
    # patterns (one of them reused), one omnidirectional; levels against the
    # oracle.  The library and the oracle number the beams each in their own
    # order, so the oracle gets the gains of the beam with the same axis
    from paper_1912_03998_gb300 import btrace
    w = synth.tiny_city(seed=6)
    n_b = 20 * 4 ** w.level
    axes = btrace.bt_beam_axes(tracer.ctx, w.level)
    assert axes.shape == (n_b, 3) and np.allclose(np.linalg.norm(axes, axis=1), 1.0, atol=1e-6)
    dirs, _ = oracle_mod.beam_table(w.level)
    ax = dirs.sum(axis=1)
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    match = (axes.astype(np.float64) @ ax.T).argmax(axis=1)  # oracle beam of each library beam
    assert np.array_equal(np.sort(match), np.arange(n_b))
    assert np.abs(axes - ax[match]).max() < 1e-6
    rng = np.random.Generator(np.random.PCG64(21))
    # a smooth pattern (louder towards +x) and a rough one (random gains)
    patterns = np.stack([1.0 + 0.8 * axes[:, 0], rng.uniform(0.0, 2.0, n_b)]).astype(np.float32)
    src = np.concatenate([w.src, w.src[:1] + np.float32([15.0, -10.0, 0.0]), w.src[:1] + np.float32([-20.0, 5.0, 0.0])])
    power = np.concatenate([w.power, w.power[:1], w.power[:1] * 0.5]).astype(np.float32)
    pattern_of = np.array([0] * len(w.src) + [1, -1], np.int32)
    sid = btrace.bt_load_scene(tracer.ctx, w.scene.verts, w.scene.tris, w.scene.mat, w.scene.refl)
    try:
        btrace.bt_set_sources(tracer.ctx, sid, src, power, w.level)
        btrace.bt_set_microphones(tracer.ctx, sid, w.mics)
        btrace.bt_set_directivity(tracer.ctx, sid, patterns, pattern_of)
        prec = {"mixed": btrace.BT_PREC_MIXED, "fp64": btrace.BT_PREC_FP64}[precision]
        btrace.bt_trace(tracer.ctx, sid, tracer.params(w.max_order, precision=prec))
        L = np.empty((len(w.mics), power.shape[1]), np.float64)
        btrace.bt_read_levels(tracer.ctx, sid, L)
        # a bad pattern index is rejected and leaves the scene omnidirectional
        with pytest.raises(btrace.BtError):
            btrace.bt_set_directivity(tracer.ctx, sid, patterns, np.array([5] * len(src), np.int32))
    finally:
        btrace.bt_unload_scene(tracer.ctx, sid)
    oracle_patterns = np.empty_like(patterns)
    oracle_patterns[:, match] = patterns
    r = oracle_mod.trace(oracle_mod.Scene(w.scene), src, power, w.level, w.mics, w.max_order,
                         directivity=oracle_patterns, pattern_of=pattern_of)
    assert_parity(L, level_db(r["I"]), f"tiny city, directional sources, {precision}")


def test_directional_workload_through_the_tracer(tracer, oracle_mod):
    # directional sources given as functions of direction: the library and
    # the oracle each sample them at their own beams' axes
    w = synth.tiny_city(seed=8, n_sources=3)
    w.directivity = synth.Directivity([synth.cardioid((0.3, -1.0, 0.2), 0.9)], np.array([0, -1, 0], np.int32))
    g = gpu_run(tracer, w)
    r, L = oracle_levels(oracle_mod, w)
    assert_parity(g["level"], L, "tiny city, cardioid sources")
    assert (g["cnt"] == r["cnt"]).mean() >= 0.999
