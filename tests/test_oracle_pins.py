"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names the fact it checks: a closed form (free field, ground plane,
one wall), an independent brute-force image-source enumeration (Section 2's
image-source method, in oracle/isrc_bruteforce.c), geometric properties of
the beam table, or invariants of the method (tile split, thread count,
order-wise energy).  The paper prints no acoustic values, so nothing here is
a stored paper number.
"""
from collections import Counter, defaultdict

import numpy as np
import pytest

from paper_1912_03998_gb300 import synth

F32_07 = float(np.float32(0.7))
F32_09 = float(np.float32(0.9))


# ------------------------------------------------------------------ beam table
@pytest.mark.parametrize("level", [0, 1, 2, 3, 4, 5])
def test_beam_count_and_solid_angles(oracle_mod, level):
    dirs, omega = oracle_mod.beam_table(level)
    assert dirs.shape == (20 * 4 ** level, 3, 3)
    assert np.allclose(np.linalg.norm(dirs, axis=2), 1.0, atol=1e-15)
    assert (omega > 0).all()
    # the faces tile the sphere: solid angles add up to 4 pi
    assert abs(omega.sum() / (4 * np.pi) - 1.0) < 1e-12
    # counter-clockwise seen from outside: det[d0, d1, d2] > 0
    det = np.einsum("ni,ni->n", dirs[:, 0], np.cross(dirs[:, 1], dirs[:, 2]))
    assert (det > 0).all()


def test_base_icosahedron_faces_are_equal(oracle_mod):
    # level 0 is the regular icosahedron: 20 congruent faces of 4 pi / 20 each,
    # edge angle arccos(1/sqrt(5)) between neighbouring vertices
    dirs, omega = oracle_mod.beam_table(0)
    assert np.allclose(omega, 4 * np.pi / 20, rtol=1e-13)
    cosines = np.einsum("nij,nkj->nik", dirs, dirs)[:, [0, 1, 2], [1, 2, 0]]
    assert np.allclose(cosines, 1 / np.sqrt(5), atol=1e-14)
    # 12 distinct vertices, each shared by 5 faces
    v = np.round(dirs.reshape(-1, 3), 12)
    uniq, counts = np.unique(v, axis=0, return_counts=True)
    assert len(uniq) == 12 and (counts == 5).all()


def test_beams_partition_directions(oracle_mod):
    # every direction lies in exactly one cone (up to measure-zero ties)
    dirs, _ = oracle_mod.beam_table(3)
    rng = np.random.Generator(np.random.PCG64(7))
    u = rng.normal(size=(20000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    n = np.cross(dirs, np.roll(dirs, -1, axis=1))  # [N,3,3] edge-plane normals
    e = np.einsum("nji,mi->mnj", n, u)  # [M,N,3]
    inside = (e >= 0).all(axis=2)
    assert (inside.sum(axis=1) == 1).all()


# ------------------------------------------------------------------ closed forms
@pytest.mark.parametrize("level", [0, 1, 2, 3])
@pytest.mark.parametrize("alpha_db", [0.0, 0.013])
def test_free_field_closed_form(oracle_mod, level, alpha_db):
    # no geometry: intensity W 10^(-alpha r/10) / (4 pi r^2) at every microphone,
    # one path each, whatever the beam count
    w = synth.free_field(seed=3, level=level)
    alpha = alpha_db * (1 + np.arange(synth.N_BANDS))
    r = oracle_mod.trace_workload(w, alpha=alpha)
    rr = np.linalg.norm(w.mics.astype(np.float64) - w.src[0].astype(np.float64), axis=1)
    expect = (w.power[0].astype(np.float64)[None, :] * 10.0 ** (-alpha[None, :] * rr[:, None] / 10)
              / (4 * np.pi * rr[:, None] ** 2))
    assert (r["cnt"] == 1).all()
    assert np.abs(r["I"] / expect - 1).max() < 1e-12
    L = oracle_mod.levels(r["I"])
    assert np.abs(L - 10 * np.log10(expect / 1e-12)).max() < 1e-9


@pytest.mark.parametrize("level", [1, 3])
def test_directional_free_field_closed_form(oracle_mod, level):
    # Section 2: a source's energy is split between the beams by its power in
    # each direction.  With no geometry a microphone receives only the beam
    # whose cone holds its direction from the source, so its intensity is
    # that beam's gain times W / (4 pi r^2); the beam is found here by the
    # cone-membership test on the beam table itself, not by the trace
    w = synth.free_field(seed=5, level=level, n_mics=400)
    dirs, _ = oracle_mod.beam_table(level)
    n_b = len(dirs)
    rng = np.random.Generator(np.random.PCG64(11))
    gains = rng.uniform(0.0, 3.0, size=(2, n_b)).astype(np.float32)
    src = np.repeat(w.src, 3, axis=0)
    power = np.repeat(w.power, 3, axis=0)
    pattern_of = np.array([0, -1, 1], np.int32)  # two patterns and one omnidirectional copy
    sc = oracle_mod.Scene(w.scene)
    r = oracle_mod.trace(sc, src, power, level, w.mics, w.max_order, directivity=gains, pattern_of=pattern_of)
    v = w.mics.astype(np.float64) - w.src[0].astype(np.float64)
    rr = np.linalg.norm(v, axis=1)
    u = v / rr[:, None]
    n = np.cross(dirs, np.roll(dirs, -1, axis=1))
    inside = (np.einsum("nji,mi->mnj", n, u) >= 0).all(axis=2)
    assert (inside.sum(axis=1) == 1).all()
    beam = inside.argmax(axis=1)
    g = 1.0 + gains[0, beam].astype(np.float64) + gains[1, beam].astype(np.float64)
    expect = g[:, None] * w.power[0].astype(np.float64)[None, :] / (4 * np.pi * rr[:, None] ** 2)
    assert (r["cnt"] == 3).all()
    assert np.abs(r["I"] / expect - 1).max() < 1e-12


def test_directivity_of_ones_is_omnidirectional(oracle_mod):
    # a pattern of unit gains leaves every result exactly as without one
    w = synth.tiny_city(seed=3)
    n_b = 20 * 4 ** w.level
    sc = oracle_mod.Scene(w.scene)
    a = oracle_mod.trace(sc, w.src, w.power, w.level, w.mics, w.max_order)
    b = oracle_mod.trace(sc, w.src, w.power, w.level, w.mics, w.max_order,
                         directivity=np.ones((1, n_b), np.float32), pattern_of=np.zeros(len(w.src), np.int32))
    assert np.array_equal(a["I"], b["I"]) and np.array_equal(a["cnt"], b["cnt"])


def _max_beam_diameter(oracle_mod, level):
    dirs, _ = oracle_mod.beam_table(level)
    c = np.einsum("nij,nkj->nik", dirs, dirs)
    return float(np.arccos(np.clip(c.min(axis=(1, 2)), -1, 1)).max())


def test_ground_plane_closed_form(oracle_mod):
    # one source over a reflecting ground: direct path plus the ground image
    # (x, y, -h_s) with energy coefficient 0.7.  Exact for microphones whose
    # image direction lies more than one beam diameter below the horizon;
    # every other microphone gets either both terms or the direct term alone.
    full_fraction = []
    for level in (3, 4, 5, 6):
        w = synth.ground_only(seed=1, level=level)
        r = oracle_mod.trace_workload(w)
        s = w.src[0].astype(np.float64)
        m = w.mics.astype(np.float64)
        img = s * np.array([1, 1, -1])
        r1 = np.linalg.norm(m - s, axis=1)
        r2 = np.linalg.norm(m - img, axis=1)
        direct = 1 / (4 * np.pi * r1 ** 2)
        image = F32_07 / (4 * np.pi * r2 ** 2)
        I = r["I"]
        both = (np.abs(I / (direct + image)[:, None] - 1) < 1e-12).all(axis=1)
        alone = (np.abs(I / direct[:, None] - 1) < 1e-12).all(axis=1)
        assert (both | alone).all()
        assert ((r["cnt"] == 2) == both).all() and ((r["cnt"] == 1) == alone).all()
        rho = np.hypot(m[:, 0] - s[0], m[:, 1] - s[1])
        margin = np.arctan2(m[:, 2] - img[2], rho) > _max_beam_diameter(oracle_mod, level)
        assert margin.sum() > 0 and both[margin].all()
        full_fraction.append(both.mean())
    # smaller beams resolve the image path for more microphones
    assert all(a < b for a, b in zip(full_fraction, full_fraction[1:]))


def test_directional_ground_plane_closed_form(oracle_mod):
    # the ground-plane closed form with a directional source: the direct term
    # carries the gain of the beam holding the direction to the microphone,
    # the image term the gain of the beam holding the direction to the
    # reflection point (the image direction mirrored in the ground)
    for level in (4, 5):
        w = synth.ground_only(seed=4, level=level, half=20.0)
        dirs, _ = oracle_mod.beam_table(level)
        gains = np.random.Generator(np.random.PCG64(level)).uniform(0.2, 2.0, (1, len(dirs))).astype(np.float32)
        r = oracle_mod.trace(oracle_mod.Scene(w.scene), w.src, w.power, level, w.mics, w.max_order,
                             directivity=gains, pattern_of=np.zeros(1, np.int32))
        s = w.src[0].astype(np.float64)
        m = w.mics.astype(np.float64)
        img = s * np.array([1, 1, -1])
        n = np.cross(dirs, np.roll(dirs, -1, axis=1))

        def beam_of(v):
            u = v / np.linalg.norm(v, axis=1, keepdims=True)
            inside = (np.einsum("nji,mi->mnj", n, u) >= 0).all(axis=2)
            assert (inside.sum(axis=1) >= 1).all()
            return inside.argmax(axis=1)

        g1 = gains[0, beam_of(m - s)].astype(np.float64)
        g2 = gains[0, beam_of((m - img) * np.array([1, 1, -1]))].astype(np.float64)
        r1 = np.linalg.norm(m - s, axis=1)
        r2 = np.linalg.norm(m - img, axis=1)
        expect = g1 / (4 * np.pi * r1 ** 2) + F32_07 * g2 / (4 * np.pi * r2 ** 2)
        rho = np.hypot(m[:, 0] - s[0], m[:, 1] - s[1])
        margin = np.arctan2(m[:, 2] - img[2], rho) > _max_beam_diameter(oracle_mod, level)
        assert margin.sum() > 10
        # ties (a direction on a shared cone edge) are measure-zero here
        got = r["I"][margin] / expect[margin][:, None]
        assert np.abs(got - 1).max() < 1e-12


def test_single_wall_closed_form(oracle_mod):
    # a vertical wall at x = 0 (energy coefficient 0.9): direct plus the image
    # mirrored to (-x, y, z); exact for microphones whose image direction lies
    # more than one beam diameter inside the wall's angular extent
    w = synth.single_wall(seed=2, level=5)
    r = oracle_mod.trace_workload(w)
    s = w.src[0].astype(np.float64)
    m = w.mics.astype(np.float64)
    img = s * np.array([-1, 1, 1])
    r1 = np.linalg.norm(m - s, axis=1)
    r2 = np.linalg.norm(m - img, axis=1)
    direct = 1 / (4 * np.pi * r1 ** 2)
    image = F32_09 / (4 * np.pi * r2 ** 2)
    both = (np.abs(r["I"] / (direct + image)[:, None] - 1) < 1e-12).all(axis=1)
    alone = (np.abs(r["I"] / direct[:, None] - 1) < 1e-12).all(axis=1)
    assert (both | alone).all()
    # the wall spans |y| <= 1000, |z| <= 500 and every microphone is within 100 m
    # of it, so every image direction is far inside the wall: all get both
    assert both.all() and (r["cnt"] == 2).all()


# ------------------------------------------------------ brute-force image sources
def _paths(log, n):
    P = defaultdict(list)
    for m, o, d in zip(log["mic"], log["order"], log["d"]):
        P[int(m)].append((int(o), round(float(d), 6)))
    return [Counter(P[i]) for i in range(n)]


@pytest.mark.parametrize("n_boxes,max_order", [(1, 4), (2, 4), (4, 3)])
def test_image_source_bruteforce_agreement(oracle_mod, n_boxes, max_order):
    # Every valid image-source path of order <= K (Section 2's image-source
    # method, enumerated by brute force) must appear in the beam oracle with
    # the same order and length, and vice versa, except near beam boundaries
    # where the hybrid method's axis-ray approximation decides.  The mismatch
    # must shrink as beams get smaller and be under 2% of paths at L = 6.
    w3 = synth.boxes(n_boxes, seed=5, level=3, max_order=max_order)
    ref = oracle_mod.isrc(w3.scene, w3.src[0], w3.power[0], w3.mics, max_order, log_cap=10 ** 6)
    assert ref["log"]["full"]
    Pr = _paths(ref["log"], len(w3.mics))
    total = sum(sum(p.values()) for p in Pr)
    assert total > 50
    bad = {}
    for level in (4, 6):
        w = synth.boxes(n_boxes, seed=5, level=level, max_order=max_order)
        r = oracle_mod.trace_workload(w, log_cap=10 ** 6)
        assert r["log"]["full"]
        P = _paths(r["log"], len(w.mics))
        mism = sum(sum(((P[i] - Pr[i]) + (Pr[i] - P[i])).values()) for i in range(len(P)))
        bad[level] = mism
        # microphones whose path sets agree also agree in intensity per band
        same = np.array([P[i] == Pr[i] for i in range(len(P))])
        assert np.allclose(r["I"][same], ref["I"][same], rtol=1e-9, atol=0)
    assert bad[6] <= bad[4]
    assert bad[6] <= 0.02 * total


def test_image_source_bruteforce_air_attenuation(oracle_mod):
    # same comparison with band-dependent air damping (Section 2): matched
    # microphones must agree band by band
    alpha = np.linspace(0.0, 0.05, synth.N_BANDS)
    w = synth.boxes(1, seed=5, level=6, max_order=2)
    ref = oracle_mod.isrc(w.scene, w.src[0], w.power[0], w.mics, 2, alpha=alpha)
    r = oracle_mod.trace_workload(w, alpha=alpha)
    same = r["cnt"] == ref["cnt"]
    assert same.mean() > 0.95
    close = np.isclose(r["I"], ref["I"], rtol=1e-9, atol=0).all(axis=1)
    assert close[same].mean() > 0.98
    # damping makes the high bands strictly weaker wherever there is a path
    hit = r["cnt"] > 0
    assert (np.diff(r["I"][hit], axis=1) < 0).all()


# ------------------------------------------------------------------ invariants
def test_hit_search_modes_agree(oracle_mod):
    # BVH and tiled searches must return exactly the brute-force closest hit
    w = synth.tiny_city(seed=4)
    rng = np.random.Generator(np.random.PCG64(11))
    n = 3000
    o = np.column_stack([rng.uniform(-50, 610, n), rng.uniform(-50, 610, n), rng.uniform(0.1, 70, n)])
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ref_t, ref_id = oracle_mod.cast_rays(oracle_mod.Scene(w.scene), o, d, mode=oracle_mod.HIT_BRUTE)
    assert (ref_id >= 0).mean() > 0.3
    for tiles, mode in (((1, 1), oracle_mod.HIT_BVH), ((4, 4), oracle_mod.HIT_TILED),
                        ((3, 5), oracle_mod.HIT_TILED)):
        t, ids = oracle_mod.cast_rays(oracle_mod.Scene(w.scene, tiles), o, d, mode=mode)
        assert (ids == ref_id).all()
        assert np.array_equal(t[ids >= 0], ref_t[ref_id >= 0])


def test_tile_split_invariance(oracle_mod):
    # Section 3: splitting geometry into sub-domains with beam hand-off must not
    # change any result
    w = synth.tiny_city(seed=1, level=4, max_order=4)
    base = oracle_mod.trace_workload(w)
    for tiles in ((2, 2), (4, 4), (3, 5)):
        r = oracle_mod.trace_workload(w, tiles=tiles)
        assert (r["cnt"] == base["cnt"]).all()
        assert np.allclose(r["I"], base["I"], rtol=1e-12, atol=0)
        assert r["stats"]["handoffs"] > 0
        assert r["stats"]["segments"] == base["stats"]["segments"]


def test_microphone_culling_is_exact(oracle_mod):
    # the cell-grid culling only skips microphones that fail the exact test
    w = synth.tiny_city(seed=2, level=3, max_order=3)
    rng = np.random.Generator(np.random.PCG64(5))
    mics = np.column_stack([rng.uniform(-20, 580, 3000), rng.uniform(-20, 580, 3000),
                            rng.uniform(0.0, 80.0, 3000)]).astype(np.float32)
    for ww in (w, w.with_mics(mics)):
        a = oracle_mod.trace_workload(ww, mic_mode=oracle_mod.MIC_BRUTE)
        b = oracle_mod.trace_workload(ww, mic_mode=oracle_mod.MIC_GRID)
        assert (a["cnt"] == b["cnt"]).all() and np.array_equal(a["I"], b["I"])
        assert a["cnt"].sum() > 100


def test_order_energy_invariants(oracle_mod):
    # the power entering order 0 is the total source power (solid angles sum to
    # 4 pi); each reflection keeps at most the largest coefficient (0.9)
    w = synth.tiny_city(seed=3, level=4, max_order=5, n_sources=2)
    r = oracle_mod.trace_workload(w)
    p = r["stats"]["order_power"]
    assert abs(p[0] / w.power.astype(np.float64).sum() - 1) < 1e-12
    assert all(p[k] <= F32_09 * p[k - 1] * (1 + 1e-12) for k in range(1, len(p)))
    assert p[-1] > 0


def test_thread_count_invariance(oracle_mod):
    w = synth.tiny_city(seed=3, level=3, max_order=3, n_sources=5)
    a = oracle_mod.trace_workload(w, n_threads=1)
    b = oracle_mod.trace_workload(w, n_threads=3)
    assert (a["cnt"] == b["cnt"]).all()
    assert np.allclose(a["I"], b["I"], rtol=1e-12, atol=0)


def test_energy_threshold_prunes_only_weak_beams(oracle_mod):
    w = synth.tiny_city(seed=3, level=3, max_order=6)
    a = oracle_mod.trace_workload(w)
    # the weakest product after at most 6 reflections is 0.7^6 = 0.118 (1 W
    # sources): a threshold of 0.1 W deletes nothing
    b = oracle_mod.trace_workload(w, energy_threshold=0.1)
    assert np.array_equal(a["I"], b["I"])
    # 0.75 W deletes every beam after one ground or three wall reflections
    c = oracle_mod.trace_workload(w, energy_threshold=0.75)
    assert c["stats"]["segments"] < a["stats"]["segments"]
    assert (c["I"] <= a["I"] * (1 + 1e-12)).all()


def test_levels_readout(oracle_mod):
    I = np.array([1e-12, 1.0, 0.0, 2e-12])
    L = oracle_mod.levels(I)
    assert L[0] == 0.0 and abs(L[1] - 120.0) < 1e-12 and L[2] == -np.inf
    assert abs(L[3] - 10 * np.log10(2)) < 1e-12
