"""Seeded synthetic inputs: cities of extruded buildings, point sources, microphone grids.

This module only builds geometry and random draws.  It holds none of the
beam-tracing arithmetic, so both the FP64 oracle and the CUDA path can take
their inputs from it.

The paper's experiment is a model of the Shinjuku district (2.5 km x 1.5 km,
towers up to ~200 m, a 4 m microphone grid, sources at major crossroads;
Section 4).  That model is not available, so the generators below produce
cities of the same shape:

* ``tiny_city``: 8x8 box buildings on 50 m blocks with 20 m streets, heights
  U(10, 60) m, 12 triangles per box plus a 2-triangle ground, one source at
  0.5 m in a street, 32x32 microphones at 1.5 m.
* ``district``: a 2 km x 2 km Manhattan grid (10 m roads on a 110 m pitch,
  18x18 blocks of 100 m), 5,000 convex extruded buildings (4-12-gon footprints,
  areas lognormal around 400 m^2, heights lognormal around 20 m clamped to
  [5, 200] m, walls split into bands of at most 15 m), sources on lane centres
  at 0.5 m with per-band power log-uniform in [0.01, 1] W, 500x500 microphones
  on a 4 m grid at 1.5 m.
* small scenes (free field, ground only, a single wall, 1-4 boxes) used by the
  closed-form and brute-force image-source checks.

Every generator takes a ``seed`` and draws from ``numpy.random.PCG64(seed)``.
All arrays are float32 / int32 / uint8 exactly as the C-ABI takes them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

#: octave band centre frequencies (Hz); the configurations use all eight
BANDS_HZ = (63, 125, 250, 500, 1000, 2000, 4000, 8000)
N_BANDS = len(BANDS_HZ)

#: material ids used by the generators
MAT_GROUND = 0
MAT_WALL = 1


@dataclass
class Scene:
    verts: np.ndarray  # float32 [n_v, 3], metres, z up, ground at z = 0
    tris: np.ndarray  # int32 [n_t, 3]
    mat: np.ndarray  # uint8 [n_t]
    refl: np.ndarray  # float32 [n_mat, n_bands], energy reflection coefficients
    info: dict = field(default_factory=dict)

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


@dataclass
class Directivity:
    """Directional sources as functions of direction, so that every tracer
    samples them at its own beams: patterns[k] maps unit directions [n, 3]
    to gains [n] (>= 0), pattern_of[s] is source s's pattern (-1 =
    omnidirectional)."""
    patterns: list
    pattern_of: np.ndarray  # int32 [n_s]

    def gains(self, axes) -> np.ndarray:
        """Gains [n_patterns, n_beams] float32 at the beam axes [n_beams, 3]."""
        axes = np.asarray(axes, np.float64)
        return np.stack([np.asarray(f(axes), np.float64) for f in self.patterns]).astype(np.float32)


def cardioid(axis, a: float = 1.0):
    """A pattern 1 + a (u . axis): louder towards `axis`; its mean over the
    sphere is 1 (the source keeps its total power), and it stays >= 0 for
    0 <= a <= 1."""
    ax = np.asarray(axis, np.float64)
    ax = ax / np.linalg.norm(ax)
    return lambda u: 1.0 + a * (np.asarray(u, np.float64) @ ax)


@dataclass
class Workload:
    name: str
    scene: Scene
    src: np.ndarray  # float32 [n_s, 3]
    power: np.ndarray  # float32 [n_s, n_bands], watts per band
    mics: np.ndarray  # float32 [n_m, 3]
    level: int  # icosahedron subdivision level L (20 * 4**L beams per source)
    max_order: int  # K: reflections 0..K are traced
    tiles: tuple = (1, 1)
    info: dict = field(default_factory=dict)
    directivity: Directivity = None  # None: every source omnidirectional

    def subset_sources(self, idx) -> "Workload":
        idx = np.asarray(idx)
        d = self.directivity
        if d is not None:
            d = Directivity(d.patterns, np.asarray(d.pattern_of)[idx].copy())
        return Workload(self.name + f"[{len(idx)} src]", self.scene, self.src[idx].copy(),
                        self.power[idx].copy(), self.mics, self.level, self.max_order,
                        self.tiles, dict(self.info), d)

    def with_mics(self, mics) -> "Workload":
        return Workload(self.name, self.scene, self.src, self.power,
                        np.ascontiguousarray(mics, dtype=np.float32), self.level,
                        self.max_order, self.tiles, dict(self.info), self.directivity)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def refl_table(ground=0.7, wall=0.9, n_bands=N_BANDS) -> np.ndarray:
    """[2, n_bands] energy coefficients: row 0 ground, row 1 walls and roofs."""
    t = np.empty((2, n_bands), dtype=np.float32)
    t[MAT_GROUND] = ground
    t[MAT_WALL] = wall
    return t


class _MeshBuilder:
    def __init__(self):
        self.v = []
        self.t = []
        self.m = []
        self.nv = 0

    def add_verts(self, pts) -> int:
        pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
        base = self.nv
        self.v.append(pts)
        self.nv += pts.shape[0]
        return base

    def add_tri(self, a, b, c, mat):
        self.t.append((a, b, c))
        self.m.append(mat)

    def scene(self, refl, info=None) -> Scene:
        v = np.concatenate(self.v).astype(np.float32) if self.v else np.zeros((0, 3), np.float32)
        t = np.asarray(self.t, dtype=np.int32).reshape(-1, 3)
        m = np.asarray(self.m, dtype=np.uint8)
        return Scene(v, t, m, refl, dict(info or {}))


def _add_box(mb: _MeshBuilder, x0, y0, x1, y1, h, floor=True):
    """Axis-aligned box, 12 triangles with floor (10 without), outward CCW."""
    b = mb.add_verts([(x0, y0, 0), (x1, y0, 0), (x1, y1, 0), (x0, y1, 0),
                      (x0, y0, h), (x1, y0, h), (x1, y1, h), (x0, y1, h)])
    quads = [(0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7), (4, 5, 6, 7)]
    if floor:
        quads.append((3, 2, 1, 0))
    for q in quads:
        mb.add_tri(b + q[0], b + q[1], b + q[2], MAT_WALL)
        mb.add_tri(b + q[0], b + q[2], b + q[3], MAT_WALL)


def _add_ground(mb: _MeshBuilder, x0, y0, x1, y1):
    b = mb.add_verts([(x0, y0, 0), (x1, y0, 0), (x1, y1, 0), (x0, y1, 0)])
    mb.add_tri(b + 0, b + 1, b + 2, MAT_GROUND)
    mb.add_tri(b + 0, b + 2, b + 3, MAT_GROUND)


def mic_grid(x0, y0, x1, y1, nx, ny, z=1.5) -> np.ndarray:
    """Cell-centred nx x ny grid over [x0,x1] x [y0,y1] at height z (row-major in y)."""
    xs = x0 + (np.arange(nx) + 0.5) * (x1 - x0) / nx
    ys = y0 + (np.arange(ny) + 0.5) * (y1 - y0) / ny
    gx, gy = np.meshgrid(xs, ys)
    m = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, z)], axis=1)
    return m.astype(np.float32)


# ---------------------------------------------------------------- tiny city
TINY_PITCH, TINY_BLOCK, TINY_MARGIN, TINY_N = 70.0, 50.0, 10.0, 8
GROUND_PAD = 500.0


def _tiny_footprints(n=TINY_N):
    fp = []
    for j in range(n):
        for i in range(n):
            x0 = TINY_MARGIN + TINY_PITCH * i
            y0 = TINY_MARGIN + TINY_PITCH * j
            fp.append((x0, y0, x0 + TINY_BLOCK, y0 + TINY_BLOCK))
    return fp


def _in_any_box(x, y, fps):
    for (x0, y0, x1, y1) in fps:
        if x0 <= x <= x1 and y0 <= y <= y1:
            return True
    return False


def _street_point(rng, fps, lo, hi):
    while True:
        x, y = rng.uniform(lo, hi, size=2)
        if not _in_any_box(x, y, fps):
            return x, y


def tiny_city(seed: int = 1, level: int = 4, max_order: int = 4, n_grid: int = 32,
              n_sources: int = 1, tiles=(1, 1)) -> Workload:
    """8x8 boxes on 50 m blocks, 20 m streets, heights U(10,60) m; 770 triangles."""
    rng = _rng(seed)
    side = TINY_PITCH * TINY_N  # 560 m
    fps = _tiny_footprints()
    heights = rng.uniform(10.0, 60.0, size=len(fps))
    mb = _MeshBuilder()
    for (x0, y0, x1, y1), h in zip(fps, heights):
        _add_box(mb, x0, y0, x1, y1, h, floor=True)
    _add_ground(mb, -GROUND_PAD, -GROUND_PAD, side + GROUND_PAD, side + GROUND_PAD)
    scene = mb.scene(refl_table(), {"kind": "tiny_city", "heights": heights})
    src = np.array([(*_street_point(rng, fps, 0.0, side), 0.5) for _ in range(n_sources)],
                   dtype=np.float32)
    power = np.ones((n_sources, N_BANDS), dtype=np.float32)
    mics = mic_grid(0.0, 0.0, side, side, n_grid, n_grid, 1.5)
    return Workload("tiny_city", scene, src, power, mics, level, max_order, tuple(tiles),
                    {"seed": seed})


# ---------------------------------------------------------------- small scenes
def free_field(seed: int = 1, level: int = 2, n_mics: int = 256) -> Workload:
    """No geometry at all: one source, microphones scattered in a 200 m cube."""
    rng = _rng(seed)
    scene = _MeshBuilder().scene(refl_table(), {"kind": "free_field"})
    src = np.array([[0.3, -0.7, 0.5]], dtype=np.float32)
    mics = rng.uniform(-100.0, 100.0, size=(n_mics, 3)).astype(np.float32)
    power = rng.uniform(0.1, 2.0, size=(1, N_BANDS)).astype(np.float32)
    return Workload("free_field", scene, src, power, mics, level, 3, (1, 1), {"seed": seed})


def ground_only(seed: int = 1, level: int = 4, n_grid: int = 24, half=200.0,
                ground=0.7) -> Workload:
    """Source at 0.5 m over a 2-triangle ground; microphones at 1.5 m."""
    rng = _rng(seed)
    mb = _MeshBuilder()
    _add_ground(mb, -half - GROUND_PAD, -half - GROUND_PAD, half + GROUND_PAD, half + GROUND_PAD)
    scene = mb.scene(refl_table(ground=ground), {"kind": "ground_only"})
    sx, sy = rng.uniform(-5.0, 5.0, size=2)
    src = np.array([[sx, sy, 0.5]], dtype=np.float32)
    mics = mic_grid(-half, -half, half, half, n_grid, n_grid, 1.5)
    power = np.ones((1, N_BANDS), dtype=np.float32)
    return Workload("ground_only", scene, src, power, mics, level, 3, (1, 1), {"seed": seed})


def single_wall(seed: int = 1, level: int = 4, n_grid: int = 24, wall=0.9) -> Workload:
    """A vertical 2-triangle wall x = 0, 2000 m wide and 1000 m tall, no ground.

    Source and microphones sit on the x < 0 side, well inside the wall's extent.
    """
    rng = _rng(seed)
    mb = _MeshBuilder()
    b = mb.add_verts([(0, -1000, -500), (0, 1000, -500), (0, 1000, 500), (0, -1000, 500)])
    mb.add_tri(b, b + 2, b + 1, MAT_WALL)  # normal -x, toward the source side
    mb.add_tri(b, b + 3, b + 2, MAT_WALL)
    scene = mb.scene(refl_table(wall=wall), {"kind": "single_wall"})
    src = np.array([[-rng.uniform(2.0, 6.0), rng.uniform(-5, 5), rng.uniform(-5, 5)]],
                   dtype=np.float32)
    g = mic_grid(-100.0, -100.0, 100.0, 100.0, n_grid, n_grid, 0.0)
    mics = np.stack([-(g[:, 0] + 100.0) / 2.0 - 0.5, g[:, 1], g[:, 0] * 0.5], axis=1)
    power = np.ones((1, N_BANDS), dtype=np.float32)
    return Workload("single_wall", scene, src, power, mics.astype(np.float32), level, 3, (1, 1),
                    {"seed": seed})


def boxes(n_boxes: int, seed: int = 1, level: int = 4, max_order: int = 3, n_grid: int = 16,
          floor=True) -> Workload:
    """The first n_boxes (1-4) boxes of the tiny-city pattern (2x2), over a padded ground."""
    assert 1 <= n_boxes <= 4
    rng = _rng(seed)
    fps = _tiny_footprints(2)[:n_boxes]
    heights = rng.uniform(10.0, 60.0, size=len(fps))
    mb = _MeshBuilder()
    for (x0, y0, x1, y1), h in zip(fps, heights):
        _add_box(mb, x0, y0, x1, y1, h, floor=floor)
    side = 2 * TINY_PITCH
    _add_ground(mb, -GROUND_PAD, -GROUND_PAD, side + GROUND_PAD, side + GROUND_PAD)
    scene = mb.scene(refl_table(), {"kind": f"boxes{n_boxes}", "heights": heights})
    src = np.array([(*_street_point(rng, _tiny_footprints(2), 0.0, side), 0.5)],
                   dtype=np.float32)
    mics = mic_grid(0.0, 0.0, side, side, n_grid, n_grid, 1.5)
    power = np.ones((1, N_BANDS), dtype=np.float32)
    return Workload(f"boxes{n_boxes}", scene, src, power, mics, level, max_order, (1, 1),
                    {"seed": seed})


# ---------------------------------------------------------------- district
DIST_PITCH, DIST_ROAD, DIST_NBLK = 110.0, 10.0, 18
DIST_EXTENT = DIST_PITCH * DIST_NBLK + DIST_ROAD  # 1990 m of roads and blocks
DIST_MIC_SIDE = 2000.0


def volume_mics(n_side: int = 500, n_heights: int = 55, pitch: float = 4.0, z0: float = 1.5) -> np.ndarray:
    """A regular 3D microphone grid over the district (the paper's receivers
    fill the city's volume on a 4 m grid): n_side x n_side cell-centred
    columns, n_heights levels from z0 up in steps of `pitch`; 500 x 500 x 55
    = 13.75 M points up to 217.5 m, above the tallest building."""
    return np.concatenate([mic_grid(0.0, 0.0, DIST_MIC_SIDE, DIST_MIC_SIDE, n_side, n_side, z0 + pitch * k)
                           for k in range(n_heights)]).astype(np.float32)


def _kd_lots(rng, x0, y0, x1, y1, depth):
    if depth == 0:
        return [(x0, y0, x1, y1)]
    f = rng.uniform(0.35, 0.65)
    if (x1 - x0) >= (y1 - y0):
        xm = x0 + f * (x1 - x0)
        return _kd_lots(rng, x0, y0, xm, y1, depth - 1) + _kd_lots(rng, xm, y0, x1, y1, depth - 1)
    ym = y0 + f * (y1 - y0)
    return _kd_lots(rng, x0, y0, x1, ym, depth - 1) + _kd_lots(rng, x0, ym, x1, y1, depth - 1)


def _polygon_area(p):
    x, y = p[:, 0], p[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def _footprint_shape(rng, lot):
    """Convex n-gon (n ~ U{4..12}) with its vertices on the lot's inscribed
    superellipse |x/a|^4 + |y/b|^4 = 1 (which fills 93 % of the lot), CCW and
    centred on the origin, and the lot's centre."""
    x0, y0, x1, y1 = lot
    a, b = 0.5 * (x1 - x0), 0.5 * (y1 - y0)
    n = int(rng.integers(4, 13))
    th0 = rng.uniform(0.0, 2.0 * math.pi)
    th = th0 + 2.0 * math.pi * (np.arange(n) + rng.uniform(-0.3, 0.3, size=n)) / n
    c, sn = np.cos(th), np.sin(th)
    unit = np.stack([a * np.sign(c) * np.sqrt(np.abs(c)), b * np.sign(sn) * np.sqrt(np.abs(sn))], axis=1)
    return unit, np.array([0.5 * (x0 + x1), 0.5 * (y0 + y1)])


# largest scale of a footprint's shape within its lot (a gap of at least 2.5 %
# of the lot's side to every neighbour)
FOOTPRINT_MAX_SCALE = 0.95


def _footprint(unit, centre, target):
    """The shape scaled to area `target`, at most FOOTPRINT_MAX_SCALE."""
    s = min(math.sqrt(target / _polygon_area(unit)), FOOTPRINT_MAX_SCALE)
    pts = unit * s + centre
    return pts, _polygon_area(pts)


def _lane_sources(rng, n_sources, log10_p_lo, log10_p_hi):
    """Car sources on lane centres of the district road grid (two 5 m lanes
    per 10 m road, centres at +-2.5 m) at 0.5 m, with per-band power
    log-uniform in [10^lo, 10^hi] W."""
    horiz = rng.random(n_sources) < 0.5
    road = rng.integers(0, DIST_NBLK + 1, size=n_sources)
    lane = np.where(rng.random(n_sources) < 0.5, -2.5, 2.5)
    along = rng.uniform(0.0, DIST_EXTENT, size=n_sources)
    across = DIST_PITCH * road + 0.5 * DIST_ROAD + lane
    sx = np.where(horiz, along, across)
    sy = np.where(horiz, across, along)
    src = np.stack([sx, sy, np.full(n_sources, 0.5)], axis=1).astype(np.float32)
    power = (10.0 ** rng.uniform(log10_p_lo, log10_p_hi, size=(n_sources, N_BANDS))).astype(np.float32)
    return src, power


def district(seed: int = 2, n_buildings: int = 5000, n_sources: int = 1000, level: int = 5,
             max_order: int = 6, n_mic_side: int = 500, tiles=(4, 4), band_h=15.0) -> Workload:
    """2 km x 2 km district of extruded convex buildings on a Manhattan road grid."""
    rng = _rng(seed)
    lots = []
    for bj in range(DIST_NBLK):
        for bi in range(DIST_NBLK):
            x0 = DIST_PITCH * bi + DIST_ROAD
            y0 = DIST_PITCH * bj + DIST_ROAD
            lots += _kd_lots(rng, x0, y0, x0 + DIST_PITCH - DIST_ROAD, y0 + DIST_PITCH - DIST_ROAD, 4)
    pick = rng.choice(len(lots), size=min(n_buildings, len(lots)), replace=False)
    pick.sort()
    # footprint areas lognormal(ln 400 m^2, 0.6), the larger areas on the
    # footprint shapes with room for more (matched by rank), so that the lots
    # do not cut the distribution's upper half
    shapes = [_footprint_shape(rng, lots[li]) for li in pick]
    room = np.array([_polygon_area(u) for u, _ in shapes]) * FOOTPRINT_MAX_SCALE ** 2
    targets = np.sort(rng.lognormal(math.log(400.0), 0.6, size=len(pick)))
    target_of = np.empty(len(pick))
    target_of[np.argsort(room, kind="stable")] = targets
    mb = _MeshBuilder()
    areas, heights, ngons = [], [], []
    for (unit, centre), target in zip(shapes, target_of):
        pts, area = _footprint(unit, centre, float(target))
        h = float(np.clip(rng.lognormal(math.log(20.0), 0.66), 5.0, 200.0))
        n = pts.shape[0]
        nb = max(1, int(math.ceil(h / band_h)))
        zs = np.linspace(0.0, h, nb + 1)
        ring = np.array([(p[0], p[1], z) for z in zs for p in pts])
        base = mb.add_verts(ring)
        for k in range(nb):
            for e in range(n):
                a0 = base + k * n + e
                a1 = base + k * n + (e + 1) % n
                b1 = base + (k + 1) * n + (e + 1) % n
                b0 = base + (k + 1) * n + e
                mb.add_tri(a0, a1, b1, MAT_WALL)
                mb.add_tri(a0, b1, b0, MAT_WALL)
        top = base + nb * n
        for e in range(1, n - 1):
            mb.add_tri(top, top + e, top + e + 1, MAT_WALL)
        areas.append(area)
        heights.append(h)
        ngons.append(n)
    _add_ground(mb, -GROUND_PAD, -GROUND_PAD, DIST_EXTENT + GROUND_PAD, DIST_EXTENT + GROUND_PAD)
    info = {"kind": "district", "n_buildings": len(pick),
            "area_quantiles": np.quantile(areas, [0.1, 0.5, 0.9]).tolist(),
            "height_quantiles": np.quantile(heights, [0.1, 0.5, 0.9, 0.999]).tolist(),
            "height_max": float(np.max(heights)), "ngon_mean": float(np.mean(ngons))}
    scene = mb.scene(refl_table(), info)
    src, power = _lane_sources(rng, n_sources, -2.0, 0.0)
    mics = mic_grid(0.0, 0.0, DIST_MIC_SIDE, DIST_MIC_SIDE, n_mic_side, n_mic_side, 1.5)
    return Workload("district", scene, src, power, mics, level, max_order, tuple(tiles),
                    {"seed": seed, **info})


def batch_cities(seed: int = 4, n: int = 64):
    """Cities of uneven size for batched tracing: each drawn like the district
    (same footprint, height and source distributions on the same 2 km road
    grid) with 100-5,000 buildings and 1-1,000 sources (both log-uniform),
    icosahedron level 3-6 (1,280-81,920 beams per source) and reflection order
    2-8 (both uniform), and 1k-250k microphones (log-uniform) on a square grid
    at 1.5 m."""
    rng = _rng(seed)
    out = []
    for i in range(n):
        n_b = int(round(math.exp(rng.uniform(math.log(100), math.log(5000)))))
        n_s = int(round(math.exp(rng.uniform(math.log(1), math.log(1000)))))
        level = int(rng.integers(3, 7))
        k = int(rng.integers(2, 9))
        n_m = math.exp(rng.uniform(math.log(1000), math.log(250000)))
        side = max(2, int(round(math.sqrt(n_m))))
        w = district(seed=seed * 1000 + i, n_buildings=n_b, n_sources=n_s, level=level, max_order=k,
                     n_mic_side=side, tiles=(1, 1))
        w.name = f"city{i}"
        out.append(w)
    return out


def serving_cities(seed: int = 5, n: int = 8):
    """Resident cities for the serving loop: drawn like the district with
    500-5,000 buildings (log-uniform); their sources and microphones come with
    the queries."""
    rng = _rng(seed)
    out = []
    for i in range(n):
        n_b = int(round(math.exp(rng.uniform(math.log(500), math.log(5000)))))
        w = district(seed=seed * 1000 + i, n_buildings=n_b, n_sources=1, level=4, max_order=3, n_mic_side=2,
                     tiles=(1, 1))
        w.name = f"resident{i}"
        out.append(w)
    return out


@dataclass
class Query:
    """One traffic-noise query against a resident city."""
    arrival_s: float
    city: int
    src: np.ndarray
    power: np.ndarray
    mics: np.ndarray
    level: int
    max_order: int
    directivity: Directivity = None  # None: every source omnidirectional


def serving_queries(seed: int, n_queries: int, n_cities: int, rate_qps: float, level: int = 4,
                    max_sources: int = 2000, max_mics: int = 250000):
    """A Poisson stream of queries: arrival gaps exponential with mean
    1/rate; a uniformly chosen city; 1-max_sources car sources (log-uniform)
    with per-band power log-uniform 0.001-1 W; 1k-max_mics microphones
    (log-uniform) on a 4 m grid at 1.5 m over a square window centred on one
    of the query's sources (kept inside the city); reflection order 3-6
    (uniform)."""
    rng = _rng(seed)
    t = 0.0
    out = []
    for _ in range(n_queries):
        t += float(rng.exponential(1.0 / rate_qps))
        city = int(rng.integers(0, n_cities))
        n_s = int(round(math.exp(rng.uniform(0.0, math.log(max_sources)))))
        src, power = _lane_sources(rng, n_s, -3.0, 0.0)
        n_m = math.exp(rng.uniform(math.log(1000), math.log(max_mics)))
        side = max(2, int(round(math.sqrt(n_m))))
        span = min(DIST_MIC_SIDE, 4.0 * side)
        cx, cy = src[int(rng.integers(0, n_s)), :2]
        x0 = float(np.clip(cx - 0.5 * span, 0.0, DIST_MIC_SIDE - span))
        y0 = float(np.clip(cy - 0.5 * span, 0.0, DIST_MIC_SIDE - span))
        mics = mic_grid(x0, y0, x0 + span, y0 + span, side, side, 1.5)
        out.append(Query(t, city, src, power, mics, level, int(rng.integers(3, 7))))
    return out
