"""ctypes front end of the FP64 CPU oracle (btrace_oracle.c, isrc_bruteforce.c).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module.  The CUDA library never
does, and this module imports nothing from the CUDA library: the two meet only
at the seeded inputs of ``paper_1912_03998_gb300.synth``.

Each function cites the step of the paper's Section 2 (hybrid beam/ray method)
or Section 3 (sub-domains) that it follows; the C sources hold the details.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = [os.path.join(HERE, "btrace_oracle.c"), os.path.join(HERE, "isrc_bruteforce.c")]
LIB_PATH = os.path.join(HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

HIT_BRUTE, HIT_BVH, HIT_TILED = 0, 1, 2
MIC_BRUTE, MIC_GRID = 0, 1
N_STAT_FIXED = 6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/liboracle.so (portable C11, -O2)."""
    newest = max(os.path.getmtime(s) for s in SOURCES)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", tmp, *SOURCES,
           "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            p, i64, i32, d = C.c_void_p, C.c_int64, C.c_int, C.c_double
            L.or_scene_new.restype = p
            L.or_scene_new.argtypes = [p, i64, p, i64, p, p, i32, i32, i32, i32]
            L.or_scene_free.argtypes = [p]
            L.or_beam_table.restype = i64
            L.or_beam_table.argtypes = [i32, p, p]
            L.or_cast_rays.restype = i32
            L.or_cast_rays.argtypes = [p, i32, i64, p, p, p, p, d, p, p]
            L.or_trace.restype = i32
            L.or_trace.argtypes = [p, p, p, i64, i32, p, i64, i32, p, d, d, i32, i32, i32,
                                   p, p, p, i64, p, p, p, p, p, p]
            L.or_trace_dir.restype = i32
            L.or_trace_dir.argtypes = [p, p, p, i64, i32, p, i32, p, p, i64, i32, p, d, d, i32, i32,
                                       i32, p, p, p, i64, p, p, p, p, p, p, p]
            L.or_levels.argtypes = [p, i64, p]
            L.or_ray_tri.restype = i32
            L.or_ray_tri.argtypes = [p, p, p, p, p, p]
            L.or_mirror_point.argtypes = [p, p, p, p]
            L.or_mirror_dir.argtypes = [p, p, p]
            L.or_reflect_cone.argtypes = [p, p, p, p, p, p]
            L.or_in_segment.restype = i32
            L.or_in_segment.argtypes = [p, p, p, p, p, p]
            L.isrc_bruteforce.restype = i64
            L.isrc_bruteforce.argtypes = [p, i64, p, i64, p, p, i32, i32, p, p, p, i64, i32,
                                          p, d, i32, p, p, i64, p, p, p, p]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Scene:
    """Oracle copy of a scene (Section 4 model: triangles with materials)."""

    def __init__(self, scene, tiles=(1, 1)):
        self.verts = _c(scene.verts, np.float32)
        self.tris = _c(scene.tris, np.int32)
        self.mat = _c(scene.mat, np.uint8)
        self.refl = _c(scene.refl, np.float32)
        self.n_bands = int(self.refl.shape[1])
        self.tiles = tuple(tiles)
        self.h = lib().or_scene_new(_ptr(self.verts), len(self.verts), _ptr(self.tris),
                                    len(self.tris), _ptr(self.mat), _ptr(self.refl),
                                    int(self.refl.shape[0]), self.n_bands, int(tiles[0]),
                                    int(tiles[1]))
        if not self.h:
            raise ValueError("oracle rejected the scene")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().or_scene_free(h)
            self.h = None


def beam_table(level: int):
    """Section 2 beams: [N,3,3] unit edge directions (CCW from outside), [N] solid angles."""
    n = 20 * 4 ** level
    dirs = np.empty((n, 3, 3), np.float64)
    omega = np.empty(n, np.float64)
    got = lib().or_beam_table(level, _ptr(dirs), _ptr(omega))
    if got != n:
        raise ValueError("bad level")
    return dirs, omega


def cast_rays(scene: Scene, o, d, has_start=None, ns=None, t_eps=1e-3, mode=HIT_BVH):
    """Closest hit of each axis ray (Section 2: only the guiding ray is tested)."""
    o = _c(o, np.float64).reshape(-1, 3)
    d = _c(d, np.float64).reshape(-1, 3)
    n = len(o)
    hs = _c(has_start if has_start is not None else np.zeros(n), np.int32)
    nsv = _c(ns if ns is not None else np.zeros((n, 3)), np.float64)
    t = np.empty(n, np.float64)
    ids = np.empty(n, np.int32)
    lib().or_cast_rays(scene.h, mode, n, _ptr(o), _ptr(d), _ptr(hs), _ptr(nsv), t_eps, _ptr(t),
                       _ptr(ids))
    return t, ids


def trace(scene: Scene, src, power, level, mics, max_order, alpha=None, energy_threshold=0.0,
          t_eps=1e-3, hit_mode=HIT_BVH, mic_mode=MIC_GRID, n_threads=1, log_cap=0,
          directivity=None, pattern_of=None, hit_log=False):
    """Full hybrid trace (Section 2), optionally tiled (Section 3).

    Directional sources (Section 2: a source's energy is split between the
    beams by its power in each direction): `directivity` [n_patterns,
    20*4**level] gains per beam, `pattern_of` [n_src] the pattern of each
    source (-1 = omnidirectional); a beam's band powers are the source's
    times its pattern's gain for that beam.

    With `hit_log`, also returns "hits" [n_src * 20*4**level, max_order + 1]
    int32: the triangle each segment's axis ray hit (-1: it escaped; -2: the
    beam did not reach that order), lineage = source * beams + the oracle's
    own beam index.

    Returns dict(I [n_m, B] W/m^2, cnt [n_m], stats dict, log dict or None).
    """
    if hit_mode == HIT_TILED and scene.tiles == (1, 1):
        hit_mode = HIT_TILED  # tiled search over one tile is still a valid mode
    src = _c(src, np.float32).reshape(-1, 3)
    power = _c(power, np.float32).reshape(len(src), scene.n_bands)
    mics = _c(mics, np.float32).reshape(-1, 3)
    nb = scene.n_bands
    a = _c(alpha if alpha is not None else np.zeros(nb), np.float64)
    I = np.zeros((len(mics), nb), np.float64)
    cnt = np.zeros(len(mics), np.int32)
    stats = np.zeros(N_STAT_FIXED + max_order + 1, np.float64)
    log = None
    ln = C.c_int64(0)
    if log_cap:
        log = dict(mic=np.empty(log_cap, np.int32), src=np.empty(log_cap, np.int32),
                   order=np.empty(log_cap, np.int32), d=np.empty(log_cap, np.float64),
                   apex=np.empty((log_cap, 3), np.float64))
    hits = np.full((len(src) * 20 * 4 ** level, max_order + 1), -2, np.int32) if hit_log else None
    if pattern_of is not None:
        gain = _c(directivity, np.float32).reshape(-1, 20 * 4 ** level)
        pat = _c(pattern_of, np.int32).reshape(len(src))
    else:
        gain, pat = None, None
    rc = lib().or_trace_dir(scene.h, _ptr(src), _ptr(power), len(src), level, _ptr(gain),
                            0 if gain is None else len(gain), _ptr(pat), _ptr(mics), len(mics),
                            max_order, _ptr(a), energy_threshold, t_eps, hit_mode, mic_mode,
                            n_threads, _ptr(I), _ptr(cnt), _ptr(stats), log_cap,
                        *(_ptr(log[k]) if log else None for k in ("mic", "src", "order", "d",
                                                                   "apex")),
                        C.byref(ln), _ptr(hits))
    if rc != 0:
        raise ValueError(f"or_trace failed: {rc}")
    if log is not None:
        k = ln.value
        log = {key: v[:k] for key, v in log.items()}
        log["full"] = k < log_cap
    st = dict(segments=stats[0], contributions=stats[1], hits=stats[2], escapes=stats[3],
              handoffs=stats[4], ties=stats[5], order_power=stats[N_STAT_FIXED:].copy())
    out = dict(I=I, cnt=cnt, stats=st, log=log)
    if hits is not None:
        out["hits"] = hits
    return out


def beam_axes(level: int):
    """Unit axes [N, 3] of the oracle's beams (normalised edge-direction sums)."""
    dirs, _ = beam_table(level)
    ax = dirs.sum(axis=1)
    return ax / np.linalg.norm(ax, axis=1, keepdims=True)


def trace_workload(w, tiles=None, **kw):
    """Convenience: trace a synth.Workload with the oracle (directional
    sources sampled at the oracle's own beam axes)."""
    sc = Scene(w.scene, tiles if tiles is not None else (1, 1))
    if tiles is not None and tuple(tiles) != (1, 1):
        kw.setdefault("hit_mode", HIT_TILED)
    d = getattr(w, "directivity", None)
    if d is not None:
        kw.setdefault("directivity", d.gains(beam_axes(w.level)))
        kw.setdefault("pattern_of", d.pattern_of)
    return trace(sc, w.src, w.power, w.level, w.mics, w.max_order, **kw)


# ------------------------------------------------------------ primitives
# One oracle building block per call, for hand-worked unit cases.
def _v(a, n=3):
    return _c(np.asarray(a, np.float64).reshape(n), np.float64)


def ray_tri(o, d, a, b, c):
    """Moller-Trumbore, two-sided, edges inclusive: t of the hit (any sign)
    or None."""
    t = np.zeros(1)
    args = [_v(x) for x in (o, d, a, b, c)]
    hit = lib().or_ray_tri(*[_ptr(x) for x in args], _ptr(t))
    return float(t[0]) if hit else None


def mirror_point(a, p, n):
    out = np.zeros(3)
    args = [_v(x) for x in (a, p, n)]
    lib().or_mirror_point(*[_ptr(x) for x in args], _ptr(out))
    return out


def mirror_dir(d, n):
    out = np.zeros(3)
    args = [_v(x) for x in (d, n)]
    lib().or_mirror_dir(*[_ptr(x) for x in args], _ptr(out))
    return out


def reflect_cone(apex, dirs, p, n):
    """The image-source step on a cone: (mirrored apex [3], edge dirs [3, 3])."""
    ao, do = np.zeros(3), np.zeros(9)
    args = [_v(apex), _v(dirs, 9), _v(p), _v(n)]
    lib().or_reflect_cone(*[_ptr(x) for x in args], _ptr(ao), _ptr(do))
    return ao, do.reshape(3, 3)


def in_segment(apex, dirs, m, start=None, end=None):
    """(inside, tie) of point m for the segment; start / end planes as
    (normal, point) pairs or None."""
    tie = np.zeros(1, np.int32)
    st = _v(np.concatenate([np.ravel(start[0]), np.ravel(start[1])]), 6) if start is not None else None
    en = _v(np.concatenate([np.ravel(end[0]), np.ravel(end[1])]), 6) if end is not None else None
    args = [_v(apex), _v(dirs, 9)]
    inside = lib().or_in_segment(_ptr(args[0]), _ptr(args[1]), _ptr(st), _ptr(en), _ptr(_v(m)), _ptr(tie))
    return bool(inside), bool(tie[0])


def levels(I):
    """Level readout: 10 log10(I / 1e-12) dB, -inf where I = 0."""
    I = _c(I, np.float64)
    L = np.empty_like(I)
    lib().or_levels(_ptr(I), I.size, _ptr(L))
    return L


def isrc(scene, src, power, mics, max_order, alpha=None, t_eps=1e-3, closed_solids=True,
         log_cap=0):
    """Brute-force image sources (Section 2's image-source method), one source."""
    v = _c(scene.verts, np.float32)
    t = _c(scene.tris, np.int32)
    m = _c(scene.mat, np.uint8)
    r = _c(scene.refl, np.float32)
    nb = r.shape[1]
    src = _c(src, np.float32).reshape(3)
    power = _c(power, np.float32).reshape(nb)
    mics = _c(mics, np.float32).reshape(-1, 3)
    a = _c(alpha if alpha is not None else np.zeros(nb), np.float64)
    I = np.zeros((len(mics), nb), np.float64)
    cnt = np.zeros(len(mics), np.int32)
    log = None
    ln = C.c_int64(0)
    if log_cap:
        log = dict(mic=np.empty(log_cap, np.int32), order=np.empty(log_cap, np.int32),
                   d=np.empty(log_cap, np.float64))
    n = lib().isrc_bruteforce(_ptr(v), len(v), _ptr(t), len(t), _ptr(m), _ptr(r), r.shape[0], nb,
                              _ptr(src), _ptr(power), _ptr(mics), len(mics), max_order, _ptr(a),
                              t_eps, 1 if closed_solids else 0, _ptr(I), _ptr(cnt), log_cap,
                              *(_ptr(log[k]) if log else None for k in ("mic", "order", "d")),
                              C.byref(ln))
    if n < 0:
        raise ValueError(f"isrc_bruteforce failed: {n}")
    if log is not None:
        k = ln.value
        log = {key: val[:k] for key, val in log.items()}
        log["full"] = k < log_cap
    return dict(I=I, cnt=cnt, n_images=int(n), log=log)
