"""Python binding of libbtrace (include/btrace.h): argument marshalling only.

The functions carry the C names and arguments.  Arrays may be numpy arrays
(host memory) or torch tensors (host or CUDA memory of the context's device);
the library copies them.  Every step of the trace runs in the CUDA kernels of
libbtrace.so; there is no fallback, and importing the binding fails loudly
when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build_lib

BT_OK = 0
BT_E_INVALID, BT_E_NOMEM, BT_E_CUDA, BT_E_STATE, BT_E_QUEUE_FULL, BT_E_TIMEOUT = -1, -2, -3, -4, -5, -6
BT_PENDING = 1
BT_MAX_BANDS = 8
BT_PREC_FP32, BT_PREC_MIXED, BT_PREC_FP64, BT_PREC_MIXED64 = 0, 1, 2, 3
BT_FAULT_WITHHOLD, BT_FAULT_SEGMENTS = 1, 2  # bt_trace_params.fault_test (test hooks)

_ERR_NAMES = {BT_E_INVALID: "BT_E_INVALID", BT_E_NOMEM: "BT_E_NOMEM", BT_E_CUDA: "BT_E_CUDA",
              BT_E_STATE: "BT_E_STATE", BT_E_QUEUE_FULL: "BT_E_QUEUE_FULL",
              BT_E_TIMEOUT: "BT_E_TIMEOUT"}


class bt_trace_params(C.Structure):
    _fields_ = [("max_order", C.c_int32), ("air_atten_db_per_m", C.c_float * BT_MAX_BANDS),
                ("energy_threshold_w", C.c_float), ("t_eps_m", C.c_float),
                ("tiles_x", C.c_int32), ("tiles_y", C.c_int32), ("precision", C.c_int32),
                ("watchdog_ms", C.c_int32), ("chunk_beams", C.c_int32), ("count_work", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("queue_depth", C.c_int32), ("leaf_size", C.c_int32),
                ("beams_per_warp", C.c_int32), ("fault_test", C.c_int32)]


class bt_stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("beams", "segments", "hits", "escapes", "emitted",
                                         "candidates", "contributions", "handoffs", "steals",
                                         "rounds", "nodes_visited", "tris_tested", "trace_launches",
                                         "scatter_launches")] + \
        [(n, C.c_double) for n in ("trace_ms", "trace_kernel_ms", "scatter_kernel_ms")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class BtError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {message}")
        self.code = code
        self.message = message


_lock = threading.Lock()
_lib = None
EXPECTED_SYMBOLS = ("bt_params_default", "bt_create", "bt_destroy", "bt_load_scene",
                    "bt_unload_scene", "bt_set_sources", "bt_set_microphones", "bt_trace",
                    "bt_read_levels", "bt_last_error", "bt_kernel_launches", "bt_cast_rays",
                    "bt_trace_noalloc", "bt_set_result", "bt_batch_create", "bt_batch_run",
                    "bt_batch_stats", "bt_batch_destroy", "bt_scene_share", "bt_trace_ranges",
                    "bt_ranges_stats", "bt_set_directivity", "bt_beam_axes", "bt_submit", "bt_poll",
                    "bt_wait", "bt_l2_bandwidth", "bt_set_hit_log", "bt_l2_atomics")


def lib_path() -> str:
    return build_lib.LIB


def lib():
    """Load libbtrace.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(build_lib.LIB):
                raise RuntimeError(f"{build_lib.LIB} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(build_lib.LIB)
            p, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
            L.bt_params_default.argtypes = [C.POINTER(bt_trace_params)]
            L.bt_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, p]
            L.bt_destroy.argtypes = [p]
            L.bt_load_scene.argtypes = [p, p, i64, p, i64, p, p, i32, i32, C.POINTER(i32)]
            L.bt_unload_scene.argtypes = [p, i32]
            L.bt_set_sources.argtypes = [p, i32, p, p, i64, i32]
            L.bt_set_microphones.argtypes = [p, i32, p, i64]
            L.bt_set_directivity.argtypes = [p, i32, p, i32, p]
            L.bt_beam_axes.argtypes = [p, i32, p]
            L.bt_trace.argtypes = [p, i32, C.POINTER(bt_trace_params)]
            L.bt_submit.argtypes = [p, i32, C.POINTER(bt_trace_params)]
            L.bt_poll.argtypes = [p, i32]
            L.bt_wait.argtypes = [p, i32]
            L.bt_read_levels.argtypes = [p, i32, p, p, p, C.POINTER(bt_stats)]
            L.bt_last_error.argtypes = [p]
            L.bt_last_error.restype = C.c_char_p
            L.bt_cast_rays.argtypes = [p, i32, p, p, p, i64, C.c_float, p, p]
            L.bt_trace_noalloc.argtypes = [p, i32, C.POINTER(bt_trace_params), p, p]
            L.bt_set_result.argtypes = [p, i32, p, p]
            L.bt_batch_create.argtypes = [p, p, i32, C.POINTER(bt_trace_params), C.POINTER(C.c_void_p)]
            L.bt_batch_run.argtypes = [p]
            L.bt_batch_stats.argtypes = [p, C.POINTER(bt_stats)]
            L.bt_batch_destroy.argtypes = [p]
            L.bt_scene_share.argtypes = [p, i32, C.POINTER(C.c_int32)]
            L.bt_trace_ranges.argtypes = [p, i32, p, p, p, C.POINTER(bt_trace_params), i32]
            L.bt_ranges_stats.argtypes = [p, C.POINTER(bt_stats)]
            L.bt_l2_bandwidth.argtypes = [p, i64, i32, i32, C.POINTER(C.c_double)]
            L.bt_l2_atomics.argtypes = [p, i64, i32, i32, C.POINTER(C.c_double)]
            L.bt_set_hit_log.argtypes = [p, i32, p, i64]
            L.bt_kernel_launches.argtypes = []
            L.bt_kernel_launches.restype = C.c_int64
            for name in EXPECTED_SYMBOLS:
                if name not in ("bt_last_error", "bt_kernel_launches"):
                    getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _arr(x, dtype):
    """(pointer, n_elements, keepalive) of a numpy array or torch tensor."""
    if x is None:
        return None, 0, None
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):  # torch tensor
        import torch
        tdt = {np.float32: torch.float32, np.int32: torch.int32, np.uint8: torch.uint8,
               np.float64: torch.float64}[np.dtype(dtype).type]
        t = x.to(tdt).contiguous()
        return C.c_void_p(t.data_ptr()), t.numel(), t
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(C.c_void_p), a.size, a


def _check(rc, ctx):
    if rc != BT_OK:
        msg = lib().bt_last_error(ctx)
        raise BtError(rc, msg.decode() if msg else "")


def bt_params_default() -> bt_trace_params:
    p = bt_trace_params()
    lib().bt_params_default(C.byref(p))
    return p


def bt_create(device: int = 0, stream=None):
    """Context on `device`; `stream` is a cudaStream_t handle (int) or None."""
    h = C.c_void_p()
    rc = lib().bt_create(C.byref(h), int(device), C.c_void_p(stream) if stream else None)
    if rc != BT_OK:
        raise BtError(rc, "bt_create failed")
    return h


def bt_destroy(ctx):
    lib().bt_destroy(ctx)


def bt_kernel_launches() -> int:
    return int(lib().bt_kernel_launches())


def bt_set_hit_log(ctx, scene_id: int, hits=None):
    """Register a device int32 tensor (lineages x (max_order + 1)) as the
    scene's hit log, or clear it with None."""
    if hits is None:
        _check(lib().bt_set_hit_log(ctx, int(scene_id), None, 0), ctx)
        return
    ph, n, keep = _arr(hits, np.int32)
    _check(lib().bt_set_hit_log(ctx, int(scene_id), ph, n), ctx)


def bt_l2_bandwidth(ctx, n_bytes: int = 48 << 20, repeats: int = 200, blocks_per_sm: int = 4) -> float:
    """Measured L2 read bandwidth of the context's GPU, GB/s."""
    g = C.c_double(0.0)
    _check(lib().bt_l2_bandwidth(ctx, int(n_bytes), int(repeats), int(blocks_per_sm), C.byref(g)), ctx)
    return g.value


def bt_l2_atomics(ctx, n_bytes: int = 32 << 20, repeats: int = 64, blocks_per_sm: int = 4) -> float:
    """Measured rate of float64 atomic additions in the context's GPU's L2,
    additions per second."""
    g = C.c_double(0.0)
    _check(lib().bt_l2_atomics(ctx, int(n_bytes), int(repeats), int(blocks_per_sm), C.byref(g)), ctx)
    return g.value


def bt_last_error(ctx) -> str:
    m = lib().bt_last_error(ctx)
    return m.decode() if m else ""


def bt_load_scene(ctx, verts, tris, tri_material, refl) -> int:
    pv, nv, kv = _arr(verts, np.float32)
    pt, nt, kt = _arr(tris, np.int32)
    pm, nm, km = _arr(tri_material, np.uint8)
    pr, nr, kr = _arr(refl, np.float32)
    shape = getattr(refl, "shape", None) or np.asarray(refl).shape
    n_mat, n_bands = int(shape[0]), int(shape[1])
    sid = C.c_int32(-1)
    rc = lib().bt_load_scene(ctx, pv, nv // 3, pt, nt // 3, pm, pr, n_mat, n_bands, C.byref(sid))
    _check(rc, ctx)
    return sid.value


def bt_unload_scene(ctx, scene_id: int):
    _check(lib().bt_unload_scene(ctx, int(scene_id)), ctx)


def bt_set_sources(ctx, scene_id: int, pos, power_w, icosa_level: int):
    pp, npos, kp = _arr(pos, np.float32)
    pw, _, kw = _arr(power_w, np.float32)
    _check(lib().bt_set_sources(ctx, int(scene_id), pp, pw, npos // 3, int(icosa_level)), ctx)


def bt_set_directivity(ctx, scene_id: int, patterns, pattern_of):
    """Directional sources: patterns [n_patterns, 20*4**L] per-beam gains,
    pattern_of [n_src] (-1 = omnidirectional); patterns None = all
    omnidirectional."""
    if patterns is None:
        _check(lib().bt_set_directivity(ctx, int(scene_id), None, 0, None), ctx)
        return
    pg, ng, kg = _arr(patterns, np.float32)
    po, _, ko = _arr(pattern_of, np.int32)
    n_pat = len(patterns) if hasattr(patterns, "__len__") else 1
    _check(lib().bt_set_directivity(ctx, int(scene_id), pg, int(n_pat), po), ctx)


def bt_beam_axes(ctx, icosa_level: int):
    """Unit axes [20*4**L, 3] float32 of the beams, in the order of the
    directivity gains."""
    axes = np.empty((20 * 4 ** int(icosa_level), 3), np.float32)
    _check(lib().bt_beam_axes(ctx, int(icosa_level), axes.ctypes.data_as(C.c_void_p)), ctx)
    return axes


def bt_set_microphones(ctx, scene_id: int, pos):
    pp, n, kp = _arr(pos, np.float32)
    _check(lib().bt_set_microphones(ctx, int(scene_id), pp, n // 3), ctx)


def bt_trace(ctx, scene_id: int, params: bt_trace_params):
    _check(lib().bt_trace(ctx, int(scene_id), C.byref(params)), ctx)


def bt_submit(ctx, scene_id: int, params: bt_trace_params):
    """Enqueue a trace of the scene and return without waiting for it."""
    _check(lib().bt_submit(ctx, int(scene_id), C.byref(params)), ctx)


def bt_poll(ctx, scene_id: int) -> bool:
    """True once the scene's submitted trace has finished, False while it
    runs; raises BtError if it failed."""
    rc = lib().bt_poll(ctx, int(scene_id))
    if rc == BT_PENDING:
        return False
    _check(rc, ctx)
    return True


def bt_wait(ctx, scene_id: int):
    """Block until the scene's submitted trace has finished; raises BtError
    if it failed."""
    _check(lib().bt_wait(ctx, int(scene_id)), ctx)


def bt_trace_noalloc(ctx, scene_id: int, params: bt_trace_params, level_db, path_count=None):
    """Trace into caller-owned device arrays without allocating (torch CUDA
    tensors: level_db float64 [n_m, n_bands], path_count int32 [n_m] or None)."""
    for x in (level_db, path_count):
        if x is not None:
            assert x.is_cuda and x.is_contiguous()
    rc = lib().bt_trace_noalloc(ctx, int(scene_id), C.byref(params), C.c_void_p(level_db.data_ptr()),
                                C.c_void_p(path_count.data_ptr()) if path_count is not None else None)
    _check(rc, ctx)


def bt_read_levels(ctx, scene_id: int, level_db=None, intensity=None, path_count=None):
    """Write into the given output arrays (numpy or torch, host or device;
    NULL where None) and return the trace's stats as a dict."""
    def out_ptr(x):
        if x is None:
            return None
        if hasattr(x, "data_ptr"):
            assert x.is_contiguous()
            return C.c_void_p(x.data_ptr())
        assert x.flags["C_CONTIGUOUS"] and x.flags["WRITEABLE"]
        return x.ctypes.data_as(C.c_void_p)
    st = bt_stats()
    rc = lib().bt_read_levels(ctx, int(scene_id), out_ptr(level_db), out_ptr(intensity),
                              out_ptr(path_count), C.byref(st))
    _check(rc, ctx)
    return st.as_dict()


def bt_set_result(ctx, scene_id: int, intensity, path_count=None):
    """Install a summed result ([n_m][n_bands] float64 intensity, [n_m] int32
    counts or None) in input microphone order."""
    pi, _, ki = _arr(intensity, np.float64)
    pc, _, kc = _arr(path_count, np.int32)
    _check(lib().bt_set_result(ctx, int(scene_id), pi, pc), ctx)


def bt_batch_create(ctx, scene_ids, params):
    """Batch of loaded scenes with one bt_trace_params each."""
    ids = np.ascontiguousarray(scene_ids, np.int32)
    arr = (bt_trace_params * len(ids))(*params)
    h = C.c_void_p()
    _check(lib().bt_batch_create(ctx, ids.ctypes.data_as(C.c_void_p), len(ids), arr, C.byref(h)), ctx)
    return h


def bt_batch_run(ctx, batch):
    _check(lib().bt_batch_run(batch), ctx)


def bt_batch_stats(batch) -> dict:
    st = bt_stats()
    rc = lib().bt_batch_stats(batch, C.byref(st))
    if rc != BT_OK:
        raise BtError(rc, "bt_batch_stats failed")
    return st.as_dict()


def bt_batch_destroy(batch):
    lib().bt_batch_destroy(batch)


BT_ACCUMULATE = 1


def bt_scene_share(ctx, base_scene_id: int) -> int:
    """New scene on the geometry of a loaded one (no copy)."""
    out = C.c_int32(-1)
    _check(lib().bt_scene_share(ctx, int(base_scene_id), C.byref(out)), ctx)
    return out.value


def bt_trace_ranges(ctx, scene_ids, begins, ends, params, accumulate=False):
    """Trace lineages [begins[i], ends[i]) of scene scene_ids[i], all scenes
    in the same launches."""
    n = len(scene_ids)
    ids = np.ascontiguousarray(scene_ids, np.int32)
    b = np.ascontiguousarray(begins, np.int64)
    e = np.ascontiguousarray(ends, np.int64)
    arr = (bt_trace_params * max(1, n))(*params)
    rc = lib().bt_trace_ranges(ctx, n, ids.ctypes.data_as(C.c_void_p), b.ctypes.data_as(C.c_void_p),
                               e.ctypes.data_as(C.c_void_p), arr, BT_ACCUMULATE if accumulate else 0)
    _check(rc, ctx)


def bt_ranges_stats(ctx) -> dict:
    st = bt_stats()
    _check(lib().bt_ranges_stats(ctx, C.byref(st)), ctx)
    return st.as_dict()


def bt_cast_rays(ctx, scene_id: int, origins, dirs, start_normals=None, t_eps_m: float = 1e-3):
    """Closest hit per ray: (t [n] float32, triangle index [n] int32)."""
    po, n, ko = _arr(origins, np.float32)
    pd, _, kd = _arr(dirs, np.float32)
    pn, _, kn = _arr(start_normals, np.float32)
    t = np.empty(n // 3, np.float32)
    ids = np.empty(n // 3, np.int32)
    rc = lib().bt_cast_rays(ctx, int(scene_id), po, pd, pn, n // 3, C.c_float(t_eps_m),
                            t.ctypes.data_as(C.c_void_p), ids.ctypes.data_as(C.c_void_p))
    _check(rc, ctx)
    return t, ids


class Tracer:
    """Convenience wrapper: one context, scenes loaded from synth.Workload-like
    objects, results returned as numpy arrays."""

    def __init__(self, device: int = 0, stream=None, ctx=None):
        """A new context on `device`, or a view of the caller's context `ctx`
        (which close() then leaves alone)."""
        self._own = ctx is None
        self.ctx = bt_create(device, stream) if ctx is None else ctx

    def close(self):
        if self.ctx and self._own:
            bt_destroy(self.ctx)
        self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_geometry(self, w) -> int:
        """Load only the city model of workload-like `w` (a resident scene)."""
        return bt_load_scene(self.ctx, w.scene.verts, w.scene.tris, w.scene.mat, w.scene.refl)

    def load(self, w) -> int:
        sid = bt_load_scene(self.ctx, w.scene.verts, w.scene.tris, w.scene.mat, w.scene.refl)
        bt_set_sources(self.ctx, sid, w.src, w.power, w.level)
        d = getattr(w, "directivity", None)
        if d is not None:
            # the patterns sampled at this library's beam axes
            bt_set_directivity(self.ctx, sid, d.gains(bt_beam_axes(self.ctx, w.level)), d.pattern_of)
        bt_set_microphones(self.ctx, sid, w.mics)
        return sid

    def params(self, max_order, **kw) -> bt_trace_params:
        p = bt_params_default()
        p.max_order = int(max_order)
        for k, v in kw.items():
            if k == "air_atten_db_per_m":
                for b, a in enumerate(v):
                    p.air_atten_db_per_m[b] = float(a)
            else:
                setattr(p, k, v)
        return p

    def run(self, w, sid=None, **kw):
        """Trace workload w; returns dict(level, I, cnt, stats) as numpy."""
        if sid is None:
            sid = self.load(w)
        bt_trace(self.ctx, sid, self.params(w.max_order, **kw))
        nb = int(w.scene.refl.shape[1])
        n = len(w.mics)
        L = np.empty((n, nb), np.float64)
        I = np.empty((n, nb), np.float64)
        cnt = np.empty(n, np.int32)
        st = bt_read_levels(self.ctx, sid, L, I, cnt)
        return dict(level=L, I=I, cnt=cnt, stats=st, scene_id=sid)
