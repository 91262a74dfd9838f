"""Comparison helpers for GPU-vs-oracle parity (test infrastructure).

The acceptance bar: per microphone, every band's level within 0.1 dB of the
FP64 oracle for at least 99.9% of microphones and within 1 dB for all; a
microphone no beam reached must be -inf on both sides.
"""
import numpy as np

TOL_DB_MOST = 0.1
TOL_DB_ALL = 1.0
FRACTION_MOST = 0.999


def level_db(I):
    I = np.asarray(I, np.float64)
    with np.errstate(divide="ignore"):
        return np.where(I > 0, 10.0 * np.log10(np.where(I > 0, I, 1.0)) + 120.0, -np.inf)


def db_error(L_gpu, L_ref):
    """Per-microphone max over bands of |L_gpu - L_ref|; -inf on both sides is 0."""
    a = np.asarray(L_gpu, np.float64)
    b = np.asarray(L_ref, np.float64)
    both_inf = np.isneginf(a) & np.isneginf(b)
    with np.errstate(invalid="ignore"):
        d = np.abs(a - b)
    d = np.where(both_inf, 0.0, d)
    d = np.where(np.isnan(d), np.inf, d)
    return d.max(axis=1) if d.ndim == 2 else d


def summary(L_gpu, L_ref):
    e = db_error(L_gpu, L_ref)
    return dict(n=len(e), frac_within_0p1=float(np.mean(e <= TOL_DB_MOST)),
                max_db=float(e.max()) if len(e) else 0.0,
                p999_db=float(np.quantile(e, 0.999)) if len(e) else 0.0,
                worst=np.argsort(-e)[:5].tolist())


def assert_parity(L_gpu, L_ref, what=""):
    s = summary(L_gpu, L_ref)
    assert s["frac_within_0p1"] >= FRACTION_MOST, f"{what}: {s}"
    assert s["max_db"] <= TOL_DB_ALL, f"{what}: {s}"
    return s
