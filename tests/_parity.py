"""Comparison helpers for GPU-vs-oracle parity tests.

Floating outputs use the condition-aware rule: |gpu - oracle| <= rtol *
(sum of |terms| of the oracle's sum + floor), where the oracle returns that
absolute-term sum beside each output.  Data ~ N(0, 1) can cancel, so a plain
relative error would be meaningless at near-zero outputs.
"""
import numpy as np

RTOL = 1e-5


def assert_cond_close(gpu, ref, abs_terms, rtol=RTOL, floor=1e-30, mask=None, what=""):
    g = np.asarray(gpu, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    a = np.asarray(abs_terms, dtype=np.float64)
    err = np.abs(g - r)
    bound = rtol * (a + floor)
    bad = err > bound
    if mask is not None:
        bad &= mask
    nbad = int(bad.sum())
    if nbad:
        idx = np.argwhere(bad)[:5]
        ratio = float(np.max(np.where(bad, err / np.maximum(bound, 1e-300), 0)))
        raise AssertionError("%s: %d elements outside %.1e * sum|terms| (worst ratio %.3g) at %s; gpu %s ref %s"
                             % (what, nbad, rtol, ratio, idx.tolist(), g[tuple(idx[0])], r[tuple(idx[0])]))
    return float(np.max(err / np.maximum(bound, 1e-300))) if err.size else 0.0


def cond_ratio(gpu, ref, abs_terms, rtol=RTOL, floor=1e-30, mask=None):
    """Largest |gpu - oracle| / (rtol * (sum|terms| + floor)) over the
    (masked) elements, without asserting: how much of a bound is used."""
    g = np.asarray(gpu, dtype=np.float64)
    r = np.asarray(ref, dtype=np.float64)
    a = np.asarray(abs_terms, dtype=np.float64)
    q = np.abs(g - r) / (rtol * (a + floor))
    if mask is not None:
        q = np.where(np.broadcast_to(mask, q.shape), q, 0.0)
    return float(q.max()) if q.size else 0.0
