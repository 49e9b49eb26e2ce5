"""Python entry points of the FP64 CPU oracle (``inpc_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this module.  Nothing here shares code with the CUDA path: the C
source is compiled with gcc into ``oracle/_build/liboracle.so``.

Every function takes and returns numpy arrays; floating inputs are converted
to float64 (exactly, since they are float32 values), outputs are float64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "inpc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available).  FP contraction
    is disabled so that the FP32 projection follows the written operation
    order exactly."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
            _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class OracleCamera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_plane", C.c_float), ("far_plane", C.c_float)]


class OracleRasterOpts(C.Structure):
    _fields_ = [("opacity_from_ch0", C.c_int32), ("n_channels", C.c_int32), ("t_min", C.c_double),
                ("alpha_max", C.c_double), ("ambiguity_rel", C.c_double)]


_P = C.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            L.oracle_num_threads.restype = C.c_int
            L.oracle_philox4x32_10.argtypes = [_P, _P, _P]
            L.oracle_philox_stream.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int64, _P]
            L.oracle_build_cdf.argtypes = [_P, C.c_int64, _P, _P]
            L.oracle_build_cdf.restype = C.c_int
            L.oracle_search_cdf.argtypes = [_P, C.c_int64, C.c_double]
            L.oracle_search_cdf.restype = C.c_int64
            L.oracle_scale_draw.argtypes = [C.c_uint64, C.c_uint64]
            L.oracle_scale_draw.restype = C.c_uint64
            L.oracle_sample_octree.argtypes = [_P, _P, _P, C.c_int64, C.c_double, C.c_uint64, C.c_uint32,
                                               C.c_int64, _P, _P, _P]
            L.oracle_draw_leaves.argtypes = [_P, C.c_int64, C.c_uint64, C.c_uint32, C.c_int64, _P]
            L.oracle_draw_leaves.restype = C.c_int
            L.oracle_sample_octree.restype = C.c_int
            L.oracle_hash_layout.argtypes = [C.c_int32, _P, C.c_int32, _P]
            L.oracle_hash_layout.restype = C.c_int64
            L.oracle_hash_vertex_index.argtypes = [C.c_int64, C.c_int32, C.c_int64, C.c_int64, C.c_int64]
            L.oracle_hash_vertex_index.restype = C.c_int64
            L.oracle_hash_fwd.argtypes = [C.c_int32, _P, C.c_int32, C.c_int32, _P, _P, C.c_int64, _P, _P]
            L.oracle_hash_fwd.restype = C.c_int
            L.oracle_hash_bwd.argtypes = [C.c_int32, _P, C.c_int32, C.c_int32, _P, _P, C.c_int64, _P, _P, _P]
            L.oracle_hash_bwd.restype = C.c_int
            L.oracle_project.argtypes = [C.POINTER(OracleCamera), _P, _P, _P, _P]
            L.oracle_project.restype = C.c_int
            L.oracle_splat_corners.argtypes = [C.c_double, C.c_double, _P, _P, _P]
            L.oracle_raster_fwd.argtypes = [C.POINTER(OracleCamera), C.POINTER(OracleRasterOpts), _P, _P, _P,
                                            C.c_int64, _P, _P, _P, _P, _P, _P, _P]
            L.oracle_raster_fwd.restype = C.c_int
            L.oracle_raster_bwd.argtypes = [C.POINTER(OracleCamera), C.POINTER(OracleRasterOpts), _P, _P, _P,
                                            C.c_int64, _P, _P, _P, _P, _P, _P]
            L.oracle_raster_bwd.restype = C.c_int
            L.oracle_fragment_lists.argtypes = [C.POINTER(OracleCamera), _P, C.c_int64, _P, _P, _P, _P]
            L.oracle_fragment_lists.restype = C.c_int64
            L.oracle_point_weights.argtypes = [C.POINTER(OracleCamera), C.POINTER(OracleRasterOpts), _P, _P, _P,
                                               C.c_int64, _P, _P]
            L.oracle_point_weights.restype = C.c_int
            L.oracle_octree_update.argtypes = [_P, _P, C.c_int64, _P, _P, C.c_int64, C.c_double]
            L.oracle_octree_update.restype = C.c_int
            L.oracle_octree_subdivide.argtypes = [_P, _P, _P, _P, C.c_int64, C.c_double, C.c_double, C.c_int64,
                                                  _P, _P, _P, _P]
            L.oracle_octree_subdivide.restype = C.c_int64
            L.oracle_octree_prune.argtypes = [_P, _P, _P, _P, C.c_int64, C.c_double, _P, _P, _P, _P]
            L.oracle_octree_prune.restype = C.c_int64
            L.oracle_view_weights.argtypes = [_P, _P, _P, C.c_int64, C.c_double, C.POINTER(OracleCamera),
                                              C.c_double, C.c_double, _P]
            L.oracle_view_weights.restype = C.c_int
            L.oracle_point_in_view.argtypes = [C.POINTER(OracleCamera), _P]
            L.oracle_point_in_view.restype = C.c_int
            L.oracle_resample_view.argtypes = [_P, _P, _P, C.c_int64, C.c_double, C.POINTER(OracleCamera),
                                               C.c_uint64, C.c_uint32, C.c_int64, C.c_int32, _P, _P, _P]
            L.oracle_resample_view.restype = C.c_int
            L.oracle_level_weights.argtypes = [_P, _P, C.c_int64, C.c_double, _P]
            L.oracle_level_weights.restype = C.c_int
            L.oracle_radical_inverse.argtypes = [C.c_uint32, C.c_uint64]
            L.oracle_radical_inverse.restype = C.c_double
            L.oracle_sample_halton.argtypes = [_P, _P, _P, C.c_int64, C.c_double, C.c_uint64, C.c_int64, _P, _P]
            L.oracle_sample_halton.restype = C.c_int
            L.oracle_contract.argtypes = [_P, C.c_int64, _P, C.c_float, _P]
            L.oracle_contract.restype = C.c_int
            L.oracle_sh_basis.argtypes = [_P, _P]
            L.oracle_sh_basis.restype = None
            L.oracle_sh_head_fwd.argtypes = [C.POINTER(OracleCamera), _P, _P, C.c_int64, C.c_int32, _P, _P, _P]
            L.oracle_sh_head_fwd.restype = C.c_int
            L.oracle_sh_head_bwd.argtypes = [C.POINTER(OracleCamera), _P, _P, C.c_int64, C.c_int32, _P, _P, _P, _P]
            L.oracle_sh_head_bwd.restype = C.c_int
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


class OracleError(RuntimeError):
    pass


# ---------------------------------------------------------------- Philox ---
def philox4x32_10(key, ctr) -> np.ndarray:
    k = np.asarray(key, dtype=np.uint32).copy()
    c = np.asarray(ctr, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(k), _ptr(c), _ptr(out))
    return out


def philox_stream(seed: int, n: int, ctr1: int = 0, ctr2: int = 0, ctr3: int = 0) -> np.ndarray:
    out = np.zeros((n, 4), dtype=np.uint32)
    lib().oracle_philox_stream(C.c_uint64(seed), ctr1, ctr2, ctr3, n, _ptr(out))
    return out


# -------------------------------------------------------------- sampling ---
def build_cdf(weights):
    w = _f64(weights)
    cdf = np.zeros(w.shape[0], dtype=np.float64)
    tot = np.zeros(1, dtype=np.float64)
    st = lib().oracle_build_cdf(_ptr(w), w.shape[0], _ptr(cdf), _ptr(tot))
    if st != 0:
        raise OracleError("build_cdf failed (%d)" % st)
    return cdf, float(tot[0])


def search_cdf(cdf, r: float) -> int:
    c = _f64(cdf)
    return int(lib().oracle_search_cdf(_ptr(c), c.shape[0], float(r)))


def scale_draw(b53: int, Q: int) -> int:
    return int(lib().oracle_scale_draw(C.c_uint64(b53), C.c_uint64(Q)))


def draw_leaves(weights, seed: int, view_id: int, n_samples: int) -> np.ndarray:
    """Leaf of each draw, in draw order (before grouping by leaf)."""
    w = _f64(weights)
    out = np.zeros(n_samples, dtype=np.int32)
    st = lib().oracle_draw_leaves(_ptr(w), w.shape[0], C.c_uint64(seed), view_id, n_samples, _ptr(out))
    if st != 0:
        raise OracleError("draw_leaves failed (%d)" % st)
    return out


def sample_octree(tree, seed: int, view_id: int, n_samples: int):
    """Leaf indices (int32 [N], grouped by leaf), exact FP64 positions
    ([N, 3]) and per-leaf counts (int64 [L])."""
    centers = _f32(tree.centers)
    levels = _i32(tree.levels)
    weights = _f64(tree.weights)
    leaf = np.zeros(n_samples, dtype=np.int32)
    pos = np.zeros((n_samples, 3), dtype=np.float64)
    counts = np.zeros(levels.shape[0], dtype=np.int64)
    st = lib().oracle_sample_octree(_ptr(centers), _ptr(levels), _ptr(weights), levels.shape[0],
                                    float(tree.root_size), C.c_uint64(seed), view_id, n_samples,
                                    _ptr(leaf), _ptr(pos), _ptr(counts))
    if st != 0:
        raise OracleError("sample_octree failed (%d)" % st)
    return leaf, pos, counts


# ------------------------------------------------------------- hash grid ---
def hash_layout(res, log2_T: int):
    r = _i32(res)
    offs = np.zeros(len(res), dtype=np.int64)
    total = lib().oracle_hash_layout(len(res), _ptr(r), log2_T, _ptr(offs))
    return int(total), offs


def hash_entries(res, log2_T: int) -> int:
    return hash_layout(res, log2_T)[0]


def hash_vertex_index(res_l: int, log2_T: int, vx: int, vy: int, vz: int) -> int:
    return int(lib().oracle_hash_vertex_index(res_l, log2_T, vx, vy, vz))


def hash_fwd(res, log2_T: int, table, pos, with_abs: bool = False):
    r = _i32(res)
    tab = _f64(table)
    p = _f64(pos)
    n = p.shape[0]
    F = tab.shape[1]
    h = np.zeros((n, len(res) * F), dtype=np.float64)
    ab = np.zeros_like(h) if with_abs else None
    st = lib().oracle_hash_fwd(len(res), _ptr(r), log2_T, F, _ptr(tab), _ptr(p), n, _ptr(h), _ptr(ab))
    if st != 0:
        raise OracleError("hash_fwd failed (%d)" % st)
    return (h, ab) if with_abs else h


def hash_bwd(res, log2_T: int, n_feats: int, pos, dh, with_abs: bool = False, dh_abs=None):
    r = _i32(res)
    p = _f64(pos)
    g = _f64(dh)
    n = p.shape[0]
    total, _ = hash_layout(res, log2_T)
    grad = np.zeros((total, n_feats), dtype=np.float64)
    ab = np.zeros_like(grad) if with_abs else None
    da = _f64(dh_abs) if dh_abs is not None else None
    st = lib().oracle_hash_bwd(len(res), _ptr(r), log2_T, n_feats, _ptr(p), _ptr(g), n, _ptr(grad), _ptr(ab),
                               _ptr(da))
    if st != 0:
        raise OracleError("hash_bwd failed (%d)" % st)
    return (grad, ab) if with_abs else grad


# ------------------------------------------------------------ rasterizer ---
def camera_struct(cam) -> OracleCamera:
    c = OracleCamera()
    R = np.asarray(cam.R, dtype=np.float32).reshape(9)
    t = np.asarray(cam.t, dtype=np.float32).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height = cam.width, cam.height
    c.near_plane, c.far_plane = cam.near, cam.far
    return c


def _opts(n_channels, head_mode, t_min, alpha_max, ambiguity_rel):
    o = OracleRasterOpts()
    o.opacity_from_ch0 = 1 if head_mode else 0
    o.n_channels = n_channels
    o.t_min = t_min
    o.alpha_max = alpha_max
    o.ambiguity_rel = ambiguity_rel
    return o


def project(cam, pos):
    """FP32 projection (u, v, depth, in_front) of each point."""
    p = _f32(pos)
    n = p.shape[0]
    cs = camera_struct(cam)
    out = np.zeros((n, 3), dtype=np.float32)
    ok = np.zeros(n, dtype=bool)
    u = np.zeros(1, np.float32); v = np.zeros(1, np.float32); d = np.zeros(1, np.float32)
    L = lib()
    for i in range(n):
        ok[i] = bool(L.oracle_project(C.byref(cs), _ptr(p[i]), _ptr(u), _ptr(v), _ptr(d)))
        out[i] = (u[0], v[0], d[0])
    return out, ok


def splat_corners(u: float, v: float):
    pi = np.zeros(4, np.int64); pj = np.zeros(4, np.int64); w = np.zeros(4, np.float64)
    lib().oracle_splat_corners(float(u), float(v), _ptr(pi), _ptr(pj), _ptr(w))
    return pi, pj, w


def raster_fwd(cam, pos, feat, opacity=None, head_mode=False, t_min=1e-4, alpha_max=0.99,
               ambiguity_rel=1e-5, with_abs=False, feat_abs=None):
    """Returns dict with image [H,W,F], T_final, n_contrib, n_frags, flags (and abs).
    ``feat_abs`` (optional, [N,F]) replaces |feat| as the channel magnitude in
    the absolute-term sums (the tolerance scale), e.g. a grid query's sum |w t|."""
    p = _f32(pos)
    f = _f64(feat)
    n, F = f.shape
    op = _f64(opacity) if opacity is not None else None
    if not head_mode and op is None:
        raise ValueError("opacity required unless head_mode")
    H, W = cam.height, cam.width
    image = np.zeros((H, W, F), np.float64)
    T = np.zeros((H, W), np.float64)
    nc = np.zeros((H, W), np.int32)
    nf = np.zeros((H, W), np.int32)
    flags = np.zeros((H, W), np.uint8)
    ab = np.zeros((H, W, F), np.float64) if with_abs else None
    cs = camera_struct(cam)
    o = _opts(F, head_mode, t_min, alpha_max, ambiguity_rel)
    fa = _f64(feat_abs) if feat_abs is not None else None
    st = lib().oracle_raster_fwd(C.byref(cs), C.byref(o), _ptr(p), _ptr(op), _ptr(f), n, _ptr(image), _ptr(T),
                                 _ptr(nc), _ptr(nf), _ptr(flags), _ptr(ab), _ptr(fa))
    if st != 0:
        raise OracleError("raster_fwd failed (%d)" % st)
    out = dict(image=image, T_final=T, n_contrib=nc, n_frags=nf, flags=flags)
    if with_abs:
        out["abs"] = ab
    return out


def raster_bwd(cam, pos, feat, d_image, opacity=None, head_mode=False, t_min=1e-4, alpha_max=0.99,
               with_abs=False, feat_abs=None):
    """Returns dict with d_feat [N,F] (and d_opacity [N] in given-opacity mode)."""
    p = _f32(pos)
    f = _f64(feat)
    n, F = f.shape
    op = _f64(opacity) if opacity is not None else None
    g = _f64(d_image)
    d_feat = np.zeros((n, F), np.float64)
    d_op = np.zeros(n, np.float64)
    ab_f = np.zeros((n, F), np.float64) if with_abs else None
    ab_o = np.zeros(n, np.float64) if with_abs else None
    cs = camera_struct(cam)
    o = _opts(F, head_mode, t_min, alpha_max, 0.0)
    fa = _f64(feat_abs) if feat_abs is not None else None
    st = lib().oracle_raster_bwd(C.byref(cs), C.byref(o), _ptr(p), _ptr(op), _ptr(f), n, _ptr(g),
                                 _ptr(d_op), _ptr(d_feat), _ptr(ab_f), _ptr(ab_o), _ptr(fa))
    if st != 0:
        raise OracleError("raster_bwd failed (%d)" % st)
    out = dict(d_feat=d_feat)
    if not head_mode:
        out["d_opacity"] = d_op
    if with_abs:
        out["abs_feat"] = ab_f
        out["abs_opacity"] = ab_o
    return out


def fragment_lists(cam, pos):
    """Per-pixel fragment counts [H,W] and the concatenated (id, corner, depth)
    lists in blending order."""
    p = _f32(pos)
    n = p.shape[0]
    cs = camera_struct(cam)
    cnt = np.zeros(cam.height * cam.width, np.int64)
    total = lib().oracle_fragment_lists(C.byref(cs), _ptr(p), n, _ptr(cnt), None, None, None)
    ids = np.zeros(max(total, 1), np.int32)
    cor = np.zeros(max(total, 1), np.int32)
    dep = np.zeros(max(total, 1), np.float32)
    lib().oracle_fragment_lists(C.byref(cs), _ptr(p), n, _ptr(cnt), _ptr(ids), _ptr(cor), _ptr(dep))
    return cnt.reshape(cam.height, cam.width), ids[:total], cor[:total], dep[:total]


# ------------------------------------------------------------------ octree ---
def point_weights(cam, pos, feat, opacity=None, head_mode=False, t_min=1e-4, alpha_max=0.99, with_pixel_sums=False):
    """Per-point blending weights b [N] for the probability updates
    (Sec. 3.1 Eq. 2/3 with App. A.6's bilinear-weighted combination); with
    ``with_pixel_sums`` also the per-pixel sum of T_k alpha_k [H,W]."""
    p = _f32(pos)
    f = _f64(feat)
    n, F = f.shape
    op = _f64(opacity) if opacity is not None else None
    if not head_mode and op is None:
        raise ValueError("opacity required unless head_mode")
    b = np.zeros(n, np.float64)
    ps = np.zeros((cam.height, cam.width), np.float64) if with_pixel_sums else None
    cs = camera_struct(cam)
    o = _opts(F, head_mode, t_min, alpha_max, 0.0)
    st = lib().oracle_point_weights(C.byref(cs), C.byref(o), _ptr(p), _ptr(op), _ptr(f), n, _ptr(b), _ptr(ps))
    if st != 0:
        raise OracleError("point_weights failed (%d)" % st)
    return (b, ps) if with_pixel_sums else b


def octree_update(leaf_idx, b, p, q, lambda_u=0.9968):
    """Eq. 2 / Eq. 3 for one step; returns the new (p, q) (float64)."""
    li = _i32(leaf_idx)
    bb = _f32(b)
    pp = _f64(p).copy()
    qq = _f64(q).copy()
    st = lib().oracle_octree_update(_ptr(li), _ptr(bb), li.shape[0], _ptr(pp), _ptr(qq), pp.shape[0],
                                    float(lambda_u))
    if st != 0:
        raise OracleError("octree_update failed (%d)" % st)
    return pp, qq


def octree_subdivide(centers, levels, p, q, root_size=1.0, tau_s=0.5, max_leaves=256 ** 3):
    """Sec. 3.1 subdivision; returns (centers, levels, p, q) of the new leaves."""
    c = _f32(centers)
    lv = _i32(levels)
    pp, qq = _f64(p), _f64(q)
    L = lv.shape[0]
    co = np.zeros((8 * max(L, 1), 3), np.float32)
    lo = np.zeros(8 * max(L, 1), np.int32)
    po = np.zeros(8 * max(L, 1), np.float64)
    qo = np.zeros(8 * max(L, 1), np.float64)
    n = lib().oracle_octree_subdivide(_ptr(c), _ptr(lv), _ptr(pp), _ptr(qq), L, float(root_size), float(tau_s),
                                      int(max_leaves), _ptr(co), _ptr(lo), _ptr(po), _ptr(qo))
    return co[:n], lo[:n], po[:n], qo[:n]


def octree_prune(centers, levels, p, q, tau_p=0.01):
    """Sec. 3.1 pruning; returns (centers, levels, p, q) of the kept leaves."""
    c = _f32(centers)
    lv = _i32(levels)
    pp, qq = _f64(p), _f64(q)
    L = lv.shape[0]
    co = np.zeros((max(L, 1), 3), np.float32)
    lo = np.zeros(max(L, 1), np.int32)
    po = np.zeros(max(L, 1), np.float64)
    qo = np.zeros(max(L, 1), np.float64)
    n = lib().oracle_octree_prune(_ptr(c), _ptr(lv), _ptr(pp), _ptr(qq), L, float(tau_p), _ptr(co), _ptr(lo),
                                  _ptr(po), _ptr(qo))
    return co[:n], lo[:n], po[:n], qo[:n]


# ---------------------------------------------------- view-specific sampling ---
def view_weights(tree, cam, p=None, lambda_l=0.5, tau_d=1e-8):
    """Eq. 4 view-specific leaf weights (float64 [L]); p defaults to the
    tree's weights."""
    c = _f32(tree.centers)
    lv = _i32(tree.levels)
    pp = _f64(tree.weights if p is None else p)
    w = np.zeros(lv.shape[0], np.float64)
    cs = camera_struct(cam)
    st = lib().oracle_view_weights(_ptr(c), _ptr(lv), _ptr(pp), lv.shape[0], float(tree.root_size), C.byref(cs),
                                   float(lambda_l), float(tau_d), _ptr(w))
    if st != 0:
        raise OracleError("view_weights failed (%d)" % st)
    return w


def points_in_view(cam, pos):
    p = _f32(pos)
    cs = camera_struct(cam)
    return np.array([lib().oracle_point_in_view(C.byref(cs), _ptr(p[j])) for j in range(p.shape[0])], bool)


def sample_view(tree, w, cam, seed: int, view_id: int, n_samples: int, max_rounds: int = 8):
    """Sampling with the view weights w, then the re-sampling rounds of App.
    A.4; returns (leaf int32 [N], pos float32 [N,3], samples left not in view)."""
    view_tree = type(tree)(centers=tree.centers, levels=tree.levels, weights=np.asarray(w, np.float64),
                           root_size=tree.root_size)
    leaf, pos64, _ = sample_octree(view_tree, seed, view_id, n_samples)
    leaf = _i32(leaf).copy()
    pos = pos64.astype(np.float32)
    left = C.c_int64(0)
    cs = camera_struct(cam)
    c, lv, ww = _f32(tree.centers), _i32(tree.levels), _f64(w)
    st = lib().oracle_resample_view(_ptr(c), _ptr(lv), _ptr(ww), lv.shape[0], float(tree.root_size), C.byref(cs),
                                    int(seed), int(view_id), n_samples, int(max_rounds), _ptr(leaf), _ptr(pos),
                                    C.byref(left))
    if st != 0:
        raise OracleError("resample_view failed (%d)" % st)
    return leaf, pos, int(left.value)


# ------------------------------------------------------------ pre-extraction ---
def level_weights(levels, p, lambda_l=0.5):
    """Eq. 4 without visibility and depth: p / 2^(l lambda_l)."""
    lv = _i32(levels)
    pp = _f64(p)
    w = np.zeros(lv.shape[0], np.float64)
    lib().oracle_level_weights(_ptr(lv), _ptr(pp), lv.shape[0], float(lambda_l), _ptr(w))
    return w


def radical_inverse(base: int, i: int) -> float:
    return float(lib().oracle_radical_inverse(int(base), int(i)))


def sample_halton(tree, w, seed: int, n_samples: int):
    """Viewpoint-independent pre-extraction: (leaf int32 [N], pos float32 [N,3])."""
    c, lv, ww = _f32(tree.centers), _i32(tree.levels), _f64(w)
    leaf = np.zeros(max(n_samples, 1), np.int32)
    pos = np.zeros((max(n_samples, 1), 3), np.float32)
    st = lib().oracle_sample_halton(_ptr(c), _ptr(lv), _ptr(ww), lv.shape[0], float(tree.root_size), int(seed),
                                    n_samples, _ptr(leaf), _ptr(pos))
    if st != 0:
        raise OracleError("sample_halton failed (%d)" % st)
    return leaf[:n_samples], pos[:n_samples]


# ------------------------------------------------------------------- SH head ---
def contract(pos, center, radius):
    """Spherical contraction into [0, 1]^3 (FP32, the kernel's operation order)."""
    p = _f32(pos)
    c = _f32(center)
    out = np.zeros_like(p)
    lib().oracle_contract(_ptr(p), p.shape[0], _ptr(c), float(radius), _ptr(out))
    return out


def sh_basis(d):
    dd = _f64(d)
    Y = np.zeros(9, np.float64)
    lib().oracle_sh_basis(_ptr(dd), _ptr(Y))
    return Y


def sh_head_fwd(cam, pos, h, with_abs=False):
    """(alpha [N], color [N,4][, abs [N,4]]) of the degree-2 SH head."""
    p = _f32(pos)
    hh = _f64(h)
    n, F = hh.shape
    a = np.zeros(n, np.float64)
    col = np.zeros((n, 4), np.float64)
    ab = np.zeros((n, 4), np.float64) if with_abs else None
    cs = camera_struct(cam)
    if lib().oracle_sh_head_fwd(C.byref(cs), _ptr(p), _ptr(hh), n, F, _ptr(a), _ptr(col), _ptr(ab)) != 0:
        raise OracleError("sh_head_fwd failed")
    return (a, col, ab) if with_abs else (a, col)


def sh_head_bwd(cam, pos, h, d_alpha, d_color, with_abs=False):
    p = _f32(pos)
    hh = _f64(h)
    n, F = hh.shape
    da, dc = _f64(d_alpha), _f64(d_color)
    dh = np.zeros((n, F), np.float64)
    ab = np.zeros((n, F), np.float64) if with_abs else None
    cs = camera_struct(cam)
    if lib().oracle_sh_head_bwd(C.byref(cs), _ptr(p), _ptr(hh), n, F, _ptr(da), _ptr(dc), _ptr(dh), _ptr(ab)) != 0:
        raise OracleError("sh_head_bwd failed")
    return (dh, ab) if with_abs else dh
