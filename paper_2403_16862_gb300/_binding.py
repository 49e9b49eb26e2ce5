"""ctypes binding of the C ABI in ``include/inpc.h`` (argument marshalling
only; every computation runs in the CUDA library).

Loading fails loudly when ``_lib/libinpc.so`` has not been built: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libinpc.so")

INPC_OK = 0
INPC_ERR_INVALID_ARG = 1
INPC_ERR_CUDA = 2
INPC_ERR_CAPACITY = 3
INPC_ERR_TIMEOUT = 4
INPC_ERR_UNSUPPORTED = 5
STATUS_NAMES = {0: "INPC_OK", 1: "INPC_ERR_INVALID_ARG", 2: "INPC_ERR_CUDA", 3: "INPC_ERR_CAPACITY",
                4: "INPC_ERR_TIMEOUT", 5: "INPC_ERR_UNSUPPORTED"}

INPC_DEV_BAD_WEIGHT = 0x1
INPC_DEV_NO_WEIGHT = 0x2
INPC_DEV_BAD_LEAF = 0x4
INPC_DEV_BAD_BLEND_WEIGHT = 0x8
INPC_DEV_TIMEOUT = 0x10

INPC_F32 = 0
INPC_BF16 = 1
INPC_OPACITY_GIVEN = 0
INPC_OPACITY_FROM_CH0 = 1

# Every symbol the header declares; tests check the library exports them.
DECLARED = [
    "inpc_last_error", "inpc_version", "inpc_kernel_launches", "inpc_read_device_status",
    "inpc_sample_workspace_size", "inpc_sample_octree", "inpc_sample_octree_noalloc",
    "inpc_hashgrid_n_entries", "inpc_query_hashgrid", "inpc_query_hashgrid_bwd",
    "inpc_rasterize_workspace_size", "inpc_rasterize_fwd", "inpc_rasterize_bwd",
    "inpc_rasterize_bwd_hashgrid_workspace_size", "inpc_rasterize_bwd_hashgrid",
    "inpc_kernel_timer_enable", "inpc_kernel_timer_read",
    "inpc_rasterize_point_weights", "inpc_octree_update_workspace_size", "inpc_octree_update",
    "inpc_octree_refine_workspace_size", "inpc_octree_subdivide", "inpc_octree_prune",
    "inpc_view_weights", "inpc_sample_octree_view",
    "inpc_level_weights", "inpc_sample_octree_halton", "inpc_accumulate_image",
    "inpc_contract_positions", "inpc_sh_head_fwd", "inpc_sh_head_bwd",
    "inpc_render_batch", "inpc_philox4x32_10",
    "inpc_sample_query_batch_workspace_size", "inpc_sample_query_batch", "inpc_render_batch_persistent",
    "inpc_set_fault", "inpc_l2_reduction_rate",
]


class InpcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class InpcOctree(C.Structure):
    _fields_ = [("centers", C.c_void_p), ("levels", C.c_void_p), ("weights", C.c_void_p),
                ("root_size", C.c_float), ("n_leaves", C.c_int64)]


class InpcFrontView(C.Structure):
    _fields_ = [("view_id", C.c_uint32), ("n_samples", C.c_int64), ("leaf_idx", C.c_void_p), ("pos", C.c_void_p),
                ("h", C.c_void_p)]


class InpcHashgridDesc(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("n_feats", C.c_int32), ("log2_T", C.c_int32),
                ("res", C.c_int32 * 32), ("table_dtype", C.c_int32), ("out_dtype", C.c_int32)]


class InpcCamera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_plane", C.c_float), ("far_plane", C.c_float)]


class InpcRasterOpts(C.Structure):
    _fields_ = [("opacity_mode", C.c_int32), ("n_channels", C.c_int32), ("feat_dtype", C.c_int32),
                ("image_dtype", C.c_int32), ("t_min", C.c_float), ("alpha_max", C.c_float),
                ("tile_w", C.c_int32), ("tile_h", C.c_int32)]


class InpcViewJob(C.Structure):
    _fields_ = [("cam", InpcCamera), ("opts", InpcRasterOpts), ("view_id", C.c_uint32), ("n_samples", C.c_int64),
                ("leaf_idx", C.c_void_p), ("pos", C.c_void_p), ("h", C.c_void_p), ("image", C.c_void_p),
                ("T_final", C.c_void_p), ("n_contrib", C.c_void_p), ("d_image", C.c_void_p),
                ("sample_ws", C.c_void_p), ("sample_ws_bytes", C.c_size_t), ("raster_ws", C.c_void_p),
                ("raster_ws_bytes", C.c_size_t)]


_P = C.c_void_p
_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libinpc.so (built by ``paper_2403_16862_gb300.build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError("libinpc.so is not built (%s); run paper_2403_16862_gb300.build.build() "
                              "or __graft_entry__.build() first" % path)
        L = C.CDLL(path)
        L.inpc_last_error.restype = C.c_char_p
        L.inpc_version.restype = C.c_char_p
        L.inpc_kernel_launches.restype = C.c_uint64
        L.inpc_read_device_status.argtypes = [_P, _P, C.POINTER(C.c_uint32)]
        L.inpc_sample_workspace_size.argtypes = [C.c_int64, C.c_int64, C.POINTER(C.c_size_t)]
        L.inpc_sample_octree.argtypes = [C.POINTER(InpcOctree), C.c_uint64, C.c_uint32, C.c_int64, _P, _P, _P, _P,
                                         C.c_size_t, _P]
        L.inpc_philox4x32_10.argtypes = [_P, _P, C.c_int64, _P, _P]
        L.inpc_sample_octree_noalloc.argtypes = [C.POINTER(InpcOctree), C.c_uint64, C.c_uint32, C.c_int64, _P, _P,
                                                 _P, _P]
        L.inpc_hashgrid_n_entries.argtypes = [C.POINTER(InpcHashgridDesc), C.POINTER(C.c_int64)]
        L.inpc_query_hashgrid.argtypes = [C.POINTER(InpcHashgridDesc), _P, _P, C.c_int64, _P, _P]
        L.inpc_query_hashgrid_bwd.argtypes = [C.POINTER(InpcHashgridDesc), _P, _P, C.c_int64, _P, _P]
        L.inpc_rasterize_workspace_size.argtypes = [C.POINTER(InpcCamera), C.POINTER(InpcRasterOpts), C.c_int64,
                                                    C.POINTER(C.c_size_t)]
        L.inpc_rasterize_fwd.argtypes = [C.POINTER(InpcCamera), C.POINTER(InpcRasterOpts), _P, _P, _P, C.c_int64,
                                         _P, _P, _P, _P, C.c_size_t, _P]
        L.inpc_rasterize_bwd.argtypes = [C.POINTER(InpcCamera), C.POINTER(InpcRasterOpts), _P, _P, _P, C.c_int64,
                                         _P, _P, _P, _P, _P, _P, C.c_size_t, _P]
        L.inpc_rasterize_bwd_hashgrid_workspace_size.argtypes = [C.POINTER(InpcCamera), C.POINTER(InpcRasterOpts),
                                                                 C.POINTER(InpcHashgridDesc), C.c_int64,
                                                                 C.POINTER(C.c_size_t)]
        L.inpc_rasterize_bwd_hashgrid.argtypes = [C.POINTER(InpcCamera), C.POINTER(InpcRasterOpts),
                                                  C.POINTER(InpcHashgridDesc), _P, _P, C.c_int64, _P, _P, _P, _P, _P,
                                                  _P, C.c_size_t, _P]
        L.inpc_rasterize_point_weights.argtypes = [C.POINTER(InpcCamera), C.POINTER(InpcRasterOpts), _P, C.c_int64,
                                                   _P, _P, _P, C.c_size_t, _P]
        L.inpc_octree_update_workspace_size.argtypes = [C.c_int64, C.POINTER(C.c_size_t)]
        L.inpc_octree_update.argtypes = [_P, _P, C.c_int64, _P, _P, C.c_int64, C.c_double, _P, C.c_size_t, _P]
        L.inpc_octree_refine_workspace_size.argtypes = [C.c_int64, C.POINTER(C.c_size_t)]
        L.inpc_octree_subdivide.argtypes = [C.POINTER(InpcOctree), _P, C.c_double, C.c_int64, _P, _P, _P, _P,
                                            C.c_int64, C.POINTER(C.c_int64), _P, C.c_size_t, _P]
        L.inpc_octree_prune.argtypes = [C.POINTER(InpcOctree), _P, C.c_double, _P, _P, _P, _P, C.c_int64,
                                        C.POINTER(C.c_int64), _P, C.c_size_t, _P]
        L.inpc_view_weights.argtypes = [C.POINTER(InpcOctree), C.POINTER(InpcCamera), C.c_double, C.c_double, _P, _P]
        L.inpc_sample_octree_view.argtypes = [C.POINTER(InpcOctree), C.POINTER(InpcCamera), C.c_uint64, C.c_uint32,
                                              C.c_int64, C.c_int32, _P, _P, _P, _P, C.c_size_t, _P]
        L.inpc_level_weights.argtypes = [C.POINTER(InpcOctree), C.c_double, _P, _P]
        L.inpc_sample_octree_halton.argtypes = [C.POINTER(InpcOctree), C.c_uint64, C.c_int64, _P, _P, _P, _P,
                                                C.c_size_t, _P]
        L.inpc_accumulate_image.argtypes = [_P, C.c_int32, C.c_int64, C.c_float, _P, _P]
        L.inpc_contract_positions.argtypes = [_P, C.c_int64, _P, C.c_float, _P, _P]
        L.inpc_sh_head_fwd.argtypes = [C.POINTER(InpcCamera), _P, _P, C.c_int32, C.c_int64, C.c_int32, _P, _P, _P]
        L.inpc_sh_head_bwd.argtypes = [C.POINTER(InpcCamera), _P, _P, C.c_int32, C.c_int64, C.c_int32, _P, _P, _P,
                                       _P]
        L.inpc_render_batch.argtypes = [C.POINTER(InpcOctree), C.c_uint64, C.POINTER(InpcHashgridDesc), _P,
                                        C.POINTER(InpcViewJob), C.c_int32, _P, C.POINTER(_P), C.c_int32]
        L.inpc_sample_query_batch_workspace_size.argtypes = [C.c_int64, C.c_int32, C.POINTER(C.c_size_t)]
        L.inpc_sample_query_batch.argtypes = [C.POINTER(InpcOctree), C.c_uint64, C.POINTER(InpcHashgridDesc), _P,
                                              C.POINTER(InpcFrontView), C.c_int32, C.c_int64, _P, C.c_size_t, _P]
        L.inpc_render_batch_persistent.argtypes = [C.POINTER(InpcOctree), C.c_uint64, C.POINTER(InpcHashgridDesc),
                                                   _P, C.POINTER(InpcViewJob), C.c_int32, _P, C.POINTER(_P),
                                                   C.c_int32, _P, C.c_size_t, C.c_int64]
        L.inpc_set_fault.argtypes = [C.c_char_p]
        L.inpc_l2_reduction_rate.argtypes = [_P, C.c_int64, C.c_int32, C.POINTER(C.c_double), _P]
        L.inpc_kernel_timer_enable.argtypes = [C.c_int]
        L.inpc_kernel_timer_read.argtypes = [C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        for name in DECLARED:
            if name not in ("inpc_last_error", "inpc_version", "inpc_kernel_launches"):
                getattr(L, name).restype = C.c_int
        _lib = L
        return L


def check(status: int):
    if status != INPC_OK:
        msg = load().inpc_last_error()
        raise InpcError(status, msg.decode() if msg else "")


def version() -> str:
    return load().inpc_version().decode()


def inpc_kernel_launches() -> int:
    return int(load().inpc_kernel_launches())


# --------------------------------------------------- same names as the ABI ---
def inpc_kernel_timer_enable(on: bool) -> bool:
    return bool(load().inpc_kernel_timer_enable(1 if on else 0))


def inpc_kernel_timer_read(kernel=None):
    """(summed device ms, launches) of the recorded launches of `kernel`
    (None: all kernels); the records are consumed."""
    ms, n = C.c_double(0.0), C.c_int64(0)
    check(load().inpc_kernel_timer_read(kernel.encode() if kernel else None, C.byref(ms), C.byref(n)))
    return float(ms.value), int(n.value)


def inpc_read_device_status(workspace: int, stream: int) -> int:
    out = C.c_uint32(0)
    check(load().inpc_read_device_status(workspace, stream, C.byref(out)))
    return int(out.value)


def inpc_sample_workspace_size(n_leaves: int, n_samples: int) -> int:
    out = C.c_size_t(0)
    check(load().inpc_sample_workspace_size(n_leaves, n_samples, C.byref(out)))
    return int(out.value)


def inpc_sample_octree(tree: InpcOctree, seed: int, view_id: int, n_samples: int, leaf_idx_out: int,
                       pos_out: int, leaf_counts_out, workspace: int, workspace_bytes: int, stream: int):
    check(load().inpc_sample_octree(C.byref(tree), C.c_uint64(seed), C.c_uint32(view_id), n_samples, leaf_idx_out,
                                    pos_out, leaf_counts_out, workspace, workspace_bytes, stream))


INPC_SAMPLE_STATIC_SCRATCH_BYTES = (4 << 20) + (576 << 10)


def inpc_sample_octree_noalloc(tree: InpcOctree, seed: int, view_id: int, n_samples: int, leaf_idx_out: int,
                               pos_out: int, leaf_counts_out, stream: int):
    check(load().inpc_sample_octree_noalloc(C.byref(tree), C.c_uint64(seed), C.c_uint32(view_id), n_samples,
                                            leaf_idx_out, pos_out, leaf_counts_out, stream))


def inpc_philox4x32_10(keys: int, ctrs: int, n: int, out: int, stream: int):
    check(load().inpc_philox4x32_10(keys, ctrs, n, out, stream))


def inpc_hashgrid_n_entries(desc: InpcHashgridDesc) -> int:
    out = C.c_int64(0)
    check(load().inpc_hashgrid_n_entries(C.byref(desc), C.byref(out)))
    return int(out.value)


def inpc_query_hashgrid(desc: InpcHashgridDesc, table: int, pos: int, n: int, h_out: int, stream: int):
    check(load().inpc_query_hashgrid(C.byref(desc), table, pos, n, h_out, stream))


def inpc_query_hashgrid_bwd(desc: InpcHashgridDesc, pos: int, dh: int, n: int, grad_table: int, stream: int):
    check(load().inpc_query_hashgrid_bwd(C.byref(desc), pos, dh, n, grad_table, stream))


def inpc_rasterize_workspace_size(cam: InpcCamera, opts: InpcRasterOpts, n: int) -> int:
    out = C.c_size_t(0)
    check(load().inpc_rasterize_workspace_size(C.byref(cam), C.byref(opts), n, C.byref(out)))
    return int(out.value)


def inpc_rasterize_fwd(cam: InpcCamera, opts: InpcRasterOpts, pos: int, opacity, feat: int, n: int, image: int,
                       T_final: int, n_contrib: int, workspace: int, workspace_bytes: int, stream: int):
    check(load().inpc_rasterize_fwd(C.byref(cam), C.byref(opts), pos, opacity, feat, n, image, T_final, n_contrib,
                                    workspace, workspace_bytes, stream))


def inpc_rasterize_bwd(cam: InpcCamera, opts: InpcRasterOpts, pos: int, opacity, feat: int, n: int, T_final: int,
                       n_contrib: int, d_image: int, d_opacity, d_feat: int, workspace: int, workspace_bytes: int,
                       stream: int):
    check(load().inpc_rasterize_bwd(C.byref(cam), C.byref(opts), pos, opacity, feat, n, T_final, n_contrib, d_image,
                                    d_opacity, d_feat, workspace, workspace_bytes, stream))


def inpc_rasterize_bwd_hashgrid_workspace_size(cam: InpcCamera, opts: InpcRasterOpts, desc: InpcHashgridDesc,
                                               n: int) -> int:
    out = C.c_size_t(0)
    check(load().inpc_rasterize_bwd_hashgrid_workspace_size(C.byref(cam), C.byref(opts), C.byref(desc), n,
                                                            C.byref(out)))
    return int(out.value)


def inpc_rasterize_bwd_hashgrid(cam: InpcCamera, opts: InpcRasterOpts, desc: InpcHashgridDesc, pos: int, feat: int,
                                n: int, T_final: int, n_contrib: int, d_image: int, grad_table: int, d_feat,
                                workspace: int, workspace_bytes: int, stream: int):
    check(load().inpc_rasterize_bwd_hashgrid(C.byref(cam), C.byref(opts), C.byref(desc), pos, feat, n, T_final,
                                             n_contrib, d_image, grad_table, d_feat, workspace, workspace_bytes,
                                             stream))


def inpc_rasterize_point_weights(cam: InpcCamera, opts: InpcRasterOpts, pos: int, n: int, n_contrib: int, b_out: int,
                                 workspace: int, workspace_bytes: int, stream: int):
    check(load().inpc_rasterize_point_weights(C.byref(cam), C.byref(opts), pos, n, n_contrib, b_out, workspace,
                                              workspace_bytes, stream))


def inpc_octree_update_workspace_size(n_leaves: int) -> int:
    out = C.c_size_t(0)
    check(load().inpc_octree_update_workspace_size(n_leaves, C.byref(out)))
    return int(out.value)


def inpc_octree_update(leaf_idx: int, b: int, n: int, p: int, q: int, n_leaves: int, lambda_u: float,
                       workspace: int, workspace_bytes: int, stream: int):
    check(load().inpc_octree_update(leaf_idx, b, n, p, q, n_leaves, lambda_u, workspace, workspace_bytes, stream))


def inpc_octree_refine_workspace_size(n_leaves: int) -> int:
    out = C.c_size_t(0)
    check(load().inpc_octree_refine_workspace_size(n_leaves, C.byref(out)))
    return int(out.value)


def inpc_octree_subdivide(tree: InpcOctree, q: int, tau_s: float, max_leaves: int, centers_out: int,
                          levels_out: int, p_out: int, q_out: int, out_capacity: int, workspace: int,
                          workspace_bytes: int, stream: int) -> int:
    n = C.c_int64(0)
    check(load().inpc_octree_subdivide(C.byref(tree), q, tau_s, max_leaves, centers_out, levels_out, p_out, q_out,
                                       out_capacity, C.byref(n), workspace, workspace_bytes, stream))
    return int(n.value)


def inpc_octree_prune(tree: InpcOctree, q: int, tau_p: float, centers_out: int, levels_out: int, p_out: int,
                      q_out: int, out_capacity: int, workspace: int, workspace_bytes: int, stream: int) -> int:
    n = C.c_int64(0)
    check(load().inpc_octree_prune(C.byref(tree), q, tau_p, centers_out, levels_out, p_out, q_out, out_capacity,
                                   C.byref(n), workspace, workspace_bytes, stream))
    return int(n.value)


def inpc_view_weights(tree: InpcOctree, cam: InpcCamera, lambda_l: float, tau_d: float, w_out: int, stream: int):
    check(load().inpc_view_weights(C.byref(tree), C.byref(cam), lambda_l, tau_d, w_out, stream))


def inpc_sample_octree_view(tree: InpcOctree, cam: InpcCamera, seed: int, view_id: int, n_samples: int,
                            max_rounds: int, leaf_idx_out: int, pos_out: int, n_left, workspace: int,
                            workspace_bytes: int, stream: int):
    check(load().inpc_sample_octree_view(C.byref(tree), C.byref(cam), seed, view_id, n_samples, max_rounds,
                                         leaf_idx_out, pos_out, n_left, workspace, workspace_bytes, stream))


def inpc_level_weights(tree: InpcOctree, lambda_l: float, w_out: int, stream: int):
    check(load().inpc_level_weights(C.byref(tree), lambda_l, w_out, stream))


def inpc_sample_octree_halton(tree: InpcOctree, seed: int, n_samples: int, leaf_idx_out: int, pos_out: int,
                              leaf_counts_out, workspace: int, workspace_bytes: int, stream: int):
    check(load().inpc_sample_octree_halton(C.byref(tree), seed, n_samples, leaf_idx_out, pos_out, leaf_counts_out,
                                           workspace, workspace_bytes, stream))


def inpc_accumulate_image(image: int, dtype: int, n_elems: int, scale: float, acc: int, stream: int):
    check(load().inpc_accumulate_image(image, dtype, n_elems, scale, acc, stream))


def inpc_contract_positions(pos: int, n: int, center, radius: float, out: int, stream: int):
    c = (C.c_float * 3)(*[float(x) for x in center])
    check(load().inpc_contract_positions(pos, n, C.cast(c, C.c_void_p), radius, out, stream))


def inpc_sh_head_fwd(cam: InpcCamera, pos: int, h: int, h_dtype: int, n: int, n_channels: int, alpha_out: int,
                     color_out: int, stream: int):
    check(load().inpc_sh_head_fwd(C.byref(cam), pos, h, h_dtype, n, n_channels, alpha_out, color_out, stream))


def inpc_sh_head_bwd(cam: InpcCamera, pos: int, h: int, h_dtype: int, n: int, n_channels: int, d_alpha: int,
                     d_color: int, dh_out: int, stream: int):
    check(load().inpc_sh_head_bwd(C.byref(cam), pos, h, h_dtype, n, n_channels, d_alpha, d_color, dh_out, stream))


def inpc_render_batch(tree: InpcOctree, seed: int, desc: InpcHashgridDesc, table: int, jobs, grad_table,
                      streams):
    """jobs: a sequence of InpcViewJob (or a ctypes array of them); streams:
    raw cudaStream_t handles, streams[0] the origin."""
    arr = jobs if isinstance(jobs, C.Array) else (InpcViewJob * len(jobs))(*jobs)
    st = (_P * len(streams))(*streams)
    check(load().inpc_render_batch(C.byref(tree), seed, C.byref(desc), table, arr, len(arr), grad_table, st,
                                   len(streams)))


def inpc_render_batch_persistent(tree: InpcOctree, seed: int, desc: InpcHashgridDesc, table: int, jobs, grad_table,
                                 streams, front_ws: int, front_ws_bytes: int, max_wait_us: int):
    arr = jobs if isinstance(jobs, C.Array) else (InpcViewJob * len(jobs))(*jobs)
    st = (_P * len(streams))(*streams)
    check(load().inpc_render_batch_persistent(C.byref(tree), seed, C.byref(desc), table, arr, len(arr), grad_table,
                                              st, len(streams), front_ws, front_ws_bytes, max_wait_us))


def inpc_sample_query_batch_workspace_size(n_leaves: int, n_views: int) -> int:
    out = C.c_size_t(0)
    check(load().inpc_sample_query_batch_workspace_size(n_leaves, n_views, C.byref(out)))
    return int(out.value)


def inpc_sample_query_batch(tree: InpcOctree, seed: int, desc: InpcHashgridDesc, table: int, views, max_wait_us: int,
                            workspace: int, workspace_bytes: int, stream: int):
    arr = views if isinstance(views, C.Array) else (InpcFrontView * len(views))(*views)
    check(load().inpc_sample_query_batch(C.byref(tree), C.c_uint64(seed), C.byref(desc), table, arr, len(arr),
                                         max_wait_us, workspace, workspace_bytes, stream))


def inpc_set_fault(spec):
    check(load().inpc_set_fault(spec.encode() if spec else None))


def inpc_l2_reduction_rate(buf: int, rows: int, paired: bool, stream) -> float:
    """Rows reduced per second / 1e9 by 16-byte FP32 vector reductions into
    random rows of the caller's region (calibration for roofline reports)."""
    out = C.c_double(0.0)
    check(load().inpc_l2_reduction_rate(buf, rows, 1 if paired else 0, C.byref(out), stream))
    return float(out.value)
