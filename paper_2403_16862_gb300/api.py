"""Torch-facing entry points of the INPC hot path.

PyTorch supplies device memory and the current stream; every computation
runs in ``libinpc.so`` through the C ABI (``_binding``).  All tensors must be
CUDA tensors, contiguous, of the documented dtype.  There is no CPU path.

Functions:
  sample_octree       -- Sec. 3.2 sampling (leaf indices grouped by leaf, positions)
  query_hashgrid      -- Sec. 3.3 multi-resolution grid query
  query_hashgrid_bwd  -- its adjoint (FP32 table gradient, accumulated)
  rasterize_fwd/bwd   -- Sec. 3.4 / Algorithm 1 bilinear point rasterizer
  HashGridQuery, Rasterize -- torch.autograd.Function wrappers
  render_view         -- one view: sample -> query -> rasterize (head mode)
"""
from __future__ import annotations

import dataclasses

import torch

from . import _binding as B


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _need(t, dtype, name, device=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


def workspace(nbytes: int, device) -> torch.Tensor:
    """Caller-owned work buffer (torch allocations are 512-byte aligned)."""
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def read_device_status(ws: torch.Tensor) -> int:
    return B.inpc_read_device_status(ws.data_ptr(), _stream())


# ---------------------------------------------------------------- sampling ---
def sample_octree(centers, levels, weights, root_size: float, seed: int, view_id: int, n_samples: int,
                  ws: torch.Tensor | None = None, out=None, with_counts: bool = False):
    """Returns (leaf_idx int32 [N], pos float32 [N,3][, counts int32 [L]])."""
    _need(centers, torch.float32, "centers")
    _need(levels, torch.int32, "levels")
    _need(weights, torch.float64, "weights")
    L = levels.shape[0]
    dev = centers.device
    need = B.inpc_sample_workspace_size(L, n_samples)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    if out is None:
        leaf = torch.empty(n_samples, dtype=torch.int32, device=dev)
        pos = torch.empty(n_samples, 3, dtype=torch.float32, device=dev)
    else:
        leaf, pos = out
    counts = torch.empty(L, dtype=torch.int32, device=dev) if with_counts else None
    tree = B.InpcOctree(_ptr(centers), _ptr(levels), _ptr(weights), float(root_size), L)
    B.inpc_sample_octree(tree, seed, view_id, n_samples, _ptr(leaf), _ptr(pos), _ptr(counts), ws.data_ptr(),
                         ws.numel(), _stream())
    return (leaf, pos, counts) if with_counts else (leaf, pos)


# --------------------------------------------------------------- hash grid ---
def hashgrid_desc(res, log2_T: int, n_feats: int = 4, table_dtype=torch.float32,
                  out_dtype=torch.float32) -> B.InpcHashgridDesc:
    d = B.InpcHashgridDesc()
    d.n_levels = len(res)
    d.n_feats = n_feats
    d.log2_T = log2_T
    for i, r in enumerate(res):
        d.res[i] = int(r)
    d.table_dtype = B.INPC_BF16 if table_dtype == torch.bfloat16 else B.INPC_F32
    d.out_dtype = B.INPC_BF16 if out_dtype == torch.bfloat16 else B.INPC_F32
    return d


def hashgrid_n_entries(res, log2_T: int, n_feats: int = 4) -> int:
    return B.inpc_hashgrid_n_entries(hashgrid_desc(res, log2_T, n_feats))


def _torch_dtype(code):
    return torch.bfloat16 if code == B.INPC_BF16 else torch.float32


def query_hashgrid(desc: B.InpcHashgridDesc, table, pos, out=None):
    _need(table, _torch_dtype(desc.table_dtype), "table")
    _need(pos, torch.float32, "pos")
    n = pos.shape[0]
    C = desc.n_levels * desc.n_feats
    h = out if out is not None else torch.empty(n, C, dtype=_torch_dtype(desc.out_dtype), device=pos.device)
    B.inpc_query_hashgrid(desc, table.data_ptr(), pos.data_ptr(), n, h.data_ptr(), _stream())
    return h


def query_hashgrid_bwd(desc: B.InpcHashgridDesc, pos, dh, grad_table):
    _need(pos, torch.float32, "pos")
    _need(dh, torch.float32, "dh")
    _need(grad_table, torch.float32, "grad_table")
    B.inpc_query_hashgrid_bwd(desc, pos.data_ptr(), dh.data_ptr(), pos.shape[0], grad_table.data_ptr(), _stream())
    return grad_table


# -------------------------------------------------------------- rasterizer ---
def camera(cam) -> B.InpcCamera:
    """C camera struct from an object with R, t, fx, fy, cx, cy, width, height, near, far."""
    c = B.InpcCamera()
    R = [float(x) for x in torch.as_tensor(cam.R, dtype=torch.float32).reshape(9).tolist()]
    t = [float(x) for x in torch.as_tensor(cam.t, dtype=torch.float32).reshape(3).tolist()]
    for i in range(9):
        c.R[i] = R[i]
    for i in range(3):
        c.t[i] = t[i]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.near_plane, c.far_plane = float(cam.near), float(cam.far)
    return c


@dataclasses.dataclass
class RasterOptions:
    n_channels: int
    head_mode: bool = False
    t_min: float = 1e-4
    alpha_max: float = 0.99
    tile_w: int = 0
    tile_h: int = 0
    bf16: bool = False  # BF16 feature rows and image (FP32 arithmetic and gradients)

    @property
    def dtype(self):
        return torch.bfloat16 if self.bf16 else torch.float32

    def c(self) -> B.InpcRasterOpts:
        o = B.InpcRasterOpts()
        o.opacity_mode = B.INPC_OPACITY_FROM_CH0 if self.head_mode else B.INPC_OPACITY_GIVEN
        o.n_channels = self.n_channels
        o.feat_dtype = B.INPC_BF16 if self.bf16 else B.INPC_F32
        o.image_dtype = o.feat_dtype
        o.t_min = self.t_min
        o.alpha_max = self.alpha_max
        o.tile_w = self.tile_w
        o.tile_h = self.tile_h
        return o


def rasterize_workspace_size(cam, opts: RasterOptions, n: int) -> int:
    return B.inpc_rasterize_workspace_size(camera(cam), opts.c(), n)


def rasterize_fwd(cam, opts: RasterOptions, pos, feat, opacity=None, ws=None, out=None):
    """Returns (image [H,W,F], T_final [H,W], n_contrib [H,W], ws)."""
    _need(pos, torch.float32, "pos")
    _need(feat, opts.dtype, "feat")
    if opacity is not None:
        _need(opacity, torch.float32, "opacity")
    n = pos.shape[0]
    cc, oc = camera(cam), opts.c()
    need = B.inpc_rasterize_workspace_size(cc, oc, n)
    if ws is None or ws.numel() < need:
        ws = workspace(need, pos.device)
    H, W, F = cam.height, cam.width, opts.n_channels
    if out is None:
        image = torch.empty(H, W, F, dtype=opts.dtype, device=pos.device)
        T_final = torch.empty(H, W, dtype=torch.float32, device=pos.device)
        n_contrib = torch.empty(H, W, dtype=torch.int32, device=pos.device)
    else:
        image, T_final, n_contrib = out
    B.inpc_rasterize_fwd(cc, oc, pos.data_ptr(), _ptr(opacity), feat.data_ptr(), n, image.data_ptr(),
                         T_final.data_ptr(), n_contrib.data_ptr(), ws.data_ptr(), ws.numel(), _stream())
    return image, T_final, n_contrib, ws


def rasterize_bwd(cam, opts: RasterOptions, pos, feat, opacity, T_final, n_contrib, d_image, ws, out=None):
    """Returns (d_opacity [N] or None, d_feat [N,F])."""
    _need(d_image, torch.float32, "d_image")
    n = pos.shape[0]
    if out is None:
        d_feat = torch.empty(feat.shape, dtype=torch.float32, device=feat.device)
        d_opacity = None if opts.head_mode else torch.empty(n, dtype=torch.float32, device=pos.device)
    else:
        d_opacity, d_feat = out
    B.inpc_rasterize_bwd(camera(cam), opts.c(), pos.data_ptr(), _ptr(opacity), feat.data_ptr(), n,
                         T_final.data_ptr(), n_contrib.data_ptr(), d_image.data_ptr(), _ptr(d_opacity),
                         d_feat.data_ptr(), ws.data_ptr(), ws.numel(), _stream())
    return d_opacity, d_feat


def rasterize_bwd_hashgrid_workspace_size(cam, opts: RasterOptions, desc, n: int) -> int:
    """Workspace for rasterize_fwd followed by rasterize_bwd_hashgrid."""
    return B.inpc_rasterize_bwd_hashgrid_workspace_size(camera(cam), opts.c(), desc, n)


def rasterize_bwd_hashgrid(cam, opts: RasterOptions, desc, pos, feat, T_final, n_contrib, d_image, ws, grad_table,
                           d_feat=None):
    """Head-mode rasterizer backward fused with the grid query's adjoint:
    accumulates the table gradient (FP32) directly; d_feat is written only
    when given."""
    _need(d_image, torch.float32, "d_image")
    _need(grad_table, torch.float32, "grad_table")
    B.inpc_rasterize_bwd_hashgrid(camera(cam), opts.c(), desc, pos.data_ptr(), feat.data_ptr(), pos.shape[0],
                                  T_final.data_ptr(), n_contrib.data_ptr(), d_image.data_ptr(), grad_table.data_ptr(),
                                  _ptr(d_feat), ws.data_ptr(), ws.numel(), _stream())
    return grad_table


# ---------------------------------------------------------------- autograd ---
class HashGridQuery(torch.autograd.Function):
    """h = query(table, pos); gradient flows to the table (FP32)."""

    @staticmethod
    def forward(ctx, table, pos, desc):
        ctx.desc = desc
        ctx.save_for_backward(pos)
        ctx.table_shape = table.shape
        return query_hashgrid(desc, table, pos)

    @staticmethod
    def backward(ctx, dh):
        (pos,) = ctx.saved_tensors
        grad = torch.zeros(ctx.table_shape, dtype=torch.float32, device=pos.device)
        query_hashgrid_bwd(ctx.desc, pos, dh.float().contiguous(), grad)
        return grad, None, None


class Rasterize(torch.autograd.Function):
    """image = rasterize(pos, feat[, opacity]); gradients to feat and opacity."""

    @staticmethod
    def forward(ctx, pos, feat, opacity, cam, opts):
        image, T_final, n_contrib, ws = rasterize_fwd(cam, opts, pos, feat, opacity)
        ctx.cam, ctx.opts = cam, opts
        ctx.save_for_backward(pos, feat, opacity if opacity is not None else torch.empty(0, device=pos.device),
                              T_final, n_contrib, ws)
        ctx.has_opacity = opacity is not None
        ctx.mark_non_differentiable(T_final, n_contrib)
        return image, T_final, n_contrib

    @staticmethod
    def backward(ctx, d_image, _dT, _dn):
        pos, feat, opacity, T_final, n_contrib, ws = ctx.saved_tensors
        op = opacity if ctx.has_opacity else None
        d_op, d_feat = rasterize_bwd(ctx.cam, ctx.opts, pos, feat, op, T_final, n_contrib,
                                     d_image.contiguous(), ws)
        return None, d_feat, d_op, None, None


def render_view(tree_t, root_size, desc, table, cam, seed, view_id, n_samples, opts=None):
    """Differentiable single-view pass of the hot path: sample points from
    the octree, query the grid (head mode: channel 0 -> opacity), rasterize.
    ``tree_t`` = (centers, levels, weights) CUDA tensors."""
    centers, levels, weights = tree_t
    _, pos = sample_octree(centers, levels, weights, root_size, seed, view_id, n_samples)
    h = HashGridQuery.apply(table, pos, desc)
    if opts is None:
        opts = RasterOptions(n_channels=desc.n_levels * desc.n_feats, head_mode=True)
    image, T_final, n_contrib = Rasterize.apply(pos, h, None, cam, opts)
    return image, T_final, n_contrib, pos


# ------------------------------------------------------ octree maintenance ---
def point_weights(cam, opts: RasterOptions, pos, n_contrib, ws, out=None):
    """Per-point blending weights b [N] (float32) of the forward that used
    ``ws`` and produced ``n_contrib`` (Sec. 3.1 Eq. 2 / App. A.6)."""
    n = pos.shape[0]
    b = out if out is not None else torch.empty(n, dtype=torch.float32, device=pos.device)
    _need(n_contrib, torch.int32, "n_contrib")
    B.inpc_rasterize_point_weights(camera(cam), opts.c(), _ptr(pos), n, _ptr(n_contrib), _ptr(b), ws.data_ptr(),
                                   ws.numel(), _stream())
    return b


def octree_update(leaf_idx, b, p, q, lambda_u: float = 0.9968, ws=None):
    """Eq. 2 / Eq. 3 in place on p, q (float64 [L]) from the points' leaves
    and blending weights."""
    _need(leaf_idx, torch.int32, "leaf_idx")
    _need(b, torch.float32, "b")
    _need(p, torch.float64, "p")
    _need(q, torch.float64, "q")
    L = p.shape[0]
    need = B.inpc_octree_update_workspace_size(L)
    if ws is None or ws.numel() < need:
        ws = workspace(need, p.device)
    B.inpc_octree_update(_ptr(leaf_idx), _ptr(b), leaf_idx.shape[0], _ptr(p), _ptr(q), L, float(lambda_u),
                         ws.data_ptr(), ws.numel(), _stream())
    return p, q


def _refine(fn, centers, levels, p, q, root_size, cap, *args):
    _need(centers, torch.float32, "centers")
    _need(levels, torch.int32, "levels")
    _need(p, torch.float64, "p")
    _need(q, torch.float64, "q")
    L = levels.shape[0]
    dev = centers.device
    co = torch.empty(cap, 3, dtype=torch.float32, device=dev)
    lo = torch.empty(cap, dtype=torch.int32, device=dev)
    po = torch.empty(cap, dtype=torch.float64, device=dev)
    qo = torch.empty(cap, dtype=torch.float64, device=dev)
    ws = workspace(B.inpc_octree_refine_workspace_size(L), dev)
    tree = B.InpcOctree(_ptr(centers), _ptr(levels), _ptr(p), float(root_size), L)
    n = fn(tree, _ptr(q), *args, _ptr(co), _ptr(lo), _ptr(po), _ptr(qo), cap, ws.data_ptr(), ws.numel(), _stream())
    return co[:n], lo[:n], po[:n], qo[:n]


def octree_subdivide(centers, levels, p, q, root_size: float, tau_s: float = 0.5, max_leaves: int = 256 ** 3):
    """Sec. 3.1 subdivision; returns the new (centers, levels, p, q)."""
    return _refine(B.inpc_octree_subdivide, centers, levels, p, q, root_size, 8 * levels.shape[0], float(tau_s),
                   int(max_leaves))


def octree_prune(centers, levels, p, q, root_size: float, tau_p: float = 0.01):
    """Sec. 3.1 pruning; returns the kept (centers, levels, p, q)."""
    return _refine(B.inpc_octree_prune, centers, levels, p, q, root_size, levels.shape[0], float(tau_p))


# -------------------------------------------------- view-specific sampling ---
def view_weights(centers, levels, p, root_size: float, cam, lambda_l: float = 0.5, tau_d: float = 1e-8, out=None):
    """Eq. 4 view-specific leaf weights (float64 [L])."""
    _need(centers, torch.float32, "centers")
    _need(levels, torch.int32, "levels")
    _need(p, torch.float64, "p")
    L = levels.shape[0]
    w = out if out is not None else torch.empty(L, dtype=torch.float64, device=p.device)
    tree = B.InpcOctree(_ptr(centers), _ptr(levels), _ptr(p), float(root_size), L)
    B.inpc_view_weights(tree, camera(cam), float(lambda_l), float(tau_d), _ptr(w), _stream())
    return w


def sample_octree_view(centers, levels, view_w, root_size: float, cam, seed: int, view_id: int, n_samples: int,
                       max_rounds: int = 8, ws=None, out=None):
    """Sampling from the view weights with the re-sampling rounds of App. A.4;
    returns (leaf_idx, pos, n_left) with n_left a device int32 scalar."""
    _need(centers, torch.float32, "centers")
    _need(levels, torch.int32, "levels")
    _need(view_w, torch.float64, "view weights")
    L = levels.shape[0]
    dev = centers.device
    need = B.inpc_sample_workspace_size(L, n_samples)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    if out is None:
        leaf = torch.empty(n_samples, dtype=torch.int32, device=dev)
        pos = torch.empty(n_samples, 3, dtype=torch.float32, device=dev)
    else:
        leaf, pos = out
    n_left = torch.zeros(1, dtype=torch.int32, device=dev)
    tree = B.InpcOctree(_ptr(centers), _ptr(levels), _ptr(view_w), float(root_size), L)
    B.inpc_sample_octree_view(tree, camera(cam), seed, view_id, n_samples, int(max_rounds), _ptr(leaf), _ptr(pos),
                              _ptr(n_left), ws.data_ptr(), ws.numel(), _stream())
    return leaf, pos, n_left


# ---------------------------------------------------------- pre-extraction ---
def level_weights(levels, p, lambda_l: float = 0.5, out=None):
    """Eq. 4 without visibility and depth: p / 2^(l lambda_l) (float64 [L])."""
    _need(levels, torch.int32, "levels")
    _need(p, torch.float64, "p")
    L = levels.shape[0]
    w = out if out is not None else torch.empty(L, dtype=torch.float64, device=p.device)
    tree = B.InpcOctree(None, _ptr(levels), _ptr(p), 1.0, L)
    B.inpc_level_weights(tree, float(lambda_l), _ptr(w), _stream())
    return w


def sample_octree_halton(centers, levels, weights, root_size: float, seed: int, n_samples: int, ws=None, out=None):
    """Viewpoint-independent pre-extraction: (leaf_idx int32 [N], pos float32 [N,3])."""
    _need(centers, torch.float32, "centers")
    _need(levels, torch.int32, "levels")
    _need(weights, torch.float64, "weights")
    L = levels.shape[0]
    dev = centers.device
    need = B.inpc_sample_workspace_size(L, n_samples)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    if out is None:
        leaf = torch.empty(n_samples, dtype=torch.int32, device=dev)
        pos = torch.empty(n_samples, 3, dtype=torch.float32, device=dev)
    else:
        leaf, pos = out
    tree = B.InpcOctree(_ptr(centers), _ptr(levels), _ptr(weights), float(root_size), L)
    B.inpc_sample_octree_halton(tree, seed, n_samples, _ptr(leaf), _ptr(pos), None, ws.data_ptr(), ws.numel(),
                                _stream())
    return leaf, pos


def accumulate_image(image, acc, scale: float):
    """acc += scale * image (FP32 accumulator; image FP32 or BF16)."""
    _need(acc, torch.float32, "acc")
    if image.shape != acc.shape or not image.is_contiguous():
        raise ValueError("image and acc must have the same shape (contiguous)")
    dt = B.INPC_BF16 if image.dtype == torch.bfloat16 else B.INPC_F32
    if dt == B.INPC_F32:
        _need(image, torch.float32, "image")
    B.inpc_accumulate_image(image.data_ptr(), dt, image.numel(), float(scale), _ptr(acc), _stream())
    return acc


def multisample_render(tree_t, root_size: float, desc, table, cam, seed: int, n_samples: int, k: int = 4,
                       opts=None, lambda_l: float = 0.5, max_rounds: int = 8):
    """Inference multisampling (Sec. 3.2): k view-specific point clouds (view
    ids 0..k-1 of this seed), each queried and rasterized, their feature
    images averaged per pixel.  Returns the FP32 average image."""
    c, l, p = tree_t
    opts = opts or RasterOptions(n_channels=desc.n_levels * desc.n_feats, head_mode=True)
    w = view_weights(c, l, p, root_size, cam, lambda_l=lambda_l)
    acc = torch.zeros(cam.height, cam.width, opts.n_channels, dtype=torch.float32, device=c.device)
    ws_r = None
    for v in range(k):
        _, pos, _ = sample_octree_view(c, l, w, root_size, cam, seed, v, n_samples, max_rounds=max_rounds)
        h = query_hashgrid(desc, table, pos)
        img, _, _, ws_r = rasterize_fwd(cam, opts, pos, h, ws=ws_r)
        accumulate_image(img, acc, 1.0 / k)
    return acc


# ------------------------------------------------------ view-dependent head ---
def contract_positions(pos, center, radius: float, out=None):
    """Spherical contraction into [0, 1]^3 (the grid query's domain)."""
    _need(pos, torch.float32, "pos")
    o = out if out is not None else torch.empty_like(pos)
    B.inpc_contract_positions(_ptr(pos), pos.shape[0], center, float(radius), _ptr(o), _stream())
    return o


def sh_head_fwd(cam, pos, h):
    """(alpha_h float32 [N], color float32 [N,4]) of the degree-2 SH head."""
    n, F = h.shape
    dt = B.INPC_BF16 if h.dtype == torch.bfloat16 else B.INPC_F32
    alpha = torch.empty(n, dtype=torch.float32, device=h.device)
    color = torch.empty(n, 4, dtype=torch.float32, device=h.device)
    B.inpc_sh_head_fwd(camera(cam), _ptr(pos), h.data_ptr(), dt, n, F, _ptr(alpha), _ptr(color), _stream())
    return alpha, color


def sh_head_bwd(cam, pos, h, d_alpha, d_color):
    """dh float32 [N, F] of the SH head."""
    n, F = h.shape
    dt = B.INPC_BF16 if h.dtype == torch.bfloat16 else B.INPC_F32
    dh = torch.empty(n, F, dtype=torch.float32, device=h.device)
    B.inpc_sh_head_bwd(camera(cam), _ptr(pos), h.data_ptr(), dt, n, F, _ptr(d_alpha), _ptr(d_color), _ptr(dh),
                       _stream())
    return dh


def render_view_sh(pos, desc, table, cam, center, radius: float, d_image=None, grad_table=None):
    """The view-dependent variant of the path: contraction -> grid query ->
    SH head -> rasterizer (4 channels, given opacities); with d_image also the
    backward into grad_table.  Returns (image, T_final, n_contrib)."""
    q = contract_positions(pos, center, radius)
    h = query_hashgrid(desc, table, q)
    alpha, color = sh_head_fwd(cam, pos, h)
    opts = RasterOptions(n_channels=4, head_mode=False)
    img, T, nc, ws = rasterize_fwd(cam, opts, pos, color, alpha)
    if d_image is not None:
        d_op, d_col = rasterize_bwd(cam, opts, pos, color, alpha, T, nc, d_image, ws)
        dh = sh_head_bwd(cam, pos, h, d_op, d_col)
        query_hashgrid_bwd(desc, q, dh, grad_table)
    return img, T, nc
