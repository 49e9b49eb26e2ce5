"""Seeded synthetic inputs for the INPC hot path.

This module only *generates inputs*: octrees (leaf centers, levels, weights),
hash-grid descriptors and tables, point clouds, cameras and upstream
gradients.  It holds none of the method's arithmetic (no sampling, no hashing,
no projection, no blending), so both the CUDA path and the CPU oracle can be
fed from it without sharing any computation.

The workloads stand in for the paper's unbounded-scene datasets
(Mip-NeRF 360 and Tanks and Temples, Sec. 4.1), which are not available:

* ``raster_points_scene``: points uniform in [-1, 1]^3, opacity ~ U(0.05, 0.95),
  features ~ N(0, 1), camera at (0, 0, -3) looking down +z (the plain
  rasterizer workload, 65,536 points at 256x256).
* ``octree_scene``: a sparse octree in the unit cube built like the paper's
  octree after refinement (uniform start grid as in App. A.4 "Initialization",
  then random subdivision and pruning as in Sec. 3.1), log-normal(0, 1.5)
  leaf weights, and a 16-level hash grid (Sec. 3.3, App. A.5) with entries
  U(-1e-4, 1e-4) + N(0, 0.1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Octree", "HashGrid", "Camera", "RasterPoints",
    "geometric_resolutions", "make_octree", "make_hashgrid", "make_camera",
    "look_at_camera", "raster_points_scene", "octree_scene", "orbit_cameras",
    "morton3", "upstream_grad",
]


@dataclasses.dataclass
class Octree:
    """Leaf arrays of a sparse point-probability octree (Sec. 3.1, App. A.4).

    centers: float32 [L, 3] world-space leaf centers.
    levels:  int32 [L] subdivision level; a level-l leaf has edge
             root_size * 2**-l.
    weights: float64 [L] non-negative sampling weights (the p_i of Sec. 3.1).
    """
    centers: np.ndarray
    levels: np.ndarray
    weights: np.ndarray
    root_size: float

    @property
    def n_leaves(self) -> int:
        return int(self.levels.shape[0])


@dataclasses.dataclass
class HashGrid:
    """Multi-resolution grid description plus its parameter table.

    res:   per-level grid resolutions (host integers, level 0 coarsest).
    log2_T: log2 of the per-level entry budget.
    n_feats: features per level.
    table: float32 [n_entries, n_feats]; the level-major concatenation of
           every level's entries.  ``n_entries`` is supplied by the caller's
           layout rule through ``entries_per_level``.
    """
    res: list
    log2_T: int
    n_feats: int
    table: np.ndarray

    @property
    def n_levels(self) -> int:
        return len(self.res)


@dataclasses.dataclass
class Camera:
    """Pinhole camera: world->camera rotation R (row-major 3x3) and
    translation t (x_cam = R @ x_world + t), focal lengths, principal point
    and image size in pixels.  near/far are the paper's planes (App. A.2)."""
    R: np.ndarray
    t: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.01
    far: float = 100.0


@dataclasses.dataclass
class RasterPoints:
    pos: np.ndarray       # float32 [N, 3]
    opacity: np.ndarray   # float32 [N]
    feat: np.ndarray      # float32 [N, F]


def geometric_resolutions(n_levels: int, base: int, finest: int) -> list:
    """Per-level grid resolutions growing geometrically from ``base`` to
    ``finest`` (the configuration space of Listing 1 in App. A.5: base
    resolution and per-level scale).  Returned as host integers so that
    every consumer works from identical values."""
    if n_levels == 1:
        return [int(base)]
    b = (finest / base) ** (1.0 / (n_levels - 1))
    return [int(math.floor(base * b ** l + 1e-9)) for l in range(n_levels)]


def morton3(ix: np.ndarray, iy: np.ndarray, iz: np.ndarray, bits: int) -> np.ndarray:
    """Interleave the low ``bits`` bits of three integer coordinates (Morton
    order), used only to lay leaves out in a spatially coherent order."""
    code = np.zeros(ix.shape, dtype=np.uint64)
    for b in range(bits):
        code |= ((ix.astype(np.uint64) >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
        code |= ((iy.astype(np.uint64) >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + 1)
        code |= ((iz.astype(np.uint64) >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + 2)
    return code


def make_octree(seed: int, n_leaves: int, start_level: int = 4, max_level: int = 12,
                root_size: float = 1.0, origin=(0.0, 0.0, 0.0),
                weight_sigma: float = 1.5) -> Octree:
    """Sparse octree with exactly ``n_leaves`` leaves in the cube
    origin + [0, root_size]^3.

    Start from the uniform (2**start_level)^3 grid of level-``start_level``
    leaves, subdivide uniformly chosen leaves of level < ``max_level`` until
    there are at least ``n_leaves``, then prune uniformly chosen leaves down
    to exactly ``n_leaves`` (a complete octree never has exactly 2**16
    leaves, since subdivision adds 7 at a time).  Leaves are returned in
    Morton order of their minimum corner at ``max_level`` resolution.
    Weights are log-normal(0, weight_sigma), normalised to sum to one.
    """
    rng = np.random.default_rng(seed)
    g = 1 << start_level
    ii = np.arange(g, dtype=np.int64)
    ix, iy, iz = np.meshgrid(ii, ii, ii, indexing="ij")
    ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
    lv = np.full(ix.shape, start_level, dtype=np.int64)
    while ix.size < n_leaves:
        need = n_leaves - ix.size
        eligible = np.nonzero(lv < max_level)[0]
        if eligible.size == 0:
            raise ValueError("octree cannot reach the requested leaf count")
        # small batches approximate one-leaf-at-a-time refinement, which
        # spreads leaves over many levels
        k = min(eligible.size, max(1, need // 48))
        pick = rng.choice(eligible, size=k, replace=False)
        keep = np.ones(ix.size, dtype=bool)
        keep[pick] = False
        cx, cy, cz, cl = ix[pick], iy[pick], iz[pick], lv[pick]
        ch = []
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    ch.append((2 * cx + dx, 2 * cy + dy, 2 * cz + dz, cl + 1))
        ix = np.concatenate([ix[keep]] + [c[0] for c in ch])
        iy = np.concatenate([iy[keep]] + [c[1] for c in ch])
        iz = np.concatenate([iz[keep]] + [c[2] for c in ch])
        lv = np.concatenate([lv[keep]] + [c[3] for c in ch])
    if ix.size > n_leaves:
        keep_idx = np.sort(rng.choice(ix.size, size=n_leaves, replace=False))
        ix, iy, iz, lv = ix[keep_idx], iy[keep_idx], iz[keep_idx], lv[keep_idx]
    shift = (max_level - lv).astype(np.uint64)
    code = morton3(ix.astype(np.uint64) << shift, iy.astype(np.uint64) << shift,
                   iz.astype(np.uint64) << shift, max_level)
    order = np.argsort(code, kind="stable")
    ix, iy, iz, lv = ix[order], iy[order], iz[order], lv[order]
    edge = root_size * np.exp2(-lv.astype(np.float64))
    o = np.asarray(origin, dtype=np.float64)
    centers = np.stack([o[0] + (ix + 0.5) * edge, o[1] + (iy + 0.5) * edge,
                        o[2] + (iz + 0.5) * edge], axis=1).astype(np.float32)
    w = rng.lognormal(mean=0.0, sigma=weight_sigma, size=ix.size)
    w = w / w.sum()
    return Octree(centers=centers, levels=lv.astype(np.int32), weights=w.astype(np.float64),
                  root_size=float(root_size))


def make_hashgrid(seed: int, n_entries: int, res: list, log2_T: int, n_feats: int = 4) -> HashGrid:
    """Hash-grid parameter table with entries U(-1e-4, 1e-4) + N(0, 0.1).

    ``n_entries`` is the total row count of the level-major table; the layout
    rule that determines it belongs to the grid implementation, not to this
    generator.
    """
    rng = np.random.default_rng(seed)
    tab = rng.uniform(-1e-4, 1e-4, size=(n_entries, n_feats)) + rng.normal(0.0, 0.1, size=(n_entries, n_feats))
    return HashGrid(res=list(res), log2_T=int(log2_T), n_feats=int(n_feats), table=tab.astype(np.float32))


def make_camera(position, fx, fy, cx, cy, width, height, R=None, near=0.01, far=100.0) -> Camera:
    """Camera at world ``position`` with world->camera rotation ``R``
    (identity: looks down +z with image y pointing down)."""
    R = np.eye(3, dtype=np.float64) if R is None else np.asarray(R, dtype=np.float64)
    p = np.asarray(position, dtype=np.float64)
    t = -R @ p
    return Camera(R=R.astype(np.float32), t=t.astype(np.float32), fx=float(fx), fy=float(fy),
                  cx=float(cx), cy=float(cy), width=int(width), height=int(height),
                  near=float(near), far=float(far))


def look_at_camera(eye, target, fx, fy, cx, cy, width, height, up=(0.0, -1.0, 0.0)) -> Camera:
    """Camera at ``eye`` whose +z axis points at ``target`` and whose image
    y axis points along ``up`` projected (default: world -y is image up)."""
    eye = np.asarray(eye, dtype=np.float64)
    z = np.asarray(target, dtype=np.float64) - eye
    z /= np.linalg.norm(z)
    upv = -np.asarray(up, dtype=np.float64)
    x = np.cross(upv, z)
    if np.linalg.norm(x) < 1e-9:
        x = np.cross(np.array([1.0, 0.0, 0.0]), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], axis=0)
    return make_camera(eye, fx, fy, cx, cy, width, height, R=R)


def raster_points_scene(seed: int = 0, n: int = 65536, n_feat: int = 8, size: int = 256,
                        focal: float = 256.0) -> tuple:
    """Points uniform in [-1,1]^3 with opacity ~ U(0.05, 0.95) and N(0,1)
    features, seen by a camera at (0,0,-3) looking at the origin."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)
    opacity = rng.uniform(0.05, 0.95, size=n).astype(np.float32)
    feat = rng.normal(0.0, 1.0, size=(n, n_feat)).astype(np.float32)
    cam = make_camera((0.0, 0.0, -3.0), focal, focal, size / 2.0, size / 2.0, size, size)
    return RasterPoints(pos=pos, opacity=opacity, feat=feat), cam


def octree_scene(seed: int = 0, n_leaves: int = 65536, start_level: int = 4,
                 log2_T: int = 19, n_levels: int = 16, base_res: int = 16,
                 finest_res: int = 4096, n_feats: int = 4, entries_fn=None):
    """Octree in the unit cube plus a hash grid; ``entries_fn(res, log2_T)``
    returns the table row count (supplied by the grid implementation)."""
    tree = make_octree(seed, n_leaves, start_level=start_level)
    res = geometric_resolutions(n_levels, base_res, finest_res)
    n_entries = entries_fn(res, log2_T) if entries_fn is not None else None
    grid = make_hashgrid(seed + 1, n_entries, res, log2_T, n_feats) if n_entries is not None else None
    return tree, res, grid


def orbit_cameras(sizes, radius: float = 1.7, center=(0.5, 0.5, 0.5), focal_ref: float = 900.0,
                  ref_height: int = 832) -> list:
    """Cameras on a horizontal orbit around ``center``, one per (W, H),
    focal length scaled with the image height."""
    cams = []
    c = np.asarray(center, dtype=np.float64)
    for k, (w, h) in enumerate(sizes):
        a = 2.0 * math.pi * k / len(sizes)
        eye = c + radius * np.array([math.sin(a), -0.25, -math.cos(a)])
        f = focal_ref * h / ref_height
        cams.append(look_at_camera(eye, c, f, f, w / 2.0, h / 2.0, w, h))
    return cams


def upstream_grad(seed: int, shape) -> np.ndarray:
    """Upstream gradient ~ N(0, 1) (the d_image of the differentiation workload)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 1.0, size=shape).astype(np.float32)
