"""Tile-size autotuner for the rasterizer.

The tile (tile_w x tile_h pixels per CTA of the tile-order blend kernels)
changes only how pixels are grouped into CTAs, never the result.  For a
given image size, sample count, channel count and precision the candidates
are timed on the caller's real inputs (forward plus fused backward, CUDA
events) and the fastest is cached in a JSON file (``INPC_TUNE_CACHE``, by
default ``_lib/tune_cache.json`` beside the library).
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import api

CANDIDATES = [(16, 8), (8, 8), (16, 16), (32, 8), (32, 4)]
_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("INPC_TUNE_CACHE",
                          os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "tune_cache.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(cache: dict):
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def key_for(cam, opts, n: int) -> str:
    return "%dx%d:n%d:F%d:%s:%s" % (cam.width, cam.height, n, opts.n_channels, "bf16" if opts.bf16 else "f32",
                                    torch.cuda.get_device_name())


def tuned_tiles(cam, opts, desc, pos, feat, d_image, reps: int = 3):
    """Best (tile_w, tile_h) for this problem shape; times the candidates on
    first use and caches the choice."""
    n = pos.shape[0]
    key = key_for(cam, opts, n)
    with _lock:
        cache = _load()
        if key in cache:
            return tuple(cache[key])
    ws = api.workspace(api.rasterize_bwd_hashgrid_workspace_size(cam, opts, desc, n), pos.device)
    gt = torch.zeros(api.hashgrid_n_entries([desc.res[i] for i in range(desc.n_levels)], desc.log2_T), 4,
                     dtype=torch.float32, device=pos.device)
    best, best_ms = None, float("inf")
    timings = {}
    for tw, th in CANDIDATES:
        o = api.RasterOptions(n_channels=opts.n_channels, head_mode=opts.head_mode, t_min=opts.t_min,
                              alpha_max=opts.alpha_max, tile_w=tw, tile_h=th, bf16=opts.bf16)
        img, T, nc, ws = api.rasterize_fwd(cam, o, pos, feat, None, ws=ws)
        api.rasterize_bwd_hashgrid(cam, o, desc, pos, feat, T, nc, d_image, ws, gt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            img, T, nc, ws = api.rasterize_fwd(cam, o, pos, feat, None, ws=ws, out=(img, T, nc))
            api.rasterize_bwd_hashgrid(cam, o, desc, pos, feat, T, nc, d_image, ws, gt)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        timings["%dx%d" % (tw, th)] = ms
        if ms < best_ms:
            best, best_ms = (tw, th), ms
    with _lock:
        cache = _load()
        cache[key] = list(best)
        cache[key + ":timings_ms"] = timings
        _save(cache)
    return best
