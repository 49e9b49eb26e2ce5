#!/usr/bin/env python3
"""Benchmark of the INPC hot path on GB300: one step = one view, forward and
backward through the whole path (octree sampling -> hash-grid query ->
bilinear rasterizer forward -> rasterizer backward -> table gradient).

Workload (the differentiation workload on the full forward scene): a
65,536-leaf octree in the unit cube with log-normal(0, 1.5) leaf weights,
4,194,304 samples per view, a 16-level hash grid (2^19 entries per level, 4
features, resolutions 16..4096), head mode (64 channels), one 1280x832
pinhole view, upstream image gradient ~ N(0, 1).  Synthetic, seeded.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd ms/view & Gpoints/s (4M pts, 1280x832), % HBM roofline, vs plain FP32"
UNIT = "Gpoints/s"
N_LEAVES = 65536
N_SAMPLES = 4_194_304
LOG2_T = 19
W, H = 1280, 832
C = 64


def workload_config(extra=None):
    cfg = {"workload": "INPC view fwd+bwd: 65,536-leaf octree, 4,194,304 samples, 16-level 2^19x4 FP32 hash grid, "
                       "head mode (64 ch), 1280x832, dImage ~ N(0,1)",
           "n_leaves": N_LEAVES, "n_samples": N_SAMPLES, "image": [W, H], "channels": C, "log2_T": LOG2_T,
           "l2": "flushed (256 MiB write) before every timed step; per-step working set > 1 GB"}
    if extra:
        cfg.update(extra)
    return cfg


def make_scene():
    from paper_2403_16862_gb300 import scenes
    from paper_2403_16862_gb300 import api
    tree = scenes.make_octree(0, N_LEAVES)
    res = scenes.geometric_resolutions(16, 16, 4096)
    grid = scenes.make_hashgrid(1, api.hashgrid_n_entries(res, LOG2_T), res, LOG2_T)
    cam = scenes.make_camera((0.5, 0.5, -1.2), 900.0, 900.0, 640.0, 416.0, W, H)
    g = scenes.upstream_grad(2, (H, W, C))
    return tree, res, grid, cam, g


def algorithmic_bytes(n, n_leaves, n_entries, n_frag, n_pix):
    """Each array read or written once; fragments written once, read once."""
    e = 4  # FP32
    s_tab = 4 * e * n_entries
    s_grad = 16 * n_entries
    return {
        "sample": 40 * n_leaves + 16 * n,
        "query_fwd": 12 * n + s_tab + C * e * n,
        "raster_fwd": (12 + C * e) * n + 16 * n_frag + (C * e + 8) * n_pix,
        "raster_bwd": (C * e + 8) * n_pix + 8 * n_frag + (12 + C * e) * n + 4 * C * n,
        "query_bwd": 12 * n + 4 * C * n + 2 * s_grad,
    }


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), p[5], p[6], p[7], p[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ oracle ---
def oracle_view(tree, res, grid, cam, g, n_samples, seed=0, view=0):
    """One view through the FP64 oracle (the CPU baseline)."""
    from oracle import oracle as O
    _, pos64, _ = O.sample_octree(tree, seed, view, n_samples)
    pos = pos64.astype(np.float32)
    h = O.hash_fwd(res, LOG2_T, grid.table, pos)
    O.raster_fwd(cam, pos, h, head_mode=True)
    dh = O.raster_bwd(cam, pos, h, g, head_mode=True)["d_feat"]
    O.hash_bwd(res, LOG2_T, 4, pos, dh)


def cpu_baseline(tree, res, grid, cam, g, n_samples):
    from oracle import oracle as O
    O.build()
    t0 = time.perf_counter()
    oracle_view(tree, res, grid, cam, g, n_samples)
    dt = time.perf_counter() - t0
    return {"value": n_samples / dt / 1e9, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": "one full view (%d samples, 1280x832) through the FP64 oracle, %.1f s" % (n_samples, dt)}


def run_reference(args, rank):
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    tree, res, grid, cam, g = make_scene()
    n_ref = 1 << 20  # bounded sample: a quarter of the view's samples per step
    for i in range(args.warmup):
        oracle_view(tree, res, grid, cam, g, n_ref, view=100 + i)
    times = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        oracle_view(tree, res, grid, cam, g, n_ref, view=i)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n_ref * args.steps / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config({"reference_sample": "%d samples per step (same scene, view, image)" % n_ref}),
            "cpu_baseline": {"kind": "oracle", "cores": O.num_threads(), "value": value, "unit": UNIT,
                             "sample": "%d of the view's 4,194,304 samples per step, full 1280x832 image" % n_ref},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- GPU ---
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--unfused", action="store_true",
                    help="separate rasterizer backward and grid adjoint (materialises dh)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    import torch.distributed as dist
    from paper_2403_16862_gb300 import build
    build.build()
    from paper_2403_16862_gb300 import _binding as B
    from paper_2403_16862_gb300 import api

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")

    tree, res, grid, cam, g_np = make_scene()
    c = torch.from_numpy(tree.centers).to(dev)
    l = torch.from_numpy(tree.levels).to(dev)
    w = torch.from_numpy(tree.weights).to(dev)
    table = torch.from_numpy(grid.table).to(dev)
    g_img = torch.from_numpy(g_np).to(dev)
    desc = api.hashgrid_desc(res, LOG2_T)
    n_entries = grid.table.shape[0]
    opts = api.RasterOptions(n_channels=C, head_mode=True)
    N = N_SAMPLES

    # preallocated buffers: the timed loop allocates nothing
    ws_s = api.workspace(B.inpc_sample_workspace_size(N_LEAVES, N), dev)
    ws_r = api.workspace(api.rasterize_bwd_hashgrid_workspace_size(cam, opts, desc, N), dev)
    leaf = torch.empty(N, dtype=torch.int32, device=dev)
    pos = torch.empty(N, 3, dtype=torch.float32, device=dev)
    h = torch.empty(N, C, dtype=torch.float32, device=dev)
    img = torch.empty(H, W, C, dtype=torch.float32, device=dev)
    T = torch.empty(H, W, dtype=torch.float32, device=dev)
    ncon = torch.empty(H, W, dtype=torch.int32, device=dev)
    dh = torch.empty(N, C, dtype=torch.float32, device=dev) if args.unfused else None
    gtab = torch.zeros(n_entries, 4, dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def view(view_id, ev=None):
        def mark(i):
            if ev is not None:
                ev[i].record(stream)
        mark(0)
        api.sample_octree(c, l, w, tree.root_size, 0, view_id, N, ws=ws_s, out=(leaf, pos))
        mark(1)
        api.query_hashgrid(desc, table, pos, out=h)
        mark(2)
        api.rasterize_fwd(cam, opts, pos, h, None, ws=ws_r, out=(img, T, ncon))
        mark(3)
        gtab.zero_()
        if args.unfused:
            api.rasterize_bwd(cam, opts, pos, h, None, T, ncon, g_img, ws_r, out=(None, dh))
            mark(4)
            api.query_hashgrid_bwd(desc, pos, dh, gtab)
        else:
            mark(4)
            api.rasterize_bwd_hashgrid(cam, opts, desc, pos, h, T, ncon, g_img, ws_r, gtab)
        mark(5)

    stages = ["sample", "query_fwd", "raster_fwd", "table_zero", "raster_bwd+query_bwd"] if not args.unfused else \
        ["sample", "query_fwd", "raster_fwd", "raster_bwd", "query_bwd"]
    for i in range(args.warmup):
        view(1000 + i + rank * 97)
    torch.cuda.synchronize()

    sampler = ClockSampler(local_rank)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    launches0 = B.inpc_kernel_launches()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)  # evict the previous step from L2 (outside the events)
        view(rank * args.steps + k, evs[k])
    torch.cuda.synchronize()
    launches = B.inpc_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()

    per_stage = {s: [evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(args.steps)] for i, s in enumerate(stages)}
    step_ms = [evs[k][0].elapsed_time(evs[k][5]) for k in range(args.steps)]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = N * args.steps * world / (total_ms * 1e-3) / 1e9
    ms_per_step = total_ms / args.steps

    # every sample of this workload lies inside the view, so each splats to
    # exactly four on-image pixels: the fragment count is 4N
    bytes_model = algorithmic_bytes(N, N_LEAVES, n_entries, 4 * N, H * W)
    if not args.unfused:
        bytes_model["table_zero"] = 0
        bytes_model["raster_bwd+query_bwd"] = bytes_model.pop("raster_bwd") + bytes_model.pop("query_bwd")
    peak, peak_kind = measured_peak_hbm()
    stage_mean = {s: statistics.mean(v) for s, v in per_stage.items()}
    dom = max(stage_mean, key=stage_mean.get)
    achieved = bytes_model[dom] / (stage_mean[dom] * 1e-3) / 1e9
    total_bytes = sum(bytes_model.values())

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, api, B, tree, grid, cam, g_np, res, desc, opts, dev, world, rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(tree, res, grid, cam, g_np, N)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config({"views_per_step_per_gpu": 1, "parallelism": "views sharded over %d GPU(s)" % world}),
            "stages_ms": {s: round(stage_mean[s], 4) for s in stages},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "algorithmic_bytes": bytes_model[dom]},
            "step_roofline": {"algorithmic_bytes": total_bytes,
                              "achieved_gbs": total_bytes / (ms_per_step * 1e-3) / 1e9,
                              "frac": total_bytes / (ms_per_step * 1e-3) / 1e9 / peak},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_e2e(args, api, B, tree, grid, cam, g_np, res, desc, opts, dev, world, rank):
    """Same metric through the public API with host inputs: every step copies
    the octree, the table and the upstream gradient from pinned host memory
    and reads back the image and the table gradient."""
    import torch
    import torch.distributed as dist
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hc, hl, hw = pin(tree.centers), pin(tree.levels), pin(tree.weights)
    htab, hg = pin(grid.table), pin(g_np)
    out_img = torch.empty(H, W, C, dtype=torch.float32).pin_memory()
    out_gt = torch.empty(grid.table.shape, dtype=torch.float32).pin_memory()
    stream = torch.cuda.current_stream()
    N = N_SAMPLES

    def step(view_id):
        c = hc.to(dev, non_blocking=True)
        l = hl.to(dev, non_blocking=True)
        w = hw.to(dev, non_blocking=True)
        table = htab.to(dev, non_blocking=True)
        g = hg.to(dev, non_blocking=True)
        _, pos = api.sample_octree(c, l, w, tree.root_size, 0, view_id, N)
        hq = api.query_hashgrid(desc, table, pos)
        ws = api.workspace(api.rasterize_bwd_hashgrid_workspace_size(cam, opts, desc, N), dev)
        img, T, n, ws = api.rasterize_fwd(cam, opts, pos, hq, ws=ws)
        gt = torch.zeros_like(table)
        api.rasterize_bwd_hashgrid(cam, opts, desc, pos, hq, T, n, g, ws, gt)
        out_img.copy_(img, non_blocking=True)
        out_gt.copy_(gt, non_blocking=True)

    for i in range(3):
        step(2000 + i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        step(3000 + rank * args.steps + k)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    h2d = sum(x.numel() * x.element_size() for x in (hc, hl, hw, htab, hg))
    d2h = out_img.numel() * 4 + out_gt.numel() * 4
    return {"value": N * args.steps * world / (ms * 1e-3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": ms / args.steps}


if __name__ == "__main__":
    sys.exit(main())
