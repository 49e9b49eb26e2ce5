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
SCALE = 1  # --scale k: the profiling case (N / k^2 samples, image and focal length / k)


def workload_config(extra=None):
    cfg = {"workload": "INPC view fwd+bwd: 65,536-leaf octree, %s samples, 16-level 2^19x4 FP32 hash grid, "
                       "head mode (64 ch), %dx%d, dImage ~ N(0,1)%s"
                       % (format(N_SAMPLES, ","), W, H, "" if SCALE == 1 else " (profiling case, scale 1/%d)" % SCALE),
           "n_leaves": N_LEAVES, "n_samples": N_SAMPLES, "image": [W, H], "channels": C, "log2_T": LOG2_T,
           "l2": "flushed (256 MiB write) before every timed step; per-step working set > 1 GB"}
    if extra:
        cfg.update(extra)
    return cfg


def make_scene(n_entries_fn=None):
    """The seeded scene.  ``n_entries_fn(res, log2_T)`` sizes the table: the
    library's layout query on the GPU arm, the oracle's on the reference arm
    (which loads nothing but the oracle)."""
    from paper_2403_16862_gb300 import scenes
    if n_entries_fn is None:
        from paper_2403_16862_gb300 import api
        n_entries_fn = api.hashgrid_n_entries
    tree = scenes.make_octree(0, N_LEAVES)
    res = scenes.geometric_resolutions(16, 16, 4096)
    grid = scenes.make_hashgrid(1, n_entries_fn(res, LOG2_T), res, LOG2_T)
    f = 900.0 / SCALE
    cam = scenes.make_camera((0.5, 0.5, -1.2), f, f, W / 2.0, H / 2.0, W, H)
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


KERNELS = ["k_draw_count", "k_place", "k_hash_fwd", "k_pix_count", "k_pix_scatter", "k_blend_fwd",
           "k_blend_fwd_large", "k_blend_fwd_heavy", "k_blend_bwd", "k_blend_bwd_large", "k_blend_bwd_heavy",
           "k_point_grad_hash", "k_grad_fine", "k_point_grad", "k_hash_bwd"]

# Counters of one launch of the dominant kernel on the full workload, from one
# ncu capture each (profiles/ holds the command and the summary):
#   traffic        dram__bytes_read.sum + dram__bytes_write.sum
#   l2_reductions  lts__t_requests_op_red.sum
# with the stamp of the kernel's sources at the time of the capture.  A
# different stamp means the kernel changed since: the counters are then
# reported as null rather than as figures of another kernel.
CAPTURED = {"k_point_grad_hash": {"traffic": 696_609_792 + 218_087_680, "l2_reductions": 243_198_353,
                                  "stamp": "5cfcc33073ce2e3f"}}
# the sources each kernel's code comes from (stamped for CAPTURED); "step":
# every kernel of one view
KERNEL_SOURCES = {"k_point_grad_hash": ["raster_bwd.cu", "raster_impl.cuh", "hashgrid_impl.cuh", "common.cuh"],
                  "k_hash_fwd": ["hashgrid.cu", "hashgrid_impl.cuh", "common.cuh"],
                  "step": ["sample.cu", "sample_impl.cuh", "scan.cuh", "hashgrid.cu", "hashgrid_impl.cuh",
                           "raster_impl.cuh", "raster_fwd.cu", "raster_bwd.cu", "common.cuh"]}
# DRAM bytes (read + write) of every kernel of one view on the full workload,
# the library's kernels and the table-gradient clear, summed from one ncu
# capture of all launches (mean of its 5 views); profiles/ holds the command
STEP_CAPTURED = {"dram_bytes": 7_219_000_000, "stamp": "fbcef1a1402290b5"}


def source_stamp(kernel):
    import hashlib
    files = KERNEL_SOURCES.get(kernel)
    if not files:
        return None
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2403_16862_gb300", "csrc", f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def captured(kernel, key):
    """A counter of CAPTURED, or None when the kernel's sources changed since
    the capture (or the run is not the full workload)."""
    c = CAPTURED.get(kernel)
    if not c or SCALE != 1 or c.get("stamp") != source_stamp(kernel):
        return None
    return c.get(key)


def kernel_bytes(kernel, n, n_entries, n_frag, n_pix):
    """Algorithmic bytes of one launch (FP32, head mode, C channels).

    k_point_grad_hash (fused rasterizer backward tail + grid adjoint): per
    point its position (12 B) and channel 0 of its feature row (4 B); per
    fragment slot the blend backward's two scalars (8 B, stored point-major);
    the upstream image gradient once (4 C per pixel); the table gradient
    read and written once (2 x 16 B per row).
    k_hash_fwd: positions, the table once, the feature rows written once."""
    if kernel == "k_point_grad_hash":
        return 16 * n + 8 * n_frag + 4 * C * n_pix + 32 * n_entries
    if kernel == "k_hash_fwd":
        return 12 * n + 16 * n_entries + 4 * C * n
    return None


def atomic_ceiling(kernel, n, ms):
    """The grid adjoint forms 8 corner contributions (16 B) per point and
    level.  Coarse levels merge runs of them before they reach L2, so the L2
    vector reductions (lts__t_requests_op_red.sum, one ncu capture) are
    fewer; their rate, not DRAM, is what the reductions cost."""
    if kernel != "k_point_grad_hash":
        return {}
    out = {"corner_contributions": 8 * 16 * n}
    red = captured(kernel, "l2_reductions")
    out.update({"l2_reductions": red, "l2_reduction_gops": red / (ms * 1e-3) / 1e9 if red else None})
    return out


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


def cpu_baseline(tree, res, grid, cam, g, n_samples, min_seconds=10.0, max_views=5):
    """Full views through the FP64 oracle until about min_seconds of CPU work."""
    from oracle import oracle as O
    O.build()
    t0 = time.perf_counter()
    views = 0
    while views < max_views and (views == 0 or time.perf_counter() - t0 < min_seconds):
        oracle_view(tree, res, grid, cam, g, n_samples, view=views)
        views += 1
    dt = time.perf_counter() - t0
    return {"value": views * n_samples / dt / 1e9, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": "%d full view(s) (%d samples, %dx%d each) through the FP64 oracle, %.1f s"
                      % (views, n_samples, W, H, dt)}


def run_reference(args, rank):
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    tree, res, grid, cam, g = make_scene(O.hash_entries)
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
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the BF16 (16M points, 1920x1080) and batched BF16 (8 views) forms")
    ap.add_argument("--scale", type=int, default=1,
                    help="profiling case: N / k^2 samples, image and focal length / k (same fragments per pixel)")
    ap.add_argument("--unfused", action="store_true",
                    help="separate rasterizer backward and grid adjoint (materialises dh)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.scale != 1:
        global SCALE, N_SAMPLES, W, H
        k = args.scale
        if k < 1 or W % k or H % k:
            ap.error("--scale must divide 1280 and 832")
        SCALE, N_SAMPLES, W, H = k, N_SAMPLES // (k * k), W // k, H // k
        args.no_forms = True

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
    from paper_2403_16862_gb300 import api, shard

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        # NVLS off: the exchange is a plain ring/tree all-reduce
        os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
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
    # N > 1: the table gradient's sum over ranks (the one exchange of the
    # step) runs asynchronously after each backward, overlapped with the next
    # view's forward, on two alternating gradient tables
    gx = shard.GradExchange((n_entries, 4), dev) if world > 1 else None
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
        if gx is not None:
            gt = gx.begin()  # waits for the sum of two steps ago on this table
        else:
            gt = gtab
            gt.zero_()
        if args.unfused:
            api.rasterize_bwd(cam, opts, pos, h, None, T, ncon, g_img, ws_r, out=(None, dh))
            mark(4)
            api.query_hashgrid_bwd(desc, pos, dh, gt)
        else:
            mark(4)
            api.rasterize_bwd_hashgrid(cam, opts, desc, pos, h, T, ncon, g_img, ws_r, gt)
        if gx is not None:
            gx.launch()
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
        view(shard.view_ids(rank, world, k)[0], evs[k])
    tail = None
    if gx is not None:
        # the last step's exchange belongs to the timed work
        gx.finish()
        tail = torch.cuda.Event(enable_timing=True)
        tail.record(stream)
    torch.cuda.synchronize()
    launches = B.inpc_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()

    # per-kernel device times in a separate pass over the same views (the
    # library's launch timer records two events around each launch, which
    # stays out of the headline region)
    k_steps = min(args.steps, 10)
    B.inpc_kernel_timer_read()  # drop records of earlier launches
    B.inpc_kernel_timer_enable(True)
    for k in range(k_steps):
        flush.fill_(k & 0xFF)
        view(shard.view_ids(rank, world, k)[0])
    if gx is not None:
        gx.finish()
    torch.cuda.synchronize()
    B.inpc_kernel_timer_enable(False)
    kernel_ms = {}
    for kname in KERNELS:
        ms, cnt = B.inpc_kernel_timer_read(kname)
        if cnt:
            kernel_ms[kname] = (ms / k_steps, cnt // k_steps)

    per_stage = {s: [evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(args.steps)] for i, s in enumerate(stages)}
    step_ms = [evs[k][0].elapsed_time(evs[k][5]) for k in range(args.steps)]
    total_ms = sum(step_ms) + (evs[-1][5].elapsed_time(tail) if tail is not None else 0.0)
    total_ms = shard.max_over_ranks(total_ms, dev)
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
    total_bytes = sum(bytes_model.values())
    # the dominant kernel: most device time per step (one launch per step)
    if not kernel_ms:
        raise RuntimeError("the library's kernel timer recorded no launch")
    dom = max(kernel_ms, key=lambda k: kernel_ms[k][0])
    dom_ms = kernel_ms[dom][0] / max(kernel_ms[dom][1], 1)
    dom_bytes = kernel_bytes(dom, N, n_entries, 4 * N, H * W)
    step_dram = STEP_CAPTURED["dram_bytes"] if (SCALE == 1 and not args.unfused
                                                and STEP_CAPTURED["stamp"] == source_stamp("step")) else None
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9 if dom_bytes else None

    # the L2 reduction ceiling the grid adjoint's table additions run into,
    # measured on this GPU after the timed region (8 MB region, the size of
    # one hashed level's gradient rows)
    l2_ceiling = None
    if dom == "k_point_grad_hash" and not args.unfused:
        cal = torch.zeros(1 << 19, 4, dtype=torch.float32, device=dev)
        cs = torch.cuda.current_stream().cuda_stream
        single = B.inpc_l2_reduction_rate(cal.data_ptr(), 1 << 19, False, cs)
        paired = B.inpc_l2_reduction_rate(cal.data_ptr(), 1 << 19, True, cs)
        del cal
        red = captured(dom, "l2_reductions")
        rate = red / (dom_ms * 1e-3) / 1e9 if red else None
        l2_ceiling = {
            "probe": "inpc_l2_reduction_rate: 16-byte red.global.add.v4.f32 into random rows of an 8 MB region, "
                     "8 CTAs x 256 threads per SM, evict_last",
            "single_row_requests_gops": single, "paired_rows_gops": paired, "paired_requests_gops": paired / 2,
            "kernel_requests_gops": rate,
            "frac_of_single_row_requests": rate / single if rate else None}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, api, B, tree, grid, cam, g_np, res, desc, opts, dev, world, rank)

    forms = None
    if not args.no_forms and not args.unfused:
        forms = run_forms(args, api, B, dev, world, rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(tree, res, grid, cam, g_np, N)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config({"views_per_step_per_gpu": 1, "parallelism": "views sharded over %d GPU(s)" % world
                                       + ("; FP32 table-gradient all-reduce per step, overlapped with the next view's "
                                          "forward" if world > 1 else "")}),
            "stages_ms": {s: round(stage_mean[s], 4) for s in stages},
            "kernels_ms": {k: round(v[0], 4) for k, v in sorted(kernel_ms.items(), key=lambda kv: -kv[1][0])},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if achieved else None,
                         "traffic": captured(dom, "traffic") if not args.unfused else None,
                         "counters_stamp": source_stamp(dom),
                         "peak_kind": peak_kind + " (copy bandwidth)", "launch_ms": dom_ms,
                         "algorithmic_bytes": dom_bytes, **atomic_ceiling(dom, N, dom_ms),
                         "l2_reduction_ceiling": l2_ceiling},
            "step_roofline": {"algorithmic_bytes": total_bytes,
                              "achieved_gbs": total_bytes / (ms_per_step * 1e-3) / 1e9,
                              "frac": total_bytes / (ms_per_step * 1e-3) / 1e9 / peak,
                              "measured_dram_bytes": step_dram,
                              "measured_dram_gbs": step_dram / (ms_per_step * 1e-3) / 1e9 if step_dram else None,
                              "measured_from": "ncu dram__bytes_read.sum + dram__bytes_write.sum of every kernel of "
                                               "one view, full workload, sources stamp %s" % source_stamp("step")},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "e2e": e2e,
            "forms": forms,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_forms(args, api, B, dev, world, rank):
    """The precision and batching forms on the same GPU.

    BF16 form: a 1,048,576-leaf octree, 16,777,216 samples, a 16-level 2^21
    BF16 grid, BF16 feature rows and image (FP32 blending, transmittance and
    gradients), 1920x1080, forward + fused backward; against the same view in
    FP32.  Batched BF16 form: 8 views of uneven size (640x480 .. 1920x1080,
    9.33 Mpixels in all) on an orbit around the scene, 8,388,608 samples per
    view from the shared octree and BF16 grid, all views in one CUDA graph
    over 4 streams with autotuned tiles; against the plain FP32 form (the
    same views one after another on one stream).  Accuracy is stated as the
    norm-wise difference to the FP32 form (the FP32 form itself matches the
    FP64 oracle to 1e-5 in the tests).  Upstream image gradients ~ N(0, 1)
    are drawn on the device from a seeded generator."""
    import torch
    from paper_2403_16862_gb300 import scenes
    from paper_2403_16862_gb300.batch import ViewBatch

    steps = max(2, min(args.steps, 5))
    res = scenes.geometric_resolutions(16, 16, 4096)
    tree = scenes.make_octree(0, 1 << 20, start_level=6)
    log2_T = 21
    n_ent = api.hashgrid_n_entries(res, log2_T)
    grid = scenes.make_hashgrid(1, n_ent, res, log2_T)
    c, l, w = (torch.from_numpy(x).to(dev) for x in (tree.centers, tree.levels, tree.weights))
    t32 = torch.from_numpy(grid.table).to(dev)
    t16 = t32.to(torch.bfloat16)
    d32 = api.hashgrid_desc(res, log2_T)
    d16 = api.hashgrid_desc(res, log2_T, table_dtype=torch.bfloat16, out_dtype=torch.bfloat16)
    gen = torch.Generator(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def dgrad(cam, seed):
        gen.manual_seed(seed)
        return torch.randn(cam.height, cam.width, C, generator=gen, device=dev)

    def nerr(a, b):
        a, b = a.double(), b.double()
        return float(torch.linalg.norm(a - b) / torch.linalg.norm(a))

    def timed(fn, n_steps):
        for i in range(3):
            fn(i)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2 * n_steps)]
        for k in range(n_steps):
            flush.fill_(k & 0xFF)
            e[2 * k].record()
            fn(k)
            e[2 * k + 1].record()
        torch.cuda.synchronize()
        return statistics.median(e[2 * k].elapsed_time(e[2 * k + 1]) for k in range(n_steps))

    class Plain:
        """One view at a time on the current stream, preallocated buffers."""
        def __init__(self, cams, n, bf16):
            self.n, self.bf16 = n, bf16
            self.desc, self.table = (d16, t16) if bf16 else (d32, t32)
            hdt = torch.bfloat16 if bf16 else torch.float32
            self.opts = api.RasterOptions(n_channels=C, head_mode=True, bf16=bf16)
            big = max(cams, key=lambda q: q.width * q.height)
            self.ws_s = api.workspace(B.inpc_sample_workspace_size(tree.n_leaves, n), dev)
            self.ws_r = api.workspace(api.rasterize_bwd_hashgrid_workspace_size(big, self.opts, self.desc, n), dev)
            self.leaf = torch.empty(n, dtype=torch.int32, device=dev)
            self.pos = torch.empty(n, 3, dtype=torch.float32, device=dev)
            self.h = torch.empty(n, C, dtype=hdt, device=dev)
            self.imgs = [torch.empty(q.height, q.width, C, dtype=hdt, device=dev) for q in cams]
            self.Ts = [torch.empty(q.height, q.width, dtype=torch.float32, device=dev) for q in cams]
            self.ncs = [torch.empty(q.height, q.width, dtype=torch.int32, device=dev) for q in cams]
            self.gt = torch.zeros(n_ent, 4, dtype=torch.float32, device=dev)
            self.cams = cams

        def run(self, grads, view0=0):
            self.gt.zero_()
            for v, cam in enumerate(self.cams):
                api.sample_octree(c, l, w, tree.root_size, 0, view0 + v, self.n, ws=self.ws_s,
                                  out=(self.leaf, self.pos))
                api.query_hashgrid(self.desc, self.table, self.pos, out=self.h)
                api.rasterize_fwd(cam, self.opts, self.pos, self.h, None, ws=self.ws_r,
                                  out=(self.imgs[v], self.Ts[v], self.ncs[v]))
                api.rasterize_bwd_hashgrid(cam, self.opts, self.desc, self.pos, self.h, self.Ts[v], self.ncs[v],
                                           grads[v], self.ws_r, self.gt)

    out = {}
    # ---- BF16 form, one 1920x1080 view of 16M samples
    n4 = 1 << 24
    cam4 = scenes.make_camera((0.5, 0.5, -1.2), 900.0 * 1080 / 832, 900.0 * 1080 / 832, 960.0, 540.0, 1920, 1080)
    g4 = [dgrad(cam4, 11)]
    p32 = Plain([cam4], n4, False)
    ms32 = timed(lambda k: p32.run(g4, view0=0), steps)
    img32, gt32 = p32.imgs[0].clone(), p32.gt.clone()
    del p32
    torch.cuda.empty_cache()
    p16 = Plain([cam4], n4, True)
    ms16 = timed(lambda k: p16.run(g4, view0=0), steps)
    out["bf16_view"] = {
        "workload": "1,048,576-leaf octree, 16,777,216 samples, 16-level 2^21x4 BF16 grid, BF16 h and image, "
                    "1920x1080, fwd + fused bwd",
        "ms_per_view": ms16, "gpoints_s": n4 / (ms16 * 1e-3) / 1e9,
        "fp32_ms_per_view": ms32, "speedup_vs_fp32": ms32 / ms16,
        "error_vs_fp32_normwise": {"image": nerr(img32, p16.imgs[0]), "grad_table": nerr(gt32, p16.gt)}}
    del p16, img32, gt32, g4
    torch.cuda.empty_cache()

    # ---- batched BF16 form, 8 uneven views of 8M samples each
    sizes = [(640, 480), (960, 540), (1024, 768), (1280, 832), (1280, 832), (1600, 900), (1920, 1080), (1920, 1080)]
    cams = scenes.orbit_cameras(sizes)
    n5 = 1 << 23
    grads = [dgrad(q, 100 + v) for v, q in enumerate(cams)]
    p32 = Plain(cams, n5, False)
    ms_plain = timed(lambda k: p32.run(grads), steps)
    imgs32 = [x.clone() for x in p32.imgs]
    gt32 = p32.gt.clone()
    del p32
    torch.cuda.empty_cache()
    vb = ViewBatch(c, l, w, tree.root_size, d16, t16, cams, n5, grads, seed=0, n_streams=4, bf16=True, tune=True)
    vb.capture()
    ms_batch = timed(lambda k: vb.step(), steps)
    errs = [nerr(imgs32[v], vb.views[v]["img"]) for v in range(len(cams))]
    tiles = [(d["opts"].tile_w, d["opts"].tile_h) for d in vb.views]
    del vb
    torch.cuda.empty_cache()
    # the same batch with the sampling and query of all views in one
    # persistent work-queue launch (same autotuned tiles)
    vp = ViewBatch(c, l, w, tree.root_size, d16, t16, cams, n5, grads, seed=0, n_streams=4, bf16=True, tune=False,
                   persistent=True)
    for d, (tw, th) in zip(vp.views, tiles):
        d["opts"].tile_w, d["opts"].tile_h = tw, th
    vp.capture()
    ms_pers = timed(lambda k: vp.step(), steps)
    errs_p = [nerr(imgs32[v], vp.views[v]["img"]) for v in range(len(cams))]
    vb = vp
    out["bf16_batched_8views"] = {
        "workload": "8 views %s, 8,388,608 samples each from one 1,048,576-leaf octree, 16-level 2^21x4 BF16 grid, "
                    "one CUDA graph over 4 streams, autotuned tiles, fwd + fused bwd" % sizes,
        "ms_per_step": ms_batch, "ms_per_view": ms_batch / len(cams),
        "gpoints_s": n5 * len(cams) / (ms_batch * 1e-3) / 1e9,
        "fp32_unbatched_ms_per_step": ms_plain, "speedup_vs_plain_fp32": ms_plain / ms_batch,
        "tiles": [list(t) for t in tiles],
        "persistent_front": {"ms_per_step": ms_pers, "speedup_vs_plain_fp32": ms_plain / ms_pers,
                             "speedup_vs_stream_fork": ms_batch / ms_pers,
                             "image_max_err_over_views": max(errs_p)},
        "error_vs_fp32_normwise": {"image_max_over_views": max(errs), "grad_table": nerr(gt32, vb.grad_table)}}
    del vb
    torch.cuda.empty_cache()

    # ---- batching where it pays: 32 small views (320x240, 1M samples each)
    small = [(320, 240)] * 32
    cams_s = scenes.orbit_cameras(small, focal_ref=300.0, ref_height=240)
    n_s = 1 << 20
    grads_s = [dgrad(q, 300 + v) for v, q in enumerate(cams_s)]
    p32 = Plain(cams_s, n_s, False)
    ms_plain_s = timed(lambda k: p32.run(grads_s), steps)
    del p32
    torch.cuda.empty_cache()
    vb = ViewBatch(c, l, w, tree.root_size, d32, t32, cams_s, n_s, grads_s, seed=0, n_streams=8, bf16=False, tune=True)
    vb.capture()
    ms_batch_s = timed(lambda k: vb.step(), steps)
    tiles_s = [(d["opts"].tile_w, d["opts"].tile_h) for d in vb.views]
    del vb
    torch.cuda.empty_cache()
    vb = ViewBatch(c, l, w, tree.root_size, d32, t32, cams_s, n_s, grads_s, seed=0, n_streams=8, bf16=False, tune=False,
                   persistent=True)
    for d, (tw, th) in zip(vb.views, tiles_s):
        d["opts"].tile_w, d["opts"].tile_h = tw, th
    vb.capture()
    ms_pers_s = timed(lambda k: vb.step(), steps)
    out["fp32_batched_32_small_views"] = {
        "workload": "32 views 320x240 on an orbit, 1,048,576 samples each from the 1,048,576-leaf octree, "
                    "16-level 2^21x4 FP32 grid, one CUDA graph over 8 streams, autotuned tiles, fwd + fused bwd",
        "ms_per_step": ms_batch_s, "ms_per_view": ms_batch_s / len(cams_s),
        "unbatched_ms_per_step": ms_plain_s, "speedup_vs_unbatched": ms_plain_s / ms_batch_s,
        "persistent_front_ms_per_step": ms_pers_s, "persistent_speedup_vs_unbatched": ms_plain_s / ms_pers_s,
        "persistent_speedup_vs_stream_fork": ms_batch_s / ms_pers_s}
    del vb
    torch.cuda.empty_cache()

    # ---- launch-dominated batch: 64 small views of 262,144 samples each,
    # stream-fork graph against the persistent front end
    tree64 = scenes.make_octree(0, 65536)
    c64, l64, w64 = (torch.from_numpy(x).to(dev) for x in (tree64.centers, tree64.levels, tree64.weights))
    n_ent19 = api.hashgrid_n_entries(res, 19)
    t19 = torch.from_numpy(scenes.make_hashgrid(1, n_ent19, res, 19).table).to(dev)
    d19 = api.hashgrid_desc(res, 19)
    cams_t = scenes.orbit_cameras([(320, 240)] * 64, focal_ref=300.0, ref_height=240)
    grads_t = [dgrad(q, 500 + v) for v, q in enumerate(cams_t)]
    n_t = 1 << 18
    res_t = {}
    for pers in (False, True):
        vb = ViewBatch(c64, l64, w64, tree64.root_size, d19, t19, cams_t, n_t, grads_t, seed=0, n_streams=8,
                       bf16=False, tune=False, persistent=pers)
        vb.capture()
        res_t[pers] = timed(lambda k: vb.step(), steps)
        del vb
        torch.cuda.empty_cache()
    out["fp32_batched_64_tiny_views"] = {
        "workload": "64 views 320x240 on an orbit, 262,144 samples each from the 65,536-leaf octree, 16-level "
                    "2^19x4 FP32 grid, one CUDA graph, fwd + fused bwd",
        "stream_fork_ms_per_step": res_t[False], "persistent_front_ms_per_step": res_t[True],
        "speedup_persistent_vs_fork": res_t[False] / res_t[True],
        "gpoints_s_persistent": 64 * n_t / (res_t[True] * 1e-3) / 1e9}
    del grads_t, t19
    torch.cuda.empty_cache()

    # ---- inference: a pre-extracted cloud rendered from several views
    n_pre = 1 << 26
    lw = api.level_weights(l, w.clone(), 0.5)
    _, pos_pre = api.sample_octree_halton(c, l, lw, tree.root_size, 5, n_pre)
    h_pre = api.query_hashgrid(d16, t16, pos_pre)
    opts_pre = api.RasterOptions(n_channels=C, head_mode=True, bf16=True)
    cams_r = scenes.orbit_cameras([(1280, 832)] * 4)
    ws_pre = api.workspace(api.rasterize_workspace_size(cams_r[0], opts_pre, n_pre), dev)
    bufs = api.rasterize_fwd(cams_r[0], opts_pre, pos_pre, h_pre, ws=ws_pre)[:3]
    ms_render = timed(lambda k: api.rasterize_fwd(cams_r[k % 4], opts_pre, pos_pre, h_pre, ws=ws_pre, out=bufs), steps)
    out["bf16_preextracted_render"] = {
        "workload": "67,108,864 points pre-extracted once (level weights, Halton positions) from the 1,048,576-leaf "
                    "octree, BF16 features queried once, rendered (rasterizer forward only) at 1280x832 per view",
        "ms_per_view": ms_render, "views_per_s": 1e3 / ms_render}
    del h_pre, pos_pre, ws_pre, bufs
    torch.cuda.empty_cache()
    return out


def run_e2e(args, api, B, tree, grid, cam, g_np, res, desc, opts, dev, world, rank):
    """Same metric through the public API with host inputs: every step copies
    the octree, the table and the upstream gradient from pinned host memory
    and reads back the image and the table gradient.  The copies run on a
    second stream with double-buffered device buffers, as a training loop
    would pipeline them: step k+1's inputs move while step k computes, and
    step k's image leaves while its backward runs."""
    import torch
    from paper_2403_16862_gb300 import shard
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hc, hl, hw = pin(tree.centers), pin(tree.levels), pin(tree.weights)
    htab, hg = pin(grid.table), pin(g_np)
    N = N_SAMPLES
    comp = torch.cuda.current_stream()
    copy_in = torch.cuda.Stream(device=dev)  # host -> device
    copy = torch.cuda.Stream(device=dev)     # device -> host
    ev = lambda: torch.cuda.Event()
    sets = []
    for _ in range(2):
        sets.append(dict(
            c=torch.empty_like(hc, device=dev), l=torch.empty_like(hl, device=dev), w=torch.empty_like(hw, device=dev),
            table=torch.empty_like(htab, device=dev), g=torch.empty_like(hg, device=dev),
            img=torch.empty(H, W, C, dtype=torch.float32, device=dev),
            T=torch.empty(H, W, dtype=torch.float32, device=dev), nc=torch.empty(H, W, dtype=torch.int32, device=dev),
            gt=torch.empty(grid.table.shape, dtype=torch.float32, device=dev),
            out_img=torch.empty(H, W, C, dtype=torch.float32).pin_memory(),
            out_gt=torch.empty(grid.table.shape, dtype=torch.float32).pin_memory(),
            ev_tree=ev(), ev_g=ev(), ev_img=ev(), ev_bwd=ev(), ev_out=ev()))
    ws_s = api.workspace(B.inpc_sample_workspace_size(tree.n_leaves, N), dev)
    ws_r = api.workspace(api.rasterize_bwd_hashgrid_workspace_size(cam, opts, desc, N), dev)
    leaf = torch.empty(N, dtype=torch.int32, device=dev)
    pos = torch.empty(N, 3, dtype=torch.float32, device=dev)
    hq = torch.empty(N, C, dtype=torch.float32, device=dev)

    def step(k, view_id):
        S = sets[k % 2]
        with torch.cuda.stream(copy_in):
            copy_in.wait_event(S["ev_bwd"])  # step k-2 no longer reads this set's inputs
            for name, host in (("c", hc), ("l", hl), ("w", hw), ("table", htab)):
                S[name].copy_(host, non_blocking=True)
            S["ev_tree"].record(copy_in)
            S["g"].copy_(hg, non_blocking=True)
            S["ev_g"].record(copy_in)
        comp.wait_event(S["ev_tree"])
        comp.wait_event(S["ev_out"])  # step k-2's outputs have left this set's buffers
        api.sample_octree(S["c"], S["l"], S["w"], tree.root_size, 0, view_id, N, ws=ws_s, out=(leaf, pos))
        api.query_hashgrid(desc, S["table"], pos, out=hq)
        api.rasterize_fwd(cam, opts, pos, hq, None, ws=ws_r, out=(S["img"], S["T"], S["nc"]))
        S["ev_img"].record(comp)
        comp.wait_event(S["ev_g"])
        S["gt"].zero_()
        api.rasterize_bwd_hashgrid(cam, opts, desc, pos, hq, S["T"], S["nc"], S["g"], ws_r, S["gt"])
        S["ev_bwd"].record(comp)
        with torch.cuda.stream(copy):
            copy.wait_event(S["ev_img"])
            S["out_img"].copy_(S["img"], non_blocking=True)
            copy.wait_event(S["ev_bwd"])
            S["out_gt"].copy_(S["gt"], non_blocking=True)
            S["ev_out"].record(copy)

    for i in range(3):
        step(i, 2000 + i)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(comp)
    copy_in.wait_event(e0)
    copy.wait_event(e0)
    t_host = time.perf_counter()
    for k in range(args.steps):
        step(k, 3000 + shard.view_ids(rank, world, k)[0])
    comp.wait_stream(copy_in)
    comp.wait_stream(copy)
    e1.record(comp)
    t_host = time.perf_counter() - t_host  # issuing the steps, before waiting for them
    torch.cuda.synchronize()
    ms = shard.max_over_ranks(e0.elapsed_time(e1), dev)
    h2d = sum(x.numel() * x.element_size() for x in (hc, hl, hw, htab, hg))
    d2h = sets[0]["out_img"].numel() * 4 + sets[0]["out_gt"].numel() * 4
    return {"value": N * args.steps * world / (ms * 1e-3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": ms / args.steps,
            "host_ms_per_step": t_host * 1e3 / args.steps,
            "copies": "pinned host memory, one stream per direction, double-buffered device buffers"}


if __name__ == "__main__":
    sys.exit(main())
