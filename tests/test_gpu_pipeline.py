"""The whole hot path on the GPU against the oracle's own pipeline: octree
sampling -> hash-grid query -> head-mode rasterizer forward and backward ->
table gradient.  The full-size case is the benchmark's workload
(65,536-leaf octree, 4,194,304 samples, 16-level 2^19 grid, 1280x832), in
the benchmark's launch configuration.  The oracle side never sees a GPU
value: it samples its own positions (exact FP64, rounded once to the FP32
interface type) and runs every stage itself."""
import numpy as np
import pytest
import torch

from paper_2403_16862_gb300 import api, scenes
from tests._parity import assert_cond_close, cond_ratio
from tests.test_gpu_raster import _excluded_points

pytestmark = pytest.mark.gpu

RES16 = scenes.geometric_resolutions(16, 16, 4096)


def _pipeline(gpu, oracle, n_leaves, n_samples, log2_T, cam, seed=0, graph_check=False, margins=False):
    tree = scenes.make_octree(seed, n_leaves)
    grid = scenes.make_hashgrid(seed + 1, oracle.hash_entries(RES16, log2_T), RES16, log2_T)
    g_img = scenes.upstream_grad(seed + 2, (cam.height, cam.width, 64))

    # ---- GPU
    c = torch.from_numpy(tree.centers).to(gpu)
    l = torch.from_numpy(tree.levels).to(gpu)
    w = torch.from_numpy(tree.weights).to(gpu)
    table = torch.from_numpy(grid.table).to(gpu)
    desc = api.hashgrid_desc(RES16, log2_T)
    opts = api.RasterOptions(n_channels=64, head_mode=True)
    leaf, pos = api.sample_octree(c, l, w, tree.root_size, seed, 0, n_samples)
    h = api.query_hashgrid(desc, table, pos)
    ws = api.workspace(api.rasterize_bwd_hashgrid_workspace_size(cam, opts, desc, n_samples), gpu)
    img, T, n, ws = api.rasterize_fwd(cam, opts, pos, h, ws=ws)
    _, dh = api.rasterize_bwd(cam, opts, pos, h, None, T, n, torch.from_numpy(g_img).to(gpu), ws)
    gt = torch.zeros_like(table)
    api.query_hashgrid_bwd(desc, pos, dh, gt)
    # the fused backward (rasterizer backward + query adjoint in one pass)
    gt_fused = torch.zeros_like(table)
    dh_fused = torch.empty_like(dh)
    api.rasterize_bwd_hashgrid(cam, opts, desc, pos, h, T, n, torch.from_numpy(g_img).to(gpu), ws, gt_fused,
                               d_feat=dh_fused)
    torch.cuda.synchronize()

    # ---- oracle
    o_leaf, o_pos64, _ = oracle.sample_octree(tree, seed, 0, n_samples)
    o_pos = o_pos64.astype(np.float32)
    o_h, o_hab = oracle.hash_fwd(RES16, log2_T, grid.table, o_pos, with_abs=True)
    # the rasterizer's tolerance scale carries the query's own sum |w t| per channel
    ref = oracle.raster_fwd(cam, o_pos, o_h, head_mode=True, with_abs=True, feat_abs=o_hab)
    rb = oracle.raster_bwd(cam, o_pos, o_h, g_img, head_mode=True, with_abs=True, feat_abs=o_hab)
    o_gt, o_gab = oracle.hash_bwd(RES16, log2_T, 4, o_pos, rb["d_feat"], with_abs=True, dh_abs=rb["abs_feat"])

    # ---- parity
    assert np.array_equal(leaf.cpu().numpy(), o_leaf)
    assert np.array_equal(pos.cpu().numpy(), o_pos)
    assert_cond_close(h.cpu().numpy(), o_h, o_hab, what="h")
    ok = ref["flags"] == 0
    assert (~ok).sum() <= max(2, 1e-4 * ok.size)
    assert np.array_equal(n.cpu().numpy()[ok], ref["n_contrib"][ok])
    assert_cond_close(img.cpu().numpy(), ref["image"], ref["abs"], mask=ok[..., None], what="image")
    assert_cond_close(T.cpu().numpy(), ref["T_final"], ref["T_final"], mask=ok, what="T_final")
    keep = ~_excluded_points(oracle, cam, o_pos, ref["flags"])
    assert_cond_close(dh.cpu().numpy(), rb["d_feat"], rb["abs_feat"], mask=keep[:, None], what="dh")
    # table rows reached by an excluded point (threshold-ambiguous pixel) are excluded too
    reach = oracle.hash_bwd(RES16, log2_T, 4, o_pos, np.repeat((~keep)[:, None], 64, 1).astype(np.float64))
    assert_cond_close(gt.cpu().numpy(), o_gt, o_gab, mask=reach == 0, what="grad_table")
    assert torch.equal(dh_fused, dh), "fused backward writes the same point gradients"
    assert_cond_close(gt_fused.cpu().numpy(), o_gt, o_gab, mask=reach == 0, what="grad_table (fused)")
    print("pipeline: %d samples, %d fragments, max blended per pixel %d, flagged pixels %d"
          % (n_samples, int(ref["n_frags"].sum()), int(ref["n_contrib"].max()), int((~ok).sum())))

    if margins:
        # how much of the bound the outputs use under the plain scale: the
        # rasterizer's sum T alpha |c| with the features' own magnitudes (not
        # the query's sum |w t|), and the table gradient's scale from that
        plain = oracle.raster_fwd(cam, o_pos, o_h, head_mode=True, with_abs=True)
        rbp = oracle.raster_bwd(cam, o_pos, o_h, g_img, head_mode=True, with_abs=True)
        _, o_gab_p = oracle.hash_bwd(RES16, log2_T, 4, o_pos, rb["d_feat"], with_abs=True, dh_abs=rbp["abs_feat"])
        used = {
            "image": (cond_ratio(img.cpu().numpy(), ref["image"], ref["abs"], mask=ok[..., None]),
                      cond_ratio(img.cpu().numpy(), ref["image"], plain["abs"], mask=ok[..., None])),
            "dh": (cond_ratio(dh.cpu().numpy(), rb["d_feat"], rb["abs_feat"], mask=keep[:, None]),
                   cond_ratio(dh.cpu().numpy(), rb["d_feat"], rbp["abs_feat"], mask=keep[:, None])),
            "grad_table": (cond_ratio(gt_fused.cpu().numpy(), o_gt, o_gab, mask=reach == 0),
                           cond_ratio(gt_fused.cpu().numpy(), o_gt, o_gab_p, mask=reach == 0)),
        }
        for k, (a, b) in used.items():
            print("bound used, %-10s scale of the test %.3f   plain scale %.3f" % (k, a, b))

    if graph_check:
        # the same sequence captured in a CUDA graph replays identically
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        outs = {}
        with torch.cuda.stream(s):
            gd = torch.from_numpy(g_img).to(gpu)
            torch.cuda.synchronize()
            with torch.cuda.graph(graph, stream=s):
                lf, ps = api.sample_octree(c, l, w, tree.root_size, seed, 0, n_samples)
                hh = api.query_hashgrid(desc, table, ps)
                im, TT, nn, ww = api.rasterize_fwd(cam, opts, ps, hh)
                outs["img"] = im
                outs["dh"] = api.rasterize_bwd(cam, opts, ps, hh, None, TT, nn, gd, ww)[1]
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(outs["img"], img)
        assert torch.allclose(outs["dh"], dh, rtol=0, atol=1e-5 * float(dh.abs().max()))


def test_pipeline_small(gpu, oracle):
    cam = scenes.make_camera((0.5, 0.5, -1.2), 900 * 0.25, 900 * 0.25, 160, 104, 320, 208)
    _pipeline(gpu, oracle, 4096 + 7 * 300, 200_000, 16, cam, seed=3, graph_check=True)


def test_pipeline_full_size(gpu, oracle):
    """65,536 leaves, 4,194,304 samples, 2^19 grid, 1280x832, fwd + bwd."""
    cam = scenes.make_camera((0.5, 0.5, -1.2), 900, 900, 640, 416, 1280, 832)
    _pipeline(gpu, oracle, 65536, 4_194_304, 19, cam, seed=0, margins=True)


def test_pipeline_large_table(gpu, oracle):
    """A 2^20 grid: the fine levels' gradient rows (8 x 16 MB) exceed the L2
    budget, so the fused backward stores them and the level-grouped pass
    (k_grad_fine) reduces them."""
    cam = scenes.make_camera((0.5, 0.5, -1.2), 900 * 0.25, 900 * 0.25, 160, 104, 320, 208)
    _pipeline(gpu, oracle, 4096 + 7 * 300, 200_000, 20, cam, seed=5)


@pytest.mark.parametrize("n_levels", [6, 8, 24, 32])
def test_fused_backward_level_counts(gpu, oracle, n_levels):
    """The fused rasterizer backward + grid adjoint for level counts other
    than 16 (its 8-, 16- and 32-lane layouts; levels past the count idle),
    on a 2^14 grid so that coarse levels are dense and the rest hashed."""
    res = scenes.geometric_resolutions(n_levels, 16, 1024)
    log2_T, F, n_samples = 14, 4 * n_levels, 60_000
    tree = scenes.make_octree(4, 4096 + 7 * 200)
    grid = scenes.make_hashgrid(5, oracle.hash_entries(res, log2_T), res, log2_T)
    cam = scenes.make_camera((0.5, 0.5, -1.2), 900 * 0.125, 900 * 0.125, 80, 52, 160, 104)
    g_img = scenes.upstream_grad(6, (cam.height, cam.width, F))
    c, l, w = (torch.from_numpy(x).to(gpu) for x in (tree.centers, tree.levels, tree.weights))
    table = torch.from_numpy(grid.table).to(gpu)
    desc = api.hashgrid_desc(res, log2_T)
    opts = api.RasterOptions(n_channels=F, head_mode=True)
    _, pos = api.sample_octree(c, l, w, tree.root_size, 4, 0, n_samples)
    h = api.query_hashgrid(desc, table, pos)
    ws = api.workspace(api.rasterize_bwd_hashgrid_workspace_size(cam, opts, desc, n_samples), gpu)
    img, T, n, ws = api.rasterize_fwd(cam, opts, pos, h, ws=ws)
    gt = torch.zeros_like(table)
    dh = torch.empty(n_samples, F, dtype=torch.float32, device=gpu)
    api.rasterize_bwd_hashgrid(cam, opts, desc, pos, h, T, n, torch.from_numpy(g_img).to(gpu), ws, gt, d_feat=dh)
    torch.cuda.synchronize()

    _, o_pos64, _ = oracle.sample_octree(tree, 4, 0, n_samples)
    o_pos = o_pos64.astype(np.float32)
    o_h, o_hab = oracle.hash_fwd(res, log2_T, grid.table, o_pos, with_abs=True)
    ref = oracle.raster_fwd(cam, o_pos, o_h, head_mode=True, with_abs=True, feat_abs=o_hab)
    rb = oracle.raster_bwd(cam, o_pos, o_h, g_img, head_mode=True, with_abs=True, feat_abs=o_hab)
    o_gt, o_gab = oracle.hash_bwd(res, log2_T, 4, o_pos, rb["d_feat"], with_abs=True, dh_abs=rb["abs_feat"])
    ok = ref["flags"] == 0
    assert (~ok).sum() <= max(2, 1e-4 * ok.size)
    assert_cond_close(img.cpu().numpy(), ref["image"], ref["abs"], mask=ok[..., None], what="image")
    keep = ~_excluded_points(oracle, cam, o_pos, ref["flags"])
    assert_cond_close(dh.cpu().numpy(), rb["d_feat"], rb["abs_feat"], mask=keep[:, None], what="dh")
    reach = oracle.hash_bwd(res, log2_T, 4, o_pos, np.repeat((~keep)[:, None], F, 1).astype(np.float64))
    assert_cond_close(gt.cpu().numpy(), o_gt, o_gab, mask=reach == 0, what="grad_table (fused)")
    assert np.abs(o_gt).max() > 0
