"""BF16 form of the path: BF16 hash table, BF16 query output (the feature
rows the rasterizer reads) and BF16 image, with FP32 arithmetic, FP32
transmittance and FP32 gradients.  Its error against the FP64 oracle (run on
the FP32 table) is stated per output; the only assertions are bounds that
BF16 storage (8 significant bits, relative rounding <= 2^-9 per value)
implies."""
import numpy as np
import pytest
import torch

from paper_2403_16862_gb300 import api, scenes

pytestmark = pytest.mark.gpu

RES16 = scenes.geometric_resolutions(16, 16, 4096)


def _err(gpu, ref, scale):
    """(norm-wise relative error, max |error| / max sum|terms|).  BF16 moves
    some pixels' stopping point, so elementwise ratios against exact zeros of
    the oracle are not meaningful; both measures here are."""
    g = np.asarray(gpu, np.float64)
    d = g - ref
    return (float(np.linalg.norm(d) / (np.linalg.norm(ref) + 1e-300)),
            float(np.abs(d).max() / (np.asarray(scale, np.float64).max() + 1e-300)))


def test_bf16_pipeline_error_statement(gpu, oracle):
    log2_T = 21
    tree = scenes.make_octree(0, 4096 + 7 * 2000)
    grid = scenes.make_hashgrid(1, oracle.hash_entries(RES16, log2_T), RES16, log2_T)
    cam = scenes.make_camera((0.5, 0.5, -1.2), 300.0, 300.0, 320.0, 180.0, 640, 360)
    g_img = scenes.upstream_grad(2, (cam.height, cam.width, 64))
    n = 500_000
    c, l, w = (torch.from_numpy(x).to(gpu) for x in (tree.centers, tree.levels, tree.weights))
    tab16 = torch.from_numpy(grid.table).to(gpu).to(torch.bfloat16)
    desc = api.hashgrid_desc(RES16, log2_T, table_dtype=torch.bfloat16, out_dtype=torch.bfloat16)
    opts = api.RasterOptions(n_channels=64, head_mode=True, bf16=True)
    _, pos = api.sample_octree(c, l, w, 1.0, 0, 0, n)
    h = api.query_hashgrid(desc, tab16, pos)
    img, T, nc, ws = api.rasterize_fwd(cam, opts, pos, h)
    _, dh = api.rasterize_bwd(cam, opts, pos, h, None, T, nc, torch.from_numpy(g_img).to(gpu), ws)
    gt = torch.zeros(grid.table.shape, dtype=torch.float32, device=gpu)
    api.query_hashgrid_bwd(desc, pos, dh, gt)
    torch.cuda.synchronize()

    _, o_pos64, _ = oracle.sample_octree(tree, 0, 0, n)
    o_pos = o_pos64.astype(np.float32)
    o_h, o_hab = oracle.hash_fwd(RES16, log2_T, grid.table, o_pos, with_abs=True)
    ref = oracle.raster_fwd(cam, o_pos, o_h, head_mode=True, with_abs=True, feat_abs=o_hab)
    rb = oracle.raster_bwd(cam, o_pos, o_h, g_img, head_mode=True, with_abs=True, feat_abs=o_hab)
    o_gt, o_gab = oracle.hash_bwd(RES16, log2_T, 4, o_pos, rb["d_feat"], with_abs=True, dh_abs=rb["abs_feat"])

    stats = {
        "h": _err(h.float().cpu().numpy(), o_h, o_hab),
        "image": _err(img.float().cpu().numpy(), ref["image"], ref["abs"]),
        "T_final": _err(T.cpu().numpy(), ref["T_final"], ref["T_final"]),
        "dh": _err(dh.cpu().numpy(), rb["d_feat"], rb["abs_feat"]),
        "grad_table": _err(gt.cpu().numpy(), o_gt, o_gab),
    }
    for k, (mx, mean) in stats.items():
        print("BF16 form, %-10s norm-wise rel. error %.3e  max|err| / max sum|terms| %.3e" % (k, mx, mean))
    # BF16 storage of the table and of h: each value carries <= 2^-9 relative
    # rounding; the image adds its own output rounding; T and the gradients
    # inherit the rounding of h (alpha from h0, colors from h) only.
    assert stats["h"][0] < 2.0 ** -7
    assert stats["image"][0] < 2.0 ** -6
    assert stats["dh"][0] < 2.0 ** -5 and stats["grad_table"][0] < 2.0 ** -5
