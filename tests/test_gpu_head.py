"""GPU view-dependent head (Sec. 3.3) against the oracle: the spherical
contraction bit-exact (FP32 with the same operation order), the SH head
forward and backward to the condition-aware 1e-5 rule, and the whole
view-dependent path (contraction -> query -> head -> 4-channel rasterizer,
and back into the table gradient) on a sampled scene."""
import numpy as np
import pytest
import torch

from paper_2403_16862_gb300 import api, scenes
from tests._parity import assert_cond_close
from tests.test_gpu_raster import _excluded_points, _product_widening

pytestmark = pytest.mark.gpu

RES16 = scenes.geometric_resolutions(16, 16, 4096)


def test_contraction_bit_exact(gpu, oracle):
    rng = np.random.default_rng(0)
    pos = np.concatenate([rng.normal(0, 1, (100_000, 3)), rng.normal(0, 30, (100_000, 3))]).astype(np.float32)
    center, radius = np.array([0.2, -0.1, 0.4], np.float32), 1.5
    q = api.contract_positions(torch.from_numpy(pos).to(gpu), center, radius).cpu().numpy()
    assert np.array_equal(q, oracle.contract(pos, center, radius))


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_sh_head_fwd_bwd(gpu, oracle, dtype):
    rng = np.random.default_rng(1)
    n, F = 50_000, 64
    cam = scenes.make_camera((0.3, -0.2, -2.0), 100.0, 100.0, 50.0, 40.0, 100, 80)
    pos = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    h32 = rng.normal(0, 0.5, (n, F)).astype(np.float32)
    h = torch.from_numpy(h32).to(gpu).to(dtype)
    hh = h.float().cpu().numpy()  # the values the kernel reads
    P = torch.from_numpy(pos).to(gpu)
    alpha, color = api.sh_head_fwd(cam, P, h)
    a, col, ab = oracle.sh_head_fwd(cam, pos, hh, with_abs=True)
    assert_cond_close(alpha.cpu().numpy(), a, a, what="alpha")
    assert_cond_close(color.cpu().numpy(), col, ab, what="color")
    da = rng.normal(size=n).astype(np.float32)
    dc = rng.normal(size=(n, 4)).astype(np.float32)
    dh = api.sh_head_bwd(cam, P, h, torch.from_numpy(da).to(gpu), torch.from_numpy(dc).to(gpu)).cpu().numpy()
    ref, rab = oracle.sh_head_bwd(cam, pos, hh, da, dc, with_abs=True)
    assert_cond_close(dh, ref, rab, what="dh")


def test_view_dependent_path(gpu, oracle):
    log2_T = 16
    tree = scenes.make_octree(5, 4096 + 7 * 700)
    grid = scenes.make_hashgrid(6, oracle.hash_entries(RES16, log2_T), RES16, log2_T)
    cam = scenes.orbit_cameras([(192, 128)], radius=1.6, focal_ref=150.0, ref_height=128)[0]
    c, l, w = (torch.from_numpy(x).to(gpu) for x in (tree.centers, tree.levels, tree.weights))
    n = 120_000
    _, pos = api.sample_octree(c, l, w, tree.root_size, 4, 0, n)
    center, radius = np.array([0.5, 0.5, 0.5], np.float32), 0.5
    desc = api.hashgrid_desc(RES16, log2_T)
    g_img = scenes.upstream_grad(7, (cam.height, cam.width, 4))
    gt = torch.zeros(grid.table.shape, dtype=torch.float32, device=gpu)
    img, T, nc = api.render_view_sh(pos, desc, torch.from_numpy(grid.table).to(gpu), cam, center, radius,
                                    d_image=torch.from_numpy(g_img).to(gpu), grad_table=gt)
    # oracle: its own samples, the same steps
    _, o_pos64, _ = oracle.sample_octree(tree, 4, 0, n)
    o_pos = o_pos64.astype(np.float32)
    q = oracle.contract(o_pos, center, radius)
    h, hab = oracle.hash_fwd(RES16, log2_T, grid.table, q, with_abs=True)
    a, col, cab = oracle.sh_head_fwd(cam, o_pos, h, with_abs=True)
    ref = oracle.raster_fwd(cam, o_pos, col, opacity=a, with_abs=True, feat_abs=cab)
    ok = ref["flags"] == 0
    assert (~ok).sum() <= max(2, 1e-4 * ok.size)
    assert np.array_equal(nc.cpu().numpy()[ok], ref["n_contrib"][ok])
    assert_cond_close(img.cpu().numpy(), ref["image"], ref["abs"], mask=ok[..., None], what="image")
    rb = oracle.raster_bwd(cam, o_pos, col, g_img, opacity=a, with_abs=True, feat_abs=cab)
    dh, dhab = oracle.sh_head_bwd(cam, o_pos, h, rb["d_opacity"], rb["d_feat"], with_abs=True)
    # the head's backward scales each incoming term by |Y|_k or by the
    # opacity derivative: carry the rasterizer's sum of |terms| through it,
    # widened for points in long blends (an n-factor FP32 product of 1 - alpha
    # carries up to n 2^-24 relative rounding)
    _, wpt = _product_widening(oracle, cam, o_pos, ref["n_contrib"])
    _, scale = oracle.sh_head_bwd(cam, o_pos, h, rb["abs_opacity"] * wpt, rb["abs_feat"] * wpt[:, None],
                                  with_abs=True)
    o_gt, o_gab = oracle.hash_bwd(RES16, log2_T, 4, q, dh, with_abs=True, dh_abs=scale)
    keep = ~_excluded_points(oracle, cam, o_pos, ref["flags"])
    reach = oracle.hash_bwd(RES16, log2_T, 4, q, np.repeat((~keep)[:, None], 64, 1).astype(np.float64))
    assert_cond_close(gt.cpu().numpy(), o_gt, o_gab, mask=reach == 0, what="grad_table")
