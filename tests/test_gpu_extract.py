"""GPU viewpoint-independent pre-extraction and inference multisampling
(Sec. 3.2) against the oracle: level weights and Halton samples bit-exact,
the image accumulation to FP32 rounding, and a 4-fold multisampled render
(view-specific sampling with re-sampling, query, rasterizer, average) to
the condition-aware 1e-5 rule."""
import numpy as np
import pytest
import torch

from paper_2403_16862_gb300 import api, scenes
from tests._parity import assert_cond_close

pytestmark = pytest.mark.gpu

RES16 = scenes.geometric_resolutions(16, 16, 4096)


def test_level_weights_and_halton_bit_exact(gpu, oracle):
    tree = scenes.make_octree(0, 65536)
    c, l, p = (torch.from_numpy(x).to(gpu) for x in (tree.centers, tree.levels, tree.weights))
    w = api.level_weights(l, p, 0.5)
    ref_w = oracle.level_weights(tree.levels, tree.weights, 0.5)
    assert np.array_equal(w.cpu().numpy(), ref_w)
    n = 2_000_000
    leaf, pos = api.sample_octree_halton(c, l, w, tree.root_size, 21, n)
    o_leaf, o_pos = oracle.sample_halton(tree, ref_w, 21, n)
    assert np.array_equal(leaf.cpu().numpy(), o_leaf)
    assert np.array_equal(pos.cpu().numpy(), o_pos)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_accumulate_image(gpu, dtype):
    rng = np.random.default_rng(1)
    imgs = [torch.from_numpy(rng.normal(size=(37, 53, 64)).astype(np.float32)).to(gpu).to(dtype) for _ in range(4)]
    acc = torch.zeros(37, 53, 64, dtype=torch.float32, device=gpu)
    for im in imgs:
        api.accumulate_image(im, acc, 0.25)
    ref = sum(im.double() for im in imgs) * 0.25
    err = (acc.double() - ref).abs().max().item()
    assert err <= 4 * 2.0 ** -24 * ref.abs().max().item() + 1e-7


def test_multisampled_render(gpu, oracle):
    log2_T = 16
    tree = scenes.make_octree(2, 4096 + 7 * 600)
    grid = scenes.make_hashgrid(3, oracle.hash_entries(RES16, log2_T), RES16, log2_T)
    cam = scenes.orbit_cameras([(160, 104)], radius=1.3, focal_ref=120.0, ref_height=104)[0]
    c, l, p = (torch.from_numpy(x).to(gpu) for x in (tree.centers, tree.levels, tree.weights))
    desc = api.hashgrid_desc(RES16, log2_T)
    n, k = 60_000, 4
    img = api.multisample_render((c, l, p), tree.root_size, desc, torch.from_numpy(grid.table).to(gpu), cam, 5, n,
                                 k=k).cpu().numpy()
    w = oracle.view_weights(tree, cam)
    acc = np.zeros((cam.height, cam.width, 64))
    acc_abs = np.zeros_like(acc)
    flagged = np.zeros((cam.height, cam.width), bool)
    for v in range(k):
        _, pos, _ = oracle.sample_view(tree, w, cam, 5, v, n)
        h, hab = oracle.hash_fwd(RES16, log2_T, grid.table, pos, with_abs=True)
        ref = oracle.raster_fwd(cam, pos, h, head_mode=True, with_abs=True, feat_abs=hab)
        acc += ref["image"] / k
        acc_abs += ref["abs"] / k
        flagged |= ref["flags"] != 0
    assert flagged.sum() <= max(2, 1e-4 * flagged.size)
    assert_cond_close(img, acc, acc_abs, mask=~flagged[..., None], what="multisampled image")
