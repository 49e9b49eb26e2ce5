"""GPU rasterizer forward/backward against the oracle.

Images, T_final and gradients follow the condition-aware 1e-5 rule; the
per-pixel blended counts are exact.  Pixels whose stopping decision falls
within 1e-5 (relative) of t_min are excluded and counted (their count must
stay below 1e-4 of the pixels); gradients of points with a fragment in such
a pixel are excluded likewise."""
import numpy as np
import pytest
import torch

from paper_2403_16862_gb300 import api, scenes
from tests._parity import assert_cond_close

pytestmark = pytest.mark.gpu


def _run(gpu, cam, pos, feat, opacity, head, tile=(0, 0), g=None):
    opts = api.RasterOptions(n_channels=feat.shape[1], head_mode=head, tile_w=tile[0], tile_h=tile[1])
    P = torch.from_numpy(pos).to(gpu)
    Fe = torch.from_numpy(np.ascontiguousarray(feat, dtype=np.float32)).to(gpu)
    O = None if head else torch.from_numpy(opacity.astype(np.float32)).to(gpu)
    img, T, n, ws = api.rasterize_fwd(cam, opts, P, Fe, O)
    out = dict(image=img.cpu().numpy(), T_final=T.cpu().numpy(), n_contrib=n.cpu().numpy())
    if g is not None:
        d_op, d_feat = api.rasterize_bwd(cam, opts, P, Fe, O, T, n, torch.from_numpy(g).to(gpu), ws)
        out["d_feat"] = d_feat.cpu().numpy()
        if d_op is not None:
            out["d_opacity"] = d_op.cpu().numpy()
    torch.cuda.synchronize()
    return out


def _excluded_points(oracle, cam, pos, flags):
    cnt, ids, _, _ = oracle.fragment_lists(cam, pos)
    start = np.concatenate([[0], np.cumsum(cnt.ravel())])
    bad = np.zeros(pos.shape[0], bool)
    for q in np.flatnonzero(flags.ravel()):
        bad[ids[start[q]:start[q + 1]]] = True
    return bad


def _product_widening(oracle, cam, pos, n_contrib):
    """Per pixel and per point, max(1, n 2^-24 / 1e-5) for the longest blend
    n they take part in.  T_k is a product of k factors (1 - alpha); in FP32
    each factor adds up to 2^-24 of relative rounding, so for pixels that
    blend more than about 170 fragments the 1e-5 relative bound of every
    output carrying T_k widens to n 2^-24."""
    wp = np.maximum(1.0, n_contrib.astype(np.float64) * 2.0 ** -24 / 1e-5)
    cnt, ids, _, _ = oracle.fragment_lists(cam, pos)
    pix = np.repeat(np.arange(cnt.size), cnt.ravel())
    wpt = np.ones(pos.shape[0])
    np.maximum.at(wpt, ids, wp.ravel()[pix])
    return wp, wpt


def _compare(gpu, oracle, cam, pos, feat, opacity, head, tile=(0, 0), with_bwd=True, seed=0):
    g = np.random.default_rng(seed + 100).normal(size=(cam.height, cam.width, feat.shape[1])).astype(np.float32) \
        if with_bwd else None
    got = _run(gpu, cam, pos, feat, opacity, head, tile, g)
    ref = oracle.raster_fwd(cam, pos, feat, opacity=opacity, head_mode=head, with_abs=True)
    ok = ref["flags"] == 0
    n_flag = int((~ok).sum())
    assert n_flag <= max(2, 1e-4 * ok.size), "too many threshold-ambiguous pixels: %d" % n_flag
    assert np.array_equal(got["n_contrib"][ok], ref["n_contrib"][ok]), "blended counts"
    wp, wpt = _product_widening(oracle, cam, pos, ref["n_contrib"])
    assert_cond_close(got["image"], ref["image"], ref["abs"] * wp[..., None], mask=ok[..., None], what="image")
    assert_cond_close(got["T_final"], ref["T_final"], ref["T_final"] * wp, mask=ok, what="T_final")
    if with_bwd:
        rb = oracle.raster_bwd(cam, pos, feat, g, opacity=opacity, head_mode=head, with_abs=True)
        keep = ~_excluded_points(oracle, cam, pos, ref["flags"])
        assert_cond_close(got["d_feat"], rb["d_feat"], rb["abs_feat"] * wpt[:, None], mask=keep[:, None],
                          what="d_feat")
        if not head:
            assert_cond_close(got["d_opacity"], rb["d_opacity"], rb["abs_opacity"] * wpt, mask=keep,
                              what="d_opacity")
    return got, ref


def test_plain_rasterizer_workload(gpu, oracle):
    """65,536 points in [-1,1]^3, 8 features, 256x256, forward and backward."""
    pts, cam = scenes.raster_points_scene(seed=0)
    _compare(gpu, oracle, cam, pts.pos, pts.feat, pts.opacity, head=False)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (16, 8), (32, 8), (5, 7)])
def test_tile_shapes_and_ragged_image(gpu, oracle, tile):
    pts, cam = scenes.raster_points_scene(seed=1, n=20000, n_feat=4, size=100, focal=100.0)
    cam.width = 97  # ragged: not a multiple of any tile width
    cam.cx = 48.5
    _compare(gpu, oracle, cam, pts.pos, pts.feat, pts.opacity, head=False, tile=tile, seed=1)


@pytest.mark.parametrize("F", [1, 3, 4, 12, 64, 128])
def test_channel_counts(gpu, oracle, F):
    pts, cam = scenes.raster_points_scene(seed=2, n=8000, n_feat=F, size=48, focal=48.0)
    _compare(gpu, oracle, cam, pts.pos, pts.feat, pts.opacity, head=False, seed=F)


def test_head_mode(gpu, oracle):
    pts, cam = scenes.raster_points_scene(seed=3, n=30000, n_feat=64, size=128, focal=128.0)
    h = np.random.default_rng(4).normal(0.0, 0.6, size=(30000, 64)).astype(np.float32)
    got, ref = _compare(gpu, oracle, cam, pts.pos, h, None, head=True, seed=3)
    np.testing.assert_allclose(got["image"][..., 0], 1 - got["T_final"], atol=2e-6)


def test_overfull_tiles_take_the_global_sort(gpu, oracle):
    """Dense clusters: tiles far above the shared-memory capacity (8192
    forward, 4096 backward) and single pixels with thousands of fragments."""
    rng = np.random.default_rng(5)
    base, cam = scenes.raster_points_scene(seed=5, n=6000, n_feat=8, size=64, focal=64.0)
    cl1 = (np.array([0.1, -0.05, 0.0]) + rng.normal(0, 0.004, size=(15000, 3))).astype(np.float32)
    cl2 = (np.array([-0.4, 0.3, 0.2]) + rng.normal(0, 0.03, size=(6000, 3))).astype(np.float32)
    pos = np.concatenate([base.pos, cl1, cl2])
    n = pos.shape[0]
    opacity = rng.uniform(0.001, 0.02, size=n).astype(np.float32)  # long lists before T < 1e-4
    feat = rng.normal(size=(n, 8)).astype(np.float32)
    got, ref = _compare(gpu, oracle, cam, pos, feat, opacity, head=False, seed=5)
    assert ref["n_frags"].max() > 8192 // 4


def test_long_blends_64_channels(gpu, oracle):
    """64 channels (the fragment-slot layout) with faint splats: pixels that
    blend more than 256 fragments (CTA backward) and more than 2,048 (its
    global scratch), and large buckets whose nearest 256 fragments do not
    reach t_min (the forward's front selection falls back to the full
    sort)."""
    rng = np.random.default_rng(11)
    base, cam = scenes.raster_points_scene(seed=11, n=3000, n_feat=64, size=40, focal=40.0)
    cl = (np.array([0.05, 0.02, 0.0]) + rng.normal(0, 0.01, size=(9000, 3))).astype(np.float32)
    pos = np.concatenate([base.pos, cl])
    n = pos.shape[0]
    opacity = rng.uniform(0.002, 0.01, size=n).astype(np.float32)
    feat = rng.normal(size=(n, 64)).astype(np.float32)
    got, ref = _compare(gpu, oracle, cam, pos, feat, opacity, head=False, seed=11)
    assert ref["n_contrib"].max() > 2048


def test_empty_and_culled(gpu, oracle):
    pts, cam = scenes.raster_points_scene(seed=6, n=1000, n_feat=4, size=32, focal=32.0)
    got = _run(gpu, cam, pts.pos[:0], pts.feat[:0], pts.opacity[:0], False)
    assert np.all(got["image"] == 0) and np.all(got["T_final"] == 1) and np.all(got["n_contrib"] == 0)
    pos = pts.pos.copy()
    pos[:, 2] = -3.5  # all behind the camera
    g = np.ones((32, 32, 4), np.float32)
    got = _run(gpu, cam, pos, pts.feat, pts.opacity, False, g=g)
    assert np.all(got["n_contrib"] == 0) and np.all(got["d_feat"] == 0) and np.all(got["d_opacity"] == 0)
    pos = pts.pos.copy()
    pos[::2, 0] += 50.0  # half of them far outside the image
    _compare(gpu, oracle, cam, pos, pts.feat, pts.opacity, head=False, seed=6)


def test_duplicate_points_tie_break(gpu, oracle):
    pts, cam = scenes.raster_points_scene(seed=7, n=3000, n_feat=4, size=32, focal=32.0)
    pos = np.concatenate([pts.pos, pts.pos[:1500]])
    op = np.concatenate([pts.opacity, pts.opacity[:1500] * 0.5])
    fe = np.concatenate([pts.feat, -pts.feat[:1500]])
    _compare(gpu, oracle, cam, pos, fe, op, head=False, seed=7)


def test_autograd_wrapper(gpu):
    pts, cam = scenes.raster_points_scene(seed=8, n=5000, n_feat=4, size=32, focal=32.0)
    P = torch.from_numpy(pts.pos).to(gpu)
    Fe = torch.from_numpy(pts.feat).to(gpu).requires_grad_(True)
    O = torch.from_numpy(pts.opacity).to(gpu).requires_grad_(True)
    opts = api.RasterOptions(n_channels=4)
    img, T, n = api.Rasterize.apply(P, Fe, O, cam, opts)
    g = torch.randn_like(img)
    (img * g).sum().backward()
    img2, T2, n2, ws = api.rasterize_fwd(cam, opts, P, Fe.detach(), O.detach())
    d_op, d_feat = api.rasterize_bwd(cam, opts, P, Fe.detach(), O.detach(), T2, n2, g, ws)
    assert torch.equal(img, img2)
    assert torch.allclose(Fe.grad, d_feat, atol=1e-6) and torch.allclose(O.grad, d_op, atol=1e-6)


@pytest.mark.parametrize("near_far", [(0.01, 100.0), (1.9, 4.1)])
def test_more_than_2_25_points(gpu, oracle, near_far):
    """n = 2^25 + 8192 points: the forward's sort key carries 26-bit point
    indices and stores the depth as its FP32 bits above those of the near
    plane.  All but 16,384 points sit behind the camera (culled); the visible
    ones are 8,192 indices spread over [0, 2^25) and the 8,192 from 2^25 on,
    of which 2,048 duplicate a low-index point exactly (same depth and pixel:
    ties broken by the point index across the 2^25 boundary).  Culled points
    contribute nothing, so the oracle renders the visible points alone, in
    their original order, which keeps the (depth, index) order."""
    n_vis = 8192
    n = (1 << 25) + n_vis
    rng = np.random.default_rng(11)
    pts, cam = scenes.raster_points_scene(seed=11, n=2 * n_vis, n_feat=4, size=64, focal=64.0)
    cam.near, cam.far = near_far
    low = np.sort(rng.choice(1 << 25, size=n_vis, replace=False))
    vis = np.concatenate([low, (1 << 25) + np.arange(n_vis)])
    pos = np.empty((n, 3), np.float32)
    pos[:] = (0.0, 0.0, -10.0)  # behind the camera at z = -3
    pos[vis] = pts.pos
    pos[vis[n_vis:n_vis + 2048]] = pos[low[:2048]]
    feat = np.zeros((n, 4), np.float32)
    feat[vis] = pts.feat
    opacity = np.full(n, 0.5, np.float32)
    opacity[vis] = pts.opacity
    got = _run(gpu, cam, pos, feat, opacity, head=False)
    ref = oracle.raster_fwd(cam, pos[vis], feat[vis], opacity=opacity[vis], head_mode=False, with_abs=True)
    ok = ref["flags"] == 0
    assert int((~ok).sum()) <= 2
    assert np.array_equal(got["n_contrib"][ok], ref["n_contrib"][ok]), "blended counts"
    assert_cond_close(got["image"], ref["image"], ref["abs"], mask=ok[..., None], what="image")
    assert_cond_close(got["T_final"], ref["T_final"], ref["T_final"], mask=ok, what="T_final")
    assert ref["n_contrib"].max() > 1



@pytest.mark.parametrize("F", [8, 64])
def test_wide_depth_spans_and_exact_ties(gpu, oracle, F):
    """The register sorts order a bucket on 32-bit keys (depth relative to
    the bucket's nearest fragment) when the depths span fewer than 2^24 FP32
    values and no two are equal, and on the full keys otherwise.  Left half
    of the image: depths log-uniform in [0.05, 50] (spans of ~2^26 values);
    right half: depths in [2, 3], 3,000 exact duplicates (equal depth and
    pixel, ordered by point index) and a dense cluster for the CTA path."""
    rng = np.random.default_rng(21)
    W = H = 32
    cam = scenes.make_camera((0.0, 0.0, 0.0), 32.0, 32.0, 16.0, 16.0, W, H)
    n = 24000
    u = rng.uniform(0.0, W, n)
    v = rng.uniform(0.0, H, n)
    d = np.where(u < W / 2, np.exp(rng.uniform(np.log(0.05), np.log(50.0), n)), rng.uniform(2.0, 3.0, n))
    pos = np.stack([(u - 16.0) / 32.0 * d, (v - 16.0) / 32.0 * d, d], 1)
    cl = np.stack([np.full(1500, 0.1), np.full(1500, -0.05), rng.uniform(2.0, 2.5, 1500)], 1)
    pos = np.concatenate([pos, cl]).astype(np.float32)
    dup = rng.choice(np.flatnonzero(pos[:, 0] > 0), 3000, replace=False)
    pos = np.concatenate([pos, pos[dup]])
    n = pos.shape[0]
    opacity = rng.uniform(0.005, 0.05, n).astype(np.float32)
    feat = rng.normal(size=(n, F)).astype(np.float32)
    got, ref = _compare(gpu, oracle, cam, pos, feat, opacity, head=False, seed=F)
    assert ref["n_frags"].max() > 256 and ref["n_contrib"].max() > 64
