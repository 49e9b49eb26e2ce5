"""GPU octree maintenance against the oracle: the per-point blending weights
of a forward (condition-aware 1e-5 rule; every term is non-negative), the
Eq. 2 / Eq. 3 update, subdivision and pruning (bit-exact: the same FP32
inputs, max / min and one FP64 rounding per value, exact copies and dyadic
child centers)."""
import numpy as np
import pytest
import torch

from paper_2403_16862_gb300 import _binding as B
from paper_2403_16862_gb300 import api, scenes
from tests._parity import assert_cond_close

pytestmark = pytest.mark.gpu

RES16 = scenes.geometric_resolutions(16, 16, 4096)


def test_point_weights_given_opacity(gpu, oracle):
    pts, cam = scenes.raster_points_scene(seed=0, n=30000, n_feat=8, size=96, focal=96.0)
    opts = api.RasterOptions(n_channels=8)
    P = torch.from_numpy(pts.pos).to(gpu)
    img, T, nc, ws = api.rasterize_fwd(cam, opts, P, torch.from_numpy(pts.feat).to(gpu),
                                       torch.from_numpy(pts.opacity).to(gpu))
    b = api.point_weights(cam, opts, P, nc, ws).cpu().numpy()
    ref = oracle.point_weights(cam, pts.pos, pts.feat, opacity=pts.opacity)
    assert_cond_close(b, ref, ref, what="b")
    assert (ref > 0).sum() > 1000


@pytest.mark.parametrize("n_samples,size", [(200_000, (320, 208)), (4_194_304, (1280, 832))])
def test_point_weights_pipeline(gpu, oracle, n_samples, size):
    """Head mode on the sampled scene; the second case is the full
    benchmark view."""
    log2_T = 19
    tree = scenes.make_octree(0, 65536)
    grid = scenes.make_hashgrid(1, oracle.hash_entries(RES16, log2_T), RES16, log2_T)
    W, H = size
    f = 900.0 * W / 1280
    cam = scenes.make_camera((0.5, 0.5, -1.2), f, f, W / 2.0, H / 2.0, W, H)
    c, l, w = (torch.from_numpy(x).to(gpu) for x in (tree.centers, tree.levels, tree.weights))
    desc = api.hashgrid_desc(RES16, log2_T)
    opts = api.RasterOptions(n_channels=64, head_mode=True)
    _, pos = api.sample_octree(c, l, w, tree.root_size, 0, 0, n_samples)
    h = api.query_hashgrid(desc, torch.from_numpy(grid.table).to(gpu), pos)
    img, T, nc, ws = api.rasterize_fwd(cam, opts, pos, h)
    b = api.point_weights(cam, opts, pos, nc, ws).cpu().numpy()
    _, o_pos64, _ = oracle.sample_octree(tree, 0, 0, n_samples)
    o_pos = o_pos64.astype(np.float32)
    o_h = oracle.hash_fwd(RES16, log2_T, grid.table, o_pos)
    ref = oracle.raster_fwd(cam, o_pos, o_h, head_mode=True)
    ok = ref["flags"] == 0
    assert np.array_equal(nc.cpu().numpy()[ok], ref["n_contrib"][ok])
    o_b = oracle.point_weights(cam, o_pos, o_h, head_mode=True)
    # points with a fragment in a threshold-ambiguous pixel are excluded
    cnt, ids, _, _ = oracle.fragment_lists(cam, o_pos)
    start = np.concatenate([[0], np.cumsum(cnt.ravel())])
    keep = np.ones(n_samples, bool)
    for q in np.flatnonzero(~ok.ravel()):
        keep[ids[start[q]:start[q + 1]]] = False
    # h carries the query's own relative rounding into alpha_h: the terms'
    # scale is b itself
    assert_cond_close(b, o_b, o_b, mask=keep, what="b")


def _leaves(seed, L, n, grouped=True):
    rng = np.random.default_rng(seed)
    leaf = rng.integers(0, L - L // 50, n).astype(np.int32)  # the last 2 % of the leaves get no point
    if grouped:
        leaf = np.sort(leaf)  # as the sampler emits them
    b = rng.uniform(0, 1, n).astype(np.float32)
    b[rng.random(n) < 0.2] = 0.0
    p = rng.uniform(0, 1, L)
    q = rng.uniform(0, 1, L)
    return leaf, b, p, q


@pytest.mark.parametrize("grouped", [True, False])
def test_update_bit_exact(gpu, oracle, grouped):
    L, n = 70_000, 3_000_000
    leaf, b, p, q = _leaves(1, L, n, grouped)
    P, Q = torch.from_numpy(p).to(gpu), torch.from_numpy(q).to(gpu)
    api.octree_update(torch.from_numpy(leaf).to(gpu), torch.from_numpy(b).to(gpu), P, Q, 0.9968)
    o_p, o_q = oracle.octree_update(leaf, b, p, q, 0.9968)
    assert np.array_equal(P.cpu().numpy(), o_p) and np.array_equal(Q.cpu().numpy(), o_q)
    assert len(np.setdiff1d(np.arange(L), leaf)) > 0  # some leaves only decay


def test_update_status_bits(gpu):
    L = 8
    p = torch.full((L,), 0.25, dtype=torch.float64, device=gpu)
    q = torch.zeros(L, dtype=torch.float64, device=gpu)
    ws = api.workspace(B.inpc_octree_update_workspace_size(L), gpu)
    leaf = torch.tensor([0, 1, 9, 2], dtype=torch.int32, device=gpu)
    b = torch.tensor([0.5, -0.25, 0.5, float("nan")], dtype=torch.float32, device=gpu)
    api.octree_update(leaf, b, p, q, 1.0, ws=ws)
    st = api.read_device_status(ws)
    assert st & B.INPC_DEV_BAD_LEAF and st & B.INPC_DEV_BAD_BLEND_WEIGHT
    # the bad values count as weight 0; the out-of-range point is ignored
    assert p.cpu().tolist() == [0.5] + [0.25] * 7 and q.cpu().tolist() == [0.0] * 8


def _tree_and_q(seed, n_leaves):
    tree = scenes.make_octree(seed, n_leaves)
    q = np.random.default_rng(seed + 1).uniform(0, 1, tree.n_leaves)
    return tree, q


def _to(gpu, *arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(gpu) for a in arrays]


def test_subdivide_bit_exact(gpu, oracle):
    tree, q = _tree_and_q(2, 65536)
    q[:100] = 0.5
    c, lv, p, qq = _to(gpu, tree.centers, tree.levels, tree.weights, q)
    got = api.octree_subdivide(c, lv, p, qq, tree.root_size, tau_s=0.5)
    ref = oracle.octree_subdivide(tree.centers, tree.levels, tree.weights, q, root_size=tree.root_size, tau_s=0.5)
    assert got[0].shape[0] == ref[0].shape[0] > tree.n_leaves
    for g, r in zip(got, ref):
        assert np.array_equal(g.cpu().numpy(), r)
    # the leaf cap: no subdivision when the count would reach max_leaves
    n_new = ref[0].shape[0]
    got = api.octree_subdivide(c, lv, p, qq, tree.root_size, tau_s=0.5, max_leaves=n_new)
    assert got[0].shape[0] == tree.n_leaves and np.array_equal(got[0].cpu().numpy(), tree.centers)
    # too small an output is refused before anything is written
    ws = api.workspace(B.inpc_octree_refine_workspace_size(tree.n_leaves), gpu)
    small = torch.empty(tree.n_leaves + 1, 3, dtype=torch.float32, device=gpu)
    sl = torch.empty(tree.n_leaves + 1, dtype=torch.int32, device=gpu)
    sp = torch.empty(tree.n_leaves + 1, dtype=torch.float64, device=gpu)
    t = B.InpcOctree(c.data_ptr(), lv.data_ptr(), p.data_ptr(), tree.root_size, tree.n_leaves)
    with pytest.raises(B.InpcError, match="CAPACITY"):
        B.inpc_octree_subdivide(t, qq.data_ptr(), 0.5, 256 ** 3, small.data_ptr(), sl.data_ptr(), sp.data_ptr(),
                                sp.data_ptr(), tree.n_leaves + 1, ws.data_ptr(), ws.numel(),
                                torch.cuda.current_stream().cuda_stream)


def test_prune_bit_exact(gpu, oracle):
    tree, q = _tree_and_q(3, 65536)
    p = tree.weights * tree.n_leaves * 0.02  # mean 0.02: a large share below 0.01
    p[:50] = 0.01
    c, lv, pp, qq = _to(gpu, tree.centers, tree.levels, p, q)
    got = api.octree_prune(c, lv, pp, qq, tree.root_size, tau_p=0.01)
    ref = oracle.octree_prune(tree.centers, tree.levels, p, q, tau_p=0.01)
    assert 0 < ref[0].shape[0] < tree.n_leaves
    for g, r in zip(got, ref):
        assert np.array_equal(g.cpu().numpy(), r)


def test_maintenance_cycle_keeps_the_sampler_valid(gpu, oracle):
    """update -> subdivide -> prune on the GPU, then the sampler draws from
    the refined tree bit-exactly like the oracle does from the same tree."""
    tree, q = _tree_and_q(4, 20000)
    c, lv, p, qq = _to(gpu, tree.centers, tree.levels, tree.weights.copy(), q)
    leaf, b, _, _ = _leaves(5, tree.n_leaves, 400_000)
    api.octree_update(torch.from_numpy(leaf).to(gpu), torch.from_numpy(b).to(gpu), p, qq, 0.9968)
    c, lv, p, qq = api.octree_subdivide(c, lv, p, qq, tree.root_size, tau_s=0.5)
    c, lv, p, qq = api.octree_prune(c, lv, p, qq, tree.root_size, tau_p=0.01)
    new = scenes.Octree(centers=c.cpu().numpy(), levels=lv.cpu().numpy(), weights=p.cpu().numpy(),
                        root_size=tree.root_size)
    g_leaf, g_pos = api.sample_octree(c, lv, p, tree.root_size, 7, 1, 300_000)
    o_leaf, o_pos, _ = oracle.sample_octree(new, 7, 1, 300_000)
    assert np.array_equal(g_leaf.cpu().numpy(), o_leaf)
    assert np.array_equal(g_pos.cpu().numpy(), o_pos.astype(np.float32))
