"""Pins of the oracle's octree maintenance (Sec. 3.1 "Probability Updates"
Eq. 2 / Eq. 3, "Subdivision", "Pruning"; App. A.4 leaf layout; App. A.6's
bilinear-weighted per-point blending weights): a hand-derived single-point
weight, two stacked points in closed form, the telescoping identity
sum_k T_k alpha_k = 1 - T_final per pixel (against the separate forward),
hand-worked Eq. 2/3 updates, subdivision of a full grid reproducing the
next finer grid in Morton order, the leaf-count cap, and pruning.  CPU
only."""
import json
import os

import numpy as np
import pytest

from paper_2403_16862_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cam(fx=1.0, fy=1.0, cx=10.0, cy=20.0, W=32, H=32):
    return scenes.Camera(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=fx, fy=fy, cx=cx, cy=cy,
                         width=W, height=H)


def test_single_point_weight_golden(oracle):
    g = json.load(open(os.path.join(GOLDEN, "single_point_splat.json")))
    c = g["camera"]
    cam = _cam(c["fx"], c["fy"], c["cx"], c["cy"], c["width"], c["height"])
    b = oracle.point_weights(cam, np.array([g["point"]], np.float32), np.array([g["feature"]]),
                             opacity=np.array([g["alpha_h"]]))
    assert b[0] == pytest.approx(g["blend_weight"], rel=1e-15)


def test_two_stacked_points_closed_form(oracle):
    """Both points project onto the center of pixel (10, 20) (weight 1 there,
    0 at the other three corners): the front one gets alpha_f, the back one
    (1 - alpha_f) alpha_b."""
    cam = _cam()
    pos = np.array([[0.5, 0.5, 1.0], [1.0, 1.0, 2.0]], np.float32)  # u = 10.5, v = 20.5 for both
    af, ab = 0.3, 0.6
    b = oracle.point_weights(cam, pos, np.zeros((2, 1)), opacity=np.array([af, ab]))
    assert b[0] == pytest.approx(af, rel=1e-15)
    assert b[1] == pytest.approx((1 - af) * ab, rel=1e-15)


@pytest.mark.parametrize("head", [False, True])
def test_pixel_weight_sums_telescope(oracle, head):
    pts, cam = scenes.raster_points_scene(seed=3, n=20000, n_feat=4, size=64, focal=64.0)
    feat = np.random.default_rng(1).normal(0, 0.5, size=(20000, 4)) if head else pts.feat
    op = None if head else pts.opacity
    b, ps = oracle.point_weights(cam, pts.pos, feat, opacity=op, head_mode=head, with_pixel_sums=True)
    fwd = oracle.raster_fwd(cam, pts.pos, feat, opacity=op, head_mode=head)
    np.testing.assert_allclose(ps, 1.0 - fwd["T_final"], atol=1e-12)
    assert np.all(b >= 0.0) and np.all(b <= 1.0)
    # the bilinear weighting makes the per-point weights sum to less than the
    # per-splat weights (w_k <= 1), with equality only for single-pixel splats
    assert b.sum() <= ps.sum() + 1e-9


def test_update_hand_example(oracle):
    # leaf 0: b in {0.2, 0.5}; leaf 1: no point; leaf 2: b = {0.1}; leaf 3: b = {0.75, 0.75}
    leaf = np.array([0, 2, 0, 3, 3])
    b = np.array([0.2, 0.1, 0.5, 0.75, 0.75], np.float32)
    p = np.array([0.9, 0.8, 1.0, 0.25])
    q = np.array([0.1, 0.6, 0.4, 0.2])
    lam = 0.5
    pn, qn = oracle.octree_update(leaf, b, p, q, lam)
    exp_p = [max(0.45, float(np.float32(0.5))), 0.4, max(0.5, float(np.float32(0.1))), float(np.float32(0.75))]
    exp_q = [max(0.05, float(np.float32(0.5)) - float(np.float32(0.2))), 0.3, max(0.2, 0.0), max(0.1, 0.0)]
    assert pn.tolist() == exp_p
    assert qn.tolist() == exp_q


def test_update_decay_and_fixed_point(oracle):
    rng = np.random.default_rng(2)
    L = 50
    p, q = rng.uniform(0, 1, L), rng.uniform(0, 1, L)
    pn, qn = oracle.octree_update(np.zeros(0, np.int32), np.zeros(0, np.float32), p, q, 0.9968)
    assert np.array_equal(pn, 0.9968 * p) and np.array_equal(qn, 0.9968 * q)
    # lambda = 1 and the same weights twice: the second update changes nothing
    leaf = rng.integers(0, L, 400)
    b = rng.uniform(0, 1, 400).astype(np.float32)
    p1, q1 = oracle.octree_update(leaf, b, p, q, 1.0)
    p2, q2 = oracle.octree_update(leaf, b, p1, q1, 1.0)
    assert np.array_equal(p1, p2) and np.array_equal(q1, q2)
    with pytest.raises(Exception):
        oracle.octree_update(np.array([L]), np.array([0.5], np.float32), p, q)


def _grid(level):
    g = 1 << level
    ii = np.arange(g)
    ix, iy, iz = (a.ravel() for a in np.meshgrid(ii, ii, ii, indexing="ij"))
    order = np.argsort(scenes.morton3(ix, iy, iz, level), kind="stable")
    ix, iy, iz = ix[order], iy[order], iz[order]
    e = 2.0 ** -level
    c = np.stack([(ix + 0.5) * e, (iy + 0.5) * e, (iz + 0.5) * e], 1).astype(np.float32)
    return c, np.full(ix.size, level, np.int32)


def test_subdivide_full_grid_gives_next_grid(oracle):
    c4, l4 = _grid(3)
    p = np.linspace(0.1, 1.0, c4.shape[0])
    q = np.ones(c4.shape[0])
    c, lv, pn, qn = oracle.octree_subdivide(c4, l4, p, q, root_size=1.0, tau_s=0.5)
    c5, l5 = _grid(4)
    assert np.array_equal(c, c5) and np.array_equal(lv, l5)
    assert np.array_equal(pn, np.repeat(p, 8)) and np.all(qn == 0.0)


def test_subdivide_geometry_and_cap(oracle):
    tree = scenes.make_octree(4, 4096 + 7 * 100)
    rng = np.random.default_rng(5)
    q = rng.uniform(0, 1, tree.n_leaves)
    q[:10] = 0.5  # exactly the threshold: not subdivided (strictly greater)
    c, lv, pn, qn = oracle.octree_subdivide(tree.centers, tree.levels, tree.weights, q)
    k = int((q > 0.5).sum())
    assert c.shape[0] == tree.n_leaves + 7 * k
    # every leaf's volume fraction is 8^-level: the total is conserved
    assert np.sum(8.0 ** -lv.astype(np.float64)) == pytest.approx(np.sum(8.0 ** -tree.levels.astype(np.float64)),
                                                                  rel=1e-15)
    # children lie inside their parent, in order
    o = 0
    for i in range(tree.n_leaves):
        if q[i] > 0.5:
            half = 2.0 ** -tree.levels[i] / 2
            ch = c[o:o + 8].astype(np.float64)
            assert np.all(np.abs(ch - tree.centers[i]) == half / 2)
            assert np.all(lv[o:o + 8] == tree.levels[i] + 1)
            o += 8
        else:
            assert np.array_equal(c[o], tree.centers[i]) and qn[o] == q[i]
            o += 1
    # the cap: the resulting count must stay below max_leaves
    c2, _, _, _ = oracle.octree_subdivide(tree.centers, tree.levels, tree.weights, q,
                                          max_leaves=tree.n_leaves + 7 * k)
    assert c2.shape[0] == tree.n_leaves
    c3, _, _, _ = oracle.octree_subdivide(tree.centers, tree.levels, tree.weights, q,
                                          max_leaves=tree.n_leaves + 7 * k + 1)
    assert c3.shape[0] == tree.n_leaves + 7 * k


def test_prune(oracle):
    tree = scenes.make_octree(6, 4096 + 7 * 50)
    rng = np.random.default_rng(6)
    p = rng.uniform(0, 0.03, tree.n_leaves)
    p[:5] = 0.01  # at the threshold: kept
    q = rng.uniform(0, 1, tree.n_leaves)
    c, lv, pn, qn = oracle.octree_prune(tree.centers, tree.levels, p, q, tau_p=0.01)
    keep = p >= 0.01
    assert c.shape[0] == keep.sum()
    assert np.array_equal(c, tree.centers[keep]) and np.array_equal(lv, tree.levels[keep])
    assert np.array_equal(pn, p[keep]) and np.array_equal(qn, q[keep])
