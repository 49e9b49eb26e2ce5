"""Pins of the oracle's view-specific re-weighting (Sec. 3.2 Eq. 4, App. A.4
"Depth Calculation") and visibility re-sampling (App. A.4 "Ensuring Sample
Count"): the frustum test against brute-force point sampling of each leaf
cube (it never culls a cube with a visible point, and every culled cube has
none), the factors of Eq. 4 as ratios (depth, level, linearity in p, the
tau_d clamp), and the re-sampling rounds (every sample ends in view, samples
already in view are untouched, redrawn samples come from visible leaves and
lie in them).  CPU only."""
import numpy as np
import pytest

from paper_2403_16862_gb300 import scenes


def _cam(W=100, H=80, f=100.0):
    return scenes.Camera(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=f, fy=f, cx=W / 2.0,
                         cy=H / 2.0, width=W, height=H, near=0.01, far=100.0)


def _tree(centers, levels, p=None, root=1.0):
    centers = np.asarray(centers, np.float32)
    levels = np.asarray(levels, np.int32)
    p = np.ones(levels.shape[0]) if p is None else np.asarray(p, np.float64)
    return scenes.Octree(centers=centers, levels=levels, weights=p, root_size=root)


def test_frustum_test_against_point_sampling(oracle):
    """A cube is culled only if none of its points is in view (conservative),
    checked with 4,096 points per cube; cubes culled here have no visible
    point at all."""
    rng = np.random.default_rng(0)
    cam = _cam()
    n = 300
    lv = rng.integers(1, 4, n).astype(np.int32)
    centers = np.stack([rng.uniform(-3, 3, n), rng.uniform(-3, 3, n), rng.uniform(-1.5, 6, n)], 1)
    tree = _tree(centers, lv)
    w = oracle.view_weights(tree, cam, lambda_l=0.0)
    g = (np.arange(16) + 0.5) / 16 - 0.5
    grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    culled = visible_seen = 0
    for i in range(n):
        pts = (centers[i] + grid * 2.0 ** -lv[i]).astype(np.float32)
        any_in = oracle.points_in_view(cam, pts).any()
        if w[i] == 0.0:
            culled += 1
            assert not any_in, "cube %d culled but has a point in view" % i
        elif any_in:
            visible_seen += 1
    assert culled > 50 and visible_seen > 50


def test_eq4_factors(oracle):
    cam = _cam()
    near = float(np.float32(0.01))
    # same level, two depths: weights inversely proportional to |z - near|
    tree = _tree([[0.0, 0.0, 2.0], [0.0, 0.0, 5.0]], [3, 3])
    w = oracle.view_weights(tree, cam, lambda_l=0.5)
    assert w[0] / w[1] == pytest.approx((5.0 - near) / (2.0 - near), rel=1e-14)
    # same depth, levels l and l + 1: the coarser leaf weighs 2^lambda_l more
    tree = _tree([[0.0, 0.0, 3.0], [0.0, 0.0, 3.0]], [2, 3])
    for lam in (0.0, 0.5, 1.0):
        w = oracle.view_weights(tree, cam, lambda_l=lam)
        assert w[0] / w[1] == pytest.approx(2.0 ** lam, rel=1e-14)  # the finer leaf is sampled less
    # linear in p; an invisible leaf (behind the camera) has weight 0
    tree = _tree([[0.0, 0.0, 3.0], [0.0, 0.0, -3.0]], [4, 4], p=[0.25, 1.0])
    w1 = oracle.view_weights(tree, cam)
    tree2 = _tree([[0.0, 0.0, 3.0], [0.0, 0.0, -3.0]], [4, 4], p=[0.75, 1.0])
    w3 = oracle.view_weights(tree2, cam)
    assert w3[0] == pytest.approx(3 * w1[0], rel=1e-15) and w1[1] == 0.0 and w3[1] == 0.0
    # tau_d: a leaf centered on the near plane gets d = tau_d
    tree = _tree([[0.0, 0.0, near], [0.0, 0.0, 1.0]], [6, 6])
    w = oracle.view_weights(tree, cam, lambda_l=0.0, tau_d=1e-8)
    assert w[0] == pytest.approx(1e8, rel=1e-12)


def _straddling_scene():
    """A 16^3 grid of the cube [-1, 1]^3 seen from z = -2.2 with a narrow
    field of view, so that many leaves straddle the frustum's side planes."""
    g = 16
    ii = (np.arange(g) + 0.5) / g * 2.0 - 1.0
    c = np.stack(np.meshgrid(ii, ii, ii, indexing="ij"), -1).reshape(-1, 3)
    tree = scenes.Octree(centers=c.astype(np.float32), levels=np.full(c.shape[0], 4, np.int32),
                         weights=np.random.default_rng(1).lognormal(0, 1, c.shape[0]), root_size=2.0)
    cam = scenes.make_camera((0.0, 0.0, -2.2), 60.0, 60.0, 32.0, 24.0, 64, 48)
    return tree, cam


def test_resampling_rounds(oracle):
    tree, cam = _straddling_scene()
    w = oracle.view_weights(tree, cam)
    assert (w == 0).sum() > 100 and (w > 0).sum() > 100
    n = 50_000
    view_tree = scenes.Octree(centers=tree.centers, levels=tree.levels, weights=w, root_size=tree.root_size)
    leaf0, pos64, _ = oracle.sample_octree(view_tree, 3, 2, n)
    pos0 = pos64.astype(np.float32)
    ok0 = oracle.points_in_view(cam, pos0)
    assert 0.02 < 1 - ok0.mean() < 0.6  # straddling leaves put a share of the samples out of view
    leaf, pos, left = oracle.sample_view(tree, w, cam, 3, 2, n, max_rounds=32)
    assert left == 0 and oracle.points_in_view(cam, pos).all()
    assert np.array_equal(leaf[ok0], leaf0[ok0]) and np.array_equal(pos[ok0], pos0[ok0])
    moved = ~ok0
    assert np.all(w[leaf[moved]] > 0)
    half = 0.5 * tree.root_size * 2.0 ** -tree.levels[leaf[moved]]
    assert np.all(np.abs(pos[moved] - tree.centers[leaf[moved]]) <= half[:, None])
    # one round leaves some samples out of view, and the count says so
    _, pos1, left1 = oracle.sample_view(tree, w, cam, 3, 2, n, max_rounds=1)
    assert left1 == (~oracle.points_in_view(cam, pos1)).sum() > 0
