"""The seeded input generators against the recipe they implement (CPU).

Every parity test and the benchmark draw their inputs from
``paper_2403_16862_gb300.scenes``; these checks pin the generated scenes to
the stated recipe: the sparse octree (exact leaf count, disjoint leaves in
Morton order, centers on their leaf grid, log-normal weights summing to
one), the grid resolutions, the table entry distribution, the plain
rasterizer scene and the orbit cameras."""
import math

import numpy as np
import pytest

from paper_2403_16862_gb300 import scenes


def _interleave(x, y, z, bits):
    """Morton code with x in the lowest bit of each triple, written out bit by
    bit for single integers."""
    code = 0
    for b in range(bits):
        code |= ((x >> b) & 1) << (3 * b)
        code |= ((y >> b) & 1) << (3 * b + 1)
        code |= ((z >> b) & 1) << (3 * b + 2)
    return code


def test_morton_bit_order():
    assert [int(scenes.morton3(np.array([x]), np.array([y]), np.array([z]), 12)[0])
            for x, y, z in ((1, 0, 0), (0, 1, 0), (0, 0, 1), (3, 0, 0), (0, 0, 2), (5, 6, 7))] == \
        [1, 2, 4, 9, 32, _interleave(5, 6, 7, 12)]


@pytest.mark.parametrize("n_leaves,start", [(65536, 4), (4096 + 7 * 300, 4), (1 << 20, 6)])
def test_octree_recipe(n_leaves, start):
    t = scenes.make_octree(0, n_leaves, start_level=start)
    L = t.centers.shape[0]
    assert L == n_leaves == t.n_leaves
    assert t.root_size == 1.0
    lv = t.levels.astype(np.int64)
    assert lv.min() >= start and lv.max() <= 12
    # centers are (i + 1/2) 2^-l exactly (FP32 holds them exactly)
    scale = np.exp2(lv.astype(np.float64))[:, None]
    idx = np.rint(t.centers.astype(np.float64) * scale - 0.5)
    assert np.all(idx >= 0) and np.all(idx < scale)
    assert np.array_equal(((idx + 0.5) / scale).astype(np.float32), t.centers)
    # disjoint leaf cubes, in ascending Morton order of their minimum corner
    # at level 12: leaf k covers the code range [code_k, code_k + 8^(12 - l))
    ii = idx.astype(np.int64)
    s = 12 - lv
    lo = scenes.morton3(ii[:, 0] << s, ii[:, 1] << s, ii[:, 2] << s, 12).astype(np.int64)
    span = np.left_shift(np.int64(1), 3 * s)
    assert np.all(np.diff(lo) > 0), "Morton order"
    assert np.all(lo[1:] >= lo[:-1] + span[:-1]), "leaves overlap"
    for k in (0, L // 3, L - 1):  # the vectorised codes match the bit-by-bit interleave
        assert lo[k] == _interleave(int(ii[k, 0]) << int(s[k]), int(ii[k, 1]) << int(s[k]),
                                    int(ii[k, 2]) << int(s[k]), 12)
    # pruning removes leaves, so the leaves cover at most the unit cube
    assert float(np.sum(np.exp2(-3.0 * lv))) <= 1.0
    # weights: positive, normalised, log-normal with sigma 1.5
    w = t.weights
    assert w.dtype == np.float64 and np.all(w > 0)
    assert abs(float(w.sum()) - 1.0) < 1e-12
    if L >= 65536:
        assert abs(float(np.std(np.log(w))) - 1.5) < 0.03


def test_octree_is_seeded():
    a, b, c = scenes.make_octree(7, 5000), scenes.make_octree(7, 5000), scenes.make_octree(8, 5000)
    assert np.array_equal(a.centers, b.centers) and np.array_equal(a.weights, b.weights)
    assert not np.array_equal(a.weights, c.weights)


def test_grid_resolutions_and_table():
    # 16 b^l for l = 0..15 with b = 256^(1/15), floored: 16 to 4096 over 16 levels
    assert scenes.geometric_resolutions(16, 16, 4096) == \
        [16, 23, 33, 48, 70, 101, 147, 212, 307, 445, 645, 933, 1351, 1955, 2830, 4096]
    g = scenes.make_hashgrid(1, 200_000, [16, 32], 17)
    assert g.table.dtype == np.float32 and g.table.shape == (200_000, 4)
    t = g.table.astype(np.float64)
    # U(-1e-4, 1e-4) + N(0, 0.1): mean 0, variance 0.01 + (2e-4)^2 / 12
    assert abs(t.mean()) < 1e-3
    assert abs(t.std() - math.sqrt(0.01 + 4e-8 / 12)) < 1e-3


def test_plain_rasterizer_scene():
    pts, cam = scenes.raster_points_scene(seed=0)
    assert pts.pos.shape == (65536, 3) and pts.feat.shape == (65536, 8)
    assert pts.pos.min() >= -1 and pts.pos.max() <= 1
    assert pts.opacity.min() >= 0.05 and pts.opacity.max() <= 0.95
    assert abs(float(pts.feat.std()) - 1.0) < 0.01
    assert (cam.width, cam.height, cam.fx, cam.cx) == (256, 256, 256.0, 128.0)
    # camera at (0, 0, -3) looking down +z: t = -R p
    assert np.allclose(cam.t, [0.0, 0.0, 3.0]) and np.allclose(cam.R, np.eye(3))


def test_orbit_cameras():
    sizes = [(640, 480), (960, 540), (1920, 1080), (1280, 832)]
    cams = scenes.orbit_cameras(sizes)
    c = np.array([0.5, 0.5, 0.5])
    for (w, h), cam in zip(sizes, cams):
        R = cam.R.astype(np.float64)
        t = cam.t.astype(np.float64)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-6)
        eye = -R.T @ t
        d = eye - c
        assert abs(math.hypot(d[0], d[2]) - 1.7) < 1e-5 and abs(d[1] + 0.425) < 1e-5
        # the orbit center projects to the principal point, in front of the camera
        xc = R @ c + t
        assert xc[2] > 0
        assert abs(cam.fx * xc[0] / xc[2] + cam.cx - w / 2) < 1e-3
        assert abs(cam.fy * xc[1] / xc[2] + cam.cy - h / 2) < 1e-3
        assert abs(cam.fx - 900.0 * h / 832) < 1e-9 and cam.width == w and cam.height == h
