"""Pins of the oracle's bilinear point rasterizer (Sec. 3.4 Eq. 5-6, Eq. 1
blending, App. A.6 early stop, Algorithm 1) and of its backward: a
hand-derived single-point splat, partition of unity of the bilinear weights,
monotone transmittance, the c == 1 identity, a pure-Python brute force on
tiny scenes, early termination, culling and FP64 central differences for
every gradient.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from paper_2403_16862_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cam(fx=1.0, fy=1.0, cx=10.0, cy=20.0, W=32, H=32, t=(0.0, 0.0, 0.0)):
    return scenes.Camera(R=np.eye(3, dtype=np.float32), t=np.asarray(t, np.float32), fx=fx, fy=fy, cx=cx, cy=cy,
                         width=W, height=H)


def test_projection_closed_form(oracle):
    cam = scenes.make_camera((0.0, 0.0, -3.0), 256.0, 256.0, 128.0, 128.0, 256, 256)
    pts = np.array([[0.0, 0.0, 0.0], [0.5, -0.25, 1.0], [-1.0, 1.0, -1.0]], np.float32)
    uvd, ok = oracle.project(cam, pts)
    assert ok.all()
    for p, (u, v, d) in zip(pts.astype(np.float64), uvd.astype(np.float64)):
        zc = p[2] + 3.0
        assert d == zc
        assert abs(u - (256.0 * p[0] / zc + 128.0)) <= 2 * np.spacing(np.float32(u))
        assert abs(v - (256.0 * p[1] / zc + 128.0)) <= 2 * np.spacing(np.float32(v))
    # near / far culling (App. A.2 planes 0.01 and 100)
    _, ok = oracle.project(cam, np.array([[0, 0, -2.995], [0, 0, 97.5], [0, 0, -2.98]], np.float32))
    assert ok.tolist() == [False, False, True]


def test_single_point_golden(oracle):
    g = json.load(open(os.path.join(GOLDEN, "single_point_splat.json")))
    c = g["camera"]
    cam = _cam(c["fx"], c["fy"], c["cx"], c["cy"], c["width"], c["height"])
    pos = np.array([g["point"]], np.float32)
    feat = np.array([g["feature"]])
    a = g["alpha_h"]
    out = oracle.raster_fwd(cam, pos, feat, opacity=np.array([a]))
    touched = np.argwhere(out["n_contrib"] > 0)
    assert sorted(map(tuple, touched.tolist())) == sorted((p["y"], p["x"]) for p in g["pixels"])
    for p in g["pixels"]:
        al = a * p["w"]
        np.testing.assert_allclose(out["image"][p["y"], p["x"]], al * np.array(g["feature"]), rtol=1e-15)
        assert out["T_final"][p["y"], p["x"]] == pytest.approx(1 - al, rel=1e-15)
    assert sum(p["w"] for p in g["pixels"]) == 1.0


def test_bilinear_weights_partition_of_unity(oracle):
    rng = np.random.default_rng(0)
    for _ in range(1000):
        u, v = rng.uniform(1, 100, size=2)
        pi, pj, w = oracle.splat_corners(u, v)
        assert abs(w.sum() - 1.0) < 1e-14 and np.all(w >= 0)
        # the 2x2 nearest pixel centers: every center within one pixel of (u, v)
        assert np.all(np.abs(pi + 0.5 - u) <= 1.0) and np.all(np.abs(pj + 0.5 - v) <= 1.0)


def _brute_force(cam, pos, opacity, feat, t_min, alpha_max, oracle):
    """Per-pixel list building, sorting and blending in plain Python."""
    uvd, ok = oracle.project(cam, pos)
    W, H = cam.width, cam.height
    lists = {}
    for p in range(len(pos)):
        if not ok[p]:
            continue
        u, v, d = map(float, uvd[p])
        if not (-0.5 <= u < W + 0.5 and -0.5 <= v < H + 0.5):
            continue
        for b in (0, 1):
            for a in (0, 1):
                i = math.floor(u - 0.5) + a
                j = math.floor(v - 0.5) + b
                if 0 <= i < W and 0 <= j < H:
                    w = (1 - abs(u - (i + 0.5))) * (1 - abs(v - (j + 0.5)))
                    lists.setdefault((j, i), []).append((float(np.float32(d)), p, w))
    F = feat.shape[1]
    img = np.zeros((H, W, F)); T = np.ones((H, W)); n = np.zeros((H, W), np.int64)
    for (j, i), L in lists.items():
        L.sort(key=lambda r: (r[0], r[1]))
        t = 1.0
        prev = 1.0
        for d, p, w in L:
            al = min(opacity[p] * w, alpha_max)
            img[j, i] += t * al * feat[p]
            t = t * (1 - al)
            assert t <= prev
            prev = t
            n[j, i] += 1
            if t < t_min:
                break
        T[j, i] = t
    return img, T, n


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_tiny(oracle, seed):
    rng = np.random.default_rng(seed)
    n = 64
    cam = scenes.make_camera((0.0, 0.0, -3.0), 3.0, 3.0, 4.0, 4.0, 8, 8)
    pos = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    pos[:8] = pos[8:16]  # exact duplicates: equal depths, tie broken by point id
    opacity = rng.uniform(0.05, 0.95, size=n)
    feat = rng.normal(size=(n, 3))
    out = oracle.raster_fwd(cam, pos, feat, opacity=opacity)
    img, T, nc = _brute_force(cam, pos, opacity, feat, 1e-4, 0.99, oracle)
    np.testing.assert_allclose(out["image"], img, atol=1e-13)
    np.testing.assert_allclose(out["T_final"], T, atol=1e-15)
    assert np.array_equal(out["n_contrib"], nc)


def test_unit_color_identity_and_monotone(oracle):
    pts, cam = scenes.raster_points_scene(seed=3, n=4000, n_feat=2, size=32, focal=32.0)
    feat = np.ones((4000, 2))
    out = oracle.raster_fwd(cam, pts.pos, feat, opacity=pts.opacity)
    np.testing.assert_allclose(out["image"][..., 0], 1 - out["T_final"], atol=1e-12)
    assert np.all(out["T_final"] <= 1) and np.all(out["T_final"] >= 0)
    # head mode: channel 0 of the blended color is 1, so image[...,0] = 1 - T
    h = np.random.default_rng(4).normal(size=(4000, 4))
    out = oracle.raster_fwd(cam, pts.pos, h, head_mode=True)
    np.testing.assert_allclose(out["image"][..., 0], 1 - out["T_final"], atol=1e-12)


def test_early_termination(oracle):
    # 20 points stacked on one pixel center, alpha 0.5 each: T = 0.5^k drops
    # below 1e-4 at k = 14 (0.5^13 = 1.22e-4, 0.5^14 = 6.1e-5)
    cam = _cam(cx=0.0, cy=0.0, W=4, H=4)
    pos = np.array([[2.5, 1.5, 1.0]] * 20, np.float32)
    out = oracle.raster_fwd(cam, pos, np.ones((20, 1)), opacity=np.full(20, 0.5))
    assert out["n_contrib"][1, 2] == 14
    assert out["T_final"][1, 2] == 0.5 ** 14
    assert out["n_frags"][1, 2] == 20
    # the zero-weight neighbours are emitted (alpha 0) and blended in full
    assert out["n_frags"][1, 3] == 20 and out["n_contrib"][1, 3] == 20 and out["T_final"][1, 3] == 1.0


def test_alpha_clamp(oracle):
    cam = _cam(cx=0.0, cy=0.0, W=4, H=4)
    pos = np.array([[1.5, 1.5, 1.0]], np.float32)
    out = oracle.raster_fwd(cam, pos, np.ones((1, 1)), opacity=np.array([1.0]), alpha_max=0.99)
    assert out["T_final"][1, 1] == pytest.approx(0.01, rel=1e-14)


def test_fragments_sorted_by_depth_then_id(oracle):
    pts, cam = scenes.raster_points_scene(seed=5, n=3000, size=24, focal=24.0)
    cnt, ids, cor, dep = oracle.fragment_lists(cam, pts.pos)
    start = 0
    for c in cnt.ravel():
        seg_d = dep[start:start + c]; seg_i = ids[start:start + c]
        key = list(zip(seg_d.tolist(), seg_i.tolist()))
        assert key == sorted(key)
        start += c
    assert start == len(ids)


def _fd_check(oracle, cam, pos, feat, opacity, head, g, eps=1e-6, samples=25, seed=0):
    base = oracle.raster_fwd(cam, pos, feat, opacity=opacity, head_mode=head)
    bwd = oracle.raster_bwd(cam, pos, feat, g, opacity=opacity, head_mode=head)
    rng = np.random.default_rng(seed)

    def loss(f, o):
        out = oracle.raster_fwd(cam, pos, f, opacity=o, head_mode=head)
        assert np.array_equal(out["n_contrib"], base["n_contrib"]), "perturbation crossed the stop threshold"
        return np.sum(out["image"] * g)

    n, F = feat.shape
    for _ in range(samples):
        p = int(rng.integers(0, n)); c = int(rng.integers(0, F))
        fp = feat.copy(); fp[p, c] += eps
        fm = feat.copy(); fm[p, c] -= eps
        fd = (loss(fp, opacity) - loss(fm, opacity)) / (2 * eps)
        assert abs(fd - bwd["d_feat"][p, c]) <= 1e-6 * (1 + abs(fd)), (p, c, fd, bwd["d_feat"][p, c])
    if not head:
        for _ in range(samples):
            p = int(rng.integers(0, n))
            op = opacity.copy(); op[p] += eps
            om = opacity.copy(); om[p] -= eps
            fd = (loss(feat, op) - loss(feat, om)) / (2 * eps)
            assert abs(fd - bwd["d_opacity"][p]) <= 1e-6 * (1 + abs(fd)), (p, fd, bwd["d_opacity"][p])


def test_backward_finite_differences_given_opacity(oracle):
    pts, cam = scenes.raster_points_scene(seed=6, n=400, n_feat=3, size=12, focal=12.0)
    g = np.random.default_rng(7).normal(size=(12, 12, 3))
    _fd_check(oracle, cam, pts.pos, pts.feat.astype(np.float64), pts.opacity.astype(np.float64), False, g)


def test_backward_finite_differences_head_mode(oracle):
    pts, cam = scenes.raster_points_scene(seed=8, n=400, n_feat=5, size=12, focal=12.0)
    h = np.random.default_rng(9).normal(0, 0.5, size=(400, 5))
    g = np.random.default_rng(10).normal(size=(12, 12, 5))
    _fd_check(oracle, cam, pts.pos, h, None, True, g)


def test_backward_gradients_vanish_for_culled_points(oracle):
    pts, cam = scenes.raster_points_scene(seed=11, n=200, n_feat=2, size=8, focal=8.0)
    pos = pts.pos.copy()
    pos[:50, 2] = -10.0  # behind the camera
    g = np.random.default_rng(12).normal(size=(8, 8, 2))
    out = oracle.raster_bwd(cam, pos, pts.feat, g, opacity=pts.opacity)
    assert np.all(out["d_feat"][:50] == 0) and np.all(out["d_opacity"][:50] == 0)


def test_pipeline_table_gradient_finite_differences(oracle):
    # end to end: table -> query -> head-mode rasterizer -> <g, image>
    res = [4, 9]
    log2_T = 8
    total, _ = oracle.hash_layout(res, log2_T)
    rng = np.random.default_rng(13)
    tab = rng.normal(0, 0.3, size=(total, 4))
    pos = rng.uniform(0, 1, size=(300, 3)).astype(np.float32)
    cam = scenes.make_camera((0.5, 0.5, -1.2), 14.0, 14.0, 8.0, 8.0, 16, 16)
    g = rng.normal(size=(16, 16, 8))

    def loss(t):
        h = oracle.hash_fwd(res, log2_T, t, pos)
        return np.sum(oracle.raster_fwd(cam, pos, h, head_mode=True)["image"] * g)

    h = oracle.hash_fwd(res, log2_T, tab, pos)
    dh = oracle.raster_bwd(cam, pos, h, g, head_mode=True)["d_feat"]
    dtab = oracle.hash_bwd(res, log2_T, 4, pos, dh)
    for _ in range(15):
        r = int(rng.integers(0, total)); f = int(rng.integers(0, 4))
        e = 1e-6
        tp = tab.copy(); tp[r, f] += e
        tm = tab.copy(); tm[r, f] -= e
        fd = (loss(tp) - loss(tm)) / (2 * e)
        assert abs(fd - dtab[r, f]) <= 1e-6 * (1 + abs(fd)), (r, f, fd, dtab[r, f])


def test_differentiation_subcase_finite_differences(oracle):
    """FP64 central differences on the differentiation workload's small case:
    the first 4,096 samples of the 65,536-leaf octree scene (seed 0, view
    0), the 16-level 2^19 grid, a 64x64 view from the benchmark camera with
    the focal length scaled to 45 (the full view's 900 / 20), upstream
    gradient ~ N(0, 1).  Checked: d h (the opacity path through h0 and the
    color channels, head mode), d alpha and d F in given-opacity mode
    (alpha = the head's alpha of the same points, F = the color channels),
    and d table through the whole pipeline.  Perturbations that change a
    pixel's blended count (the early stop) are rejected and not counted."""
    res = scenes.geometric_resolutions(16, 16, 4096)
    tree = scenes.make_octree(0, 65536)
    grid = scenes.make_hashgrid(1, oracle.hash_entries(res, 19), res, 19)
    _, pos64, _ = oracle.sample_octree(tree, 0, 0, 4096)
    pos = pos64.astype(np.float32)
    cam = scenes.make_camera((0.5, 0.5, -1.2), 45.0, 45.0, 32.0, 32.0, 64, 64)
    g = scenes.upstream_grad(2, (64, 64, 64)).astype(np.float64)
    tab = grid.table.astype(np.float64)
    h = oracle.hash_fwd(res, 19, tab, pos)
    base = oracle.raster_fwd(cam, pos, h, head_mode=True)
    assert base["n_contrib"].max() > 8 and (base["n_contrib"] > 0).mean() > 0.2, "a blended scene"
    rng = np.random.default_rng(20)
    eps = 1e-6

    def central(loss, perturb, n_want, draw):
        done = tried = 0
        while done < n_want:
            tried += 1
            assert tried < 4 * n_want, "too many perturbations crossed the stop threshold"
            k = draw()
            lp, lm = loss(perturb(k, eps)), loss(perturb(k, -eps))
            if lp is None or lm is None:
                continue
            yield k, (lp - lm) / (2 * eps)
            done += 1

    # head mode: d h (channel 0 carries the opacity path)
    bh = oracle.raster_bwd(cam, pos, h, g, head_mode=True)["d_feat"]

    def loss_h(hh):
        out = oracle.raster_fwd(cam, pos, hh, head_mode=True)
        return None if not np.array_equal(out["n_contrib"], base["n_contrib"]) else float(np.sum(out["image"] * g))

    def pert_h(k, e):
        hh = h.copy()
        hh[k] += e
        return hh

    vis = np.flatnonzero(np.abs(bh).sum(axis=1) > 0)
    draws = iter([(int(rng.choice(vis)), 0) for _ in range(40)] + [(int(rng.choice(vis)), int(rng.integers(1, 64)))
                                                                   for _ in range(40)])
    for k, fd in central(lambda x: loss_h(x), pert_h, 30, lambda: next(draws)):
        assert abs(fd - bh[k]) <= 1e-6 * (1 + abs(fd)), ("dh", k, fd, bh[k])

    # given-opacity mode on the same points: d alpha and d F
    alpha = 1.0 - np.exp(-np.exp(h[:, 0]))
    F = h[:, 1:].copy()
    base_g = oracle.raster_fwd(cam, pos, F, opacity=alpha)
    bg = oracle.raster_bwd(cam, pos, F, g[..., 1:], opacity=alpha)

    def loss_g(f, o):
        out = oracle.raster_fwd(cam, pos, f, opacity=o)
        return None if not np.array_equal(out["n_contrib"], base_g["n_contrib"]) else \
            float(np.sum(out["image"] * g[..., 1:]))

    def pert_a(k, e):
        o = alpha.copy()
        o[k] += e
        return o

    def pert_f(k, e):
        f = F.copy()
        f[k] += e
        return f

    da = iter([int(rng.choice(vis)) for _ in range(40)])
    for k, fd in central(lambda o: loss_g(F, o), pert_a, 20, lambda: next(da)):
        assert abs(fd - bg["d_opacity"][k]) <= 1e-6 * (1 + abs(fd)), ("d alpha", k, fd, bg["d_opacity"][k])
    df = iter([(int(rng.choice(vis)), int(rng.integers(0, 63))) for _ in range(40)])
    for k, fd in central(lambda f: loss_g(f, alpha), pert_f, 20, lambda: next(df)):
        assert abs(fd - bg["d_feat"][k]) <= 1e-6 * (1 + abs(fd)), ("dF", k, fd, bg["d_feat"][k])

    # d table through query -> rasterizer, on rows the points reach
    dtab = oracle.hash_bwd(res, 19, 4, pos, bh)
    rows = np.flatnonzero(np.abs(dtab).sum(axis=1) > 0)

    def loss_t(k, e):
        r, f = k
        old = tab[r, f]
        tab[r, f] = old + e
        try:
            return loss_h(oracle.hash_fwd(res, 19, tab, pos))
        finally:
            tab[r, f] = old

    dt = iter([(int(rng.choice(rows)), int(rng.integers(0, 4))) for _ in range(40)])
    done = 0
    for _ in range(40):
        k = next(dt)
        lp, lm = loss_t(k, eps), loss_t(k, -eps)
        if lp is None or lm is None:
            continue
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - dtab[k]) <= 1e-6 * (1 + abs(fd)), ("d table", k, fd, dtab[k])
        done += 1
        if done == 20:
            break
    assert done == 20


def test_projection_against_the_fp64_definition(oracle):
    """The oracle's FP32 projection (Eq. 5 in the kernel's operation order)
    against Eq. 5 evaluated in FP64: within the rounding bound of the FP32
    steps, and the same top-left pixel (floor(u - 1/2), floor(v - 1/2))
    wherever the FP64 value is farther than that bound from a pixel border.
    A wrong operand, sign or order in the FP32 steps fails it."""
    rng = np.random.default_rng(21)
    eps = 2.0 ** -24
    cams = [scenes.make_camera((0.5, 0.5, -1.2), 900.0, 900.0, 640.0, 416.0, 1280, 832)]
    cams += scenes.orbit_cameras([(1920, 1080), (640, 480)])
    pts = rng.uniform(0.0, 1.0, size=(20000, 3)).astype(np.float32)
    ambiguous = 0
    for cam in cams:
        uvd, ok = oracle.project(cam, pts)
        R = np.asarray(cam.R, np.float64)
        t = np.asarray(cam.t, np.float64)
        x = pts.astype(np.float64)
        xc = x @ R.T + t
        mag = np.abs(x) @ np.abs(R).T + np.abs(t)  # size of the camera coordinates' terms
        z = xc[:, 2]
        assert np.array_equal(ok, (z > cam.near) & (z < cam.far))
        for k, (f, c) in enumerate(((cam.fx, cam.cx), (cam.fy, cam.cy))):
            q = xc[:, k] / z
            u64 = f * q + c
            # rounding of the FP32 steps: three roundings in each camera
            # coordinate, one in the division, one in the final fma
            dq = (3 * eps * mag[:, k] + np.abs(q) * 3 * eps * mag[:, 2]) / z + eps * np.abs(q)
            bound = 2.0 * (f * dq + eps * np.abs(u64) + eps * abs(c))
            u32 = uvd[:, k].astype(np.float64)
            assert np.all(np.abs(u32 - u64)[ok] <= bound[ok])
            # the pixel decision (Sec. 3.4: the 2x2 nearest pixel centers)
            far_from_border = np.abs((u64 - 0.5) - np.rint(u64 - 0.5)) > bound
            same = np.floor(u32 - 0.5) == np.floor(u64 - 0.5)
            assert np.all(same[ok & far_from_border])
            ambiguous += int((ok & ~far_from_border).sum())
        assert np.array_equal(uvd[ok, 2].astype(np.float64), z[ok].astype(np.float32).astype(np.float64)) or \
            np.all(np.abs(uvd[ok, 2] - z[ok]) <= 3 * eps * mag[ok, 2])
    assert ambiguous < 1e-3 * 3 * 2 * len(pts)
