"""Pins of the oracle's view-dependent head (Sec. 3.3): the degree-2 real
SH basis (orthonormal on the sphere by Gauss-Legendre x uniform quadrature,
the per-band addition theorem sum_m Y_lm^2 = (2l+1)/(4 pi), the documented
ordering at the axis directions), the head forward in closed form (a
direction-independent degree-0 color, alpha_h(0) = 1 - 1/e), the head
backward against FP64 central differences, and the spherical contraction
(identity inside the unit ball, continuity at its surface, radial
monotonicity, the image inside [0, 1]^3).  CPU only."""
import math

import numpy as np
import pytest

from paper_2403_16862_gb300 import scenes


def _sphere_quadrature(n_theta=24, n_phi=48):
    x, wx = np.polynomial.legendre.leggauss(n_theta)  # cos(theta)
    phi = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wx[:, None] * np.full(n_phi, 2 * math.pi / n_phi)[None, :]).ravel()
    return d, w


def test_sh_orthonormal(oracle):
    d, w = _sphere_quadrature()
    Y = np.stack([oracle.sh_basis(v) for v in d])
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(9), atol=1e-12)


def test_sh_addition_theorem_and_order(oracle):
    rng = np.random.default_rng(0)
    for _ in range(100):
        v = rng.normal(size=3)
        Y = oracle.sh_basis(v / np.linalg.norm(v))
        assert Y[0] ** 2 == pytest.approx(1 / (4 * math.pi), rel=1e-14)
        assert np.sum(Y[1:4] ** 2) == pytest.approx(3 / (4 * math.pi), rel=1e-13)
        assert np.sum(Y[4:9] ** 2) == pytest.approx(5 / (4 * math.pi), rel=1e-13)
    c1 = math.sqrt(3 / (4 * math.pi))
    for axis, k in ((1, 1), (2, 2), (0, 3)):  # Y_1..3 follow (y, z, x)
        d = np.zeros(3)
        d[axis] = 1.0
        Y = oracle.sh_basis(d)
        assert Y[k] == pytest.approx(c1, rel=1e-15)
        assert np.all(Y[[i for i in (1, 2, 3) if i != k]] == 0.0)


def _cam():
    return scenes.make_camera((0.3, -0.2, -2.0), 100.0, 100.0, 50.0, 40.0, 100, 80)


def test_head_forward_closed_forms(oracle):
    rng = np.random.default_rng(1)
    n, F = 200, 64
    pos = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    h = np.zeros((n, F))
    dc = rng.normal(size=4)
    for c in range(4):
        h[:, 1 + 9 * c] = dc[c]  # degree-0 coefficients only
    a, col = oracle.sh_head_fwd(_cam(), pos, h)
    np.testing.assert_allclose(col, np.broadcast_to(dc / (2 * math.sqrt(math.pi)), (n, 4)), rtol=1e-15)
    assert np.allclose(a, 1 - math.exp(-1), rtol=1e-15)


def test_head_backward_central_differences(oracle):
    rng = np.random.default_rng(2)
    n, F = 12, 40
    pos = rng.uniform(-1, 1, (n, 3)).astype(np.float32)
    h = rng.normal(0, 0.5, (n, F))
    da = rng.normal(size=n)
    dcol = rng.normal(size=(n, 4))
    dh = oracle.sh_head_bwd(_cam(), pos, h, da, dcol)
    eps = 1e-6
    for p in range(n):
        for f in range(F):
            hp, hm = h.copy(), h.copy()
            hp[p, f] += eps
            hm[p, f] -= eps
            ap, cp = oracle.sh_head_fwd(_cam(), pos, hp)
            am, cm = oracle.sh_head_fwd(_cam(), pos, hm)
            fd = (np.dot(ap - am, da) + np.sum((cp - cm) * dcol)) / (2 * eps)
            assert dh[p, f] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    assert np.all(dh[:, 37:] == 0.0)


def test_contraction(oracle):
    rng = np.random.default_rng(3)
    center, radius = np.array([0.5, 0.25, -1.0], np.float32), np.float32(2.0)
    # inside the unit ball: the identity (scaled into [1/4, 3/4])
    u = rng.normal(size=(2000, 3))
    u = u / np.linalg.norm(u, axis=1, keepdims=True) * rng.uniform(0, 0.999, (2000, 1))
    pin = (center + u * radius).astype(np.float32)
    q = oracle.contract(pin, center, radius).astype(np.float64)
    y = (pin.astype(np.float64) - center) / radius
    np.testing.assert_allclose(q, y / 4 + 0.5, atol=2e-7)
    # outside: |contract| = 2 - 1/|y| < 2, monotone in |y|, continuous at 1
    dirn = rng.normal(size=3)
    dirn /= np.linalg.norm(dirn)
    r = np.concatenate([np.linspace(0.5, 1.5, 201), np.geomspace(1.5, 1e6, 200)])
    pts = (center + np.outer(r, dirn) * radius).astype(np.float32)
    qq = (oracle.contract(pts, center, radius).astype(np.float64) - 0.5) * 4
    norm = np.linalg.norm(qq, axis=1)
    assert np.all(np.diff(norm) >= -1e-6) and norm.max() < 2.0 + 1e-6
    far = r > 2
    np.testing.assert_allclose(norm[far], 2 - 1 / r[far], atol=1e-5)
    assert np.all((qq / 4 + 0.5 >= 0) & (qq / 4 + 0.5 <= 1))


def test_contraction_against_the_fp64_definition(oracle):
    # the FP32 contraction (kernel operation order) against the plain FP64
    # definition: y = (x - c)/r, y for |y| <= 1, else (2 - 1/|y|) y/|y|,
    # query position contract(y)/4 + 1/2; within a few FP32 roundings, and
    # the same grid cell at the finest resolution wherever the FP64 value is
    # not within that distance of a cell border
    rng = np.random.default_rng(22)
    center = np.array([0.1, -0.2, 0.3], np.float32)
    radius = np.float32(0.75)
    pts = np.concatenate([rng.normal(0, 1, size=(20000, 3)), rng.normal(0, 30, size=(20000, 3))]).astype(np.float32)
    got = oracle.contract(pts, center, radius).astype(np.float64)
    y = (pts.astype(np.float64) - center.astype(np.float64)) / float(radius)
    n = np.linalg.norm(y, axis=1, keepdims=True)
    want = np.where(n <= 1.0, y, (2.0 - 1.0 / n) * y / n) / 4.0 + 0.5
    tol = 16 * 2.0 ** -24
    assert np.all(np.abs(got - want) <= tol)
    N = 4096
    far = np.abs(want * N - np.rint(want * N)) > tol * N
    assert np.all((np.floor(got * N) == np.floor(want * N))[far])
    assert np.all((got >= 0.0) & (got <= 1.0))
