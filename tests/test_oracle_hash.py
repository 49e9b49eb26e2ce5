"""Pins of the oracle's multi-resolution grid query (Sec. 3.3, App. A.5)
against closed forms: partition of unity, exact reproduction of linear
functions, a hand-derived unit cell, the adjoint identity between the query
and its gradient, and the table layout.  CPU only."""
import json
import os

import numpy as np

from paper_2403_16862_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RES16 = scenes.geometric_resolutions(16, 16, 4096)


def _up16(x):
    return (x + 15) // 16 * 16


def test_resolutions_and_layout(oracle):
    assert RES16 == [16, 23, 33, 48, 70, 101, 147, 212, 307, 445, 645, 933, 1351, 1955, 2830, 4096]
    total, offs = oracle.hash_layout(RES16, 19)
    dense = [(r + 1) ** 3 for r in RES16[:5]]
    assert dense == [4913, 13824, 39304, 117649, 357911]
    assert all(d <= 2 ** 19 for d in dense) and (RES16[5] + 1) ** 3 > 2 ** 19
    # every level starts on a multiple of 16 rows
    want, off = [], 0
    for e in dense + [2 ** 19] * 11:
        off = _up16(off)
        want.append(off)
        off += e
    assert list(offs) == want and total == _up16(off)
    assert offs[1] == 4928 and offs[5] == 533648 and total == 533648 + 11 * 2 ** 19 == 6300816
    total21, _ = oracle.hash_layout(RES16, 21)
    off = 0
    for e in [(r + 1) ** 3 for r in RES16[:6]] + [2 ** 21] * 10:
        off = _up16(off) + e
    assert total21 == _up16(off)


def test_dense_index_is_bijective(oracle):
    res = 5
    seen = set()
    for z in range(res + 1):
        for y in range(res + 1):
            for x in range(res + 1):
                seen.add(oracle.hash_vertex_index(res, 10, x, y, z))
    assert seen == set(range((res + 1) ** 3))


def test_hashed_index_range(oracle):
    rng = np.random.default_rng(0)
    for _ in range(500):
        v = rng.integers(0, 4097, size=3)
        i = oracle.hash_vertex_index(4096, 19, *map(int, v))
        assert 0 <= i < 2 ** 19
    # x-neighbours at even x differ only in the lowest index bit
    assert oracle.hash_vertex_index(4096, 19, 10, 7, 3) ^ oracle.hash_vertex_index(4096, 19, 11, 7, 3) == 1


def test_unit_cell_golden(oracle):
    g = json.load(open(os.path.join(GOLDEN, "trilinear_unit_cell.json")))
    tab = np.zeros((8, 2))
    for bz in (0, 1):
        for by in (0, 1):
            for bx in (0, 1):
                row = oracle.hash_vertex_index(1, g["log2_T"], bx, by, bz)
                tab[row] = (1 + 2 * bx + 4 * by + 8 * bz, bx * by * bz)
    h = oracle.hash_fwd([g["res"]], g["log2_T"], tab, np.array([g["point"]]))
    np.testing.assert_allclose(h[0], g["h"], rtol=0, atol=1e-15)


def test_constant_table_partition_of_unity(oracle):
    res = RES16[:6]
    total, _ = oracle.hash_layout(res, 12)
    tab = np.tile(np.array([[0.5, -2.0, 3.0, 7.25]]), (total, 1))
    pos = np.random.default_rng(1).uniform(-0.1, 1.1, size=(2000, 3))
    h = oracle.hash_fwd(res, 12, tab, pos)
    np.testing.assert_allclose(h, np.tile([0.5, -2.0, 3.0, 7.25], len(res))[None, :].repeat(2000, 0), atol=1e-13)


def test_linear_function_reproduced_exactly(oracle):
    # trilinear interpolation reproduces a function linear in the vertex
    # coordinates, so on dense levels h(x) is that linear function of x
    res = [4, 7, 13]
    log2_T = 12
    total, offs = oracle.hash_layout(res, log2_T)
    coef = np.array([[0.3, 1.5, -2.0, 0.75], [-1.0, 0.25, 0.5, 2.0]])  # a, b, c, d per feature
    tab = np.zeros((total, 2))
    for l, r in enumerate(res):
        for z in range(r + 1):
            for y in range(r + 1):
                for x in range(r + 1):
                    row = offs[l] + oracle.hash_vertex_index(r, log2_T, x, y, z)
                    tab[row] = coef[:, 0] + coef[:, 1] * x / r + coef[:, 2] * y / r + coef[:, 3] * z / r
    pos = np.random.default_rng(2).uniform(0, 1, size=(3000, 3))
    pos[:10] = [[1, 1, 1], [0, 0, 0], [1, 0, 0.5], [0.25, 1, 0], [0.5, 0.5, 0.5],
                [0.75, 0.75, 1], [1, 1, 0], [0, 1, 1], [0.125, 0.625, 0.375], [0.999999, 0.000001, 0.5]]
    h = oracle.hash_fwd(res, log2_T, tab, pos)
    want = coef[:, 0][None] + pos[:, 0:1] * coef[:, 1][None] + pos[:, 1:2] * coef[:, 2][None] + pos[:, 2:3] * coef[:, 3][None]
    for l in range(len(res)):
        np.testing.assert_allclose(h[:, 2 * l:2 * l + 2], want, atol=1e-12)


def test_continuity_across_cell_faces(oracle):
    res = RES16[:8]
    total, _ = oracle.hash_layout(res, 14)
    tab = np.random.default_rng(3).normal(size=(total, 4))
    rng = np.random.default_rng(4)
    for l, r in enumerate(res):
        k = rng.integers(1, r, size=50)
        p = rng.uniform(0, 1, size=(50, 3))
        lo = p.copy(); hi = p.copy()
        lo[:, 0] = k / r - 1e-9
        hi[:, 0] = k / r + 1e-9
        d = oracle.hash_fwd(res, 14, tab, lo) - oracle.hash_fwd(res, 14, tab, hi)
        # a discontinuity would be O(|table|); continuity leaves only the
        # slope (at most 2 r max|table| per unit x) times the 2e-9 gap
        assert np.max(np.abs(d[:, 4 * l:4 * l + 4])) <= 2e-9 * 2 * r * np.max(np.abs(tab)) * 1.01


def test_adjoint_identity_and_mass(oracle):
    # the query is linear in the table; its gradient must be the adjoint:
    # <query(table), dh> == <table, grad(dh)> for random table and dh
    res = RES16[:10]
    log2_T = 13
    total, offs = oracle.hash_layout(res, log2_T)
    rng = np.random.default_rng(5)
    tab = rng.normal(size=(total, 4))
    pos = rng.uniform(0, 1, size=(4000, 3))
    dh = rng.normal(size=(4000, 4 * len(res)))
    h = oracle.hash_fwd(res, log2_T, tab, pos)
    grad = oracle.hash_bwd(res, log2_T, 4, pos, dh)
    lhs = np.sum(h * dh)
    rhs = np.sum(tab * grad)
    assert abs(lhs - rhs) <= 1e-10 * (np.sum(np.abs(h * dh)) + 1)
    # trilinear weights sum to one: each level's gradient mass equals the dh mass
    for l in range(len(res)):
        end = offs[l + 1] if l + 1 < len(res) else total
        np.testing.assert_allclose(grad[offs[l]:end].sum(0), dh[:, 4 * l:4 * l + 4].sum(0), rtol=1e-10, atol=1e-9)


def test_finite_difference_table_gradient(oracle):
    res = RES16[:4]
    log2_T = 10
    total, _ = oracle.hash_layout(res, log2_T)
    rng = np.random.default_rng(6)
    tab = rng.normal(size=(total, 4))
    pos = rng.uniform(0, 1, size=(300, 3))
    dh = rng.normal(size=(300, 16))
    grad = oracle.hash_bwd(res, log2_T, 4, pos, dh)
    for _ in range(20):
        r = int(rng.integers(0, total)); f = int(rng.integers(0, 4))
        e = 1e-6
        tp = tab.copy(); tp[r, f] += e
        tm = tab.copy(); tm[r, f] -= e
        fd = (np.sum(oracle.hash_fwd(res, log2_T, tp, pos) * dh) - np.sum(oracle.hash_fwd(res, log2_T, tm, pos) * dh)) / (2 * e)
        assert abs(fd - grad[r, f]) < 1e-6 * (1 + abs(fd))


def test_hashed_index_golden(oracle):
    # hand-derived spatial-hash indices (uint32 products, XOR, mod T) on a
    # hashed level: a wrong prime or + in place of XOR fails one of them
    g = json.load(open(os.path.join(GOLDEN, "hash_index.json")))
    assert (g["res"] + 1) ** 3 > 2 ** g["log2_T"], "the level must be hashed"
    for case in g["cases"]:
        assert oracle.hash_vertex_index(g["res"], g["log2_T"], *case["v"]) == case["index"], case
