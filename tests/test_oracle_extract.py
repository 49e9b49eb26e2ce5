"""Pins of the oracle's viewpoint-independent pre-extraction (Sec. 3.2):
hand-derived radical inverses (tests/golden/halton_radical_inverse.json),
the van der Corput stratification of the first b^m indices, the level
weights of Eq. 4 without visibility and depth, per-leaf counts equal to the
sampler's (the same draws), and Halton positions inside their leaves with
the closed-form first point of every leaf.  CPU only."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2403_16862_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_radical_inverse_golden(oracle):
    g = json.load(open(os.path.join(GOLDEN, "halton_radical_inverse.json")))
    for b, i, num, den in g["cases"]:
        assert oracle.radical_inverse(b, i) == num / den


@pytest.mark.parametrize("b,m", [(2, 10), (3, 6), (5, 4)])
def test_van_der_corput_stratification(oracle, b, m):
    """The first b^m radical inverses (index 0 included) are exactly the
    points j / b^m, each once."""
    vals = sorted(Fraction(oracle.radical_inverse(b, i)).limit_denominator(b ** m) for i in range(b ** m))
    assert vals == [Fraction(j, b ** m) for j in range(b ** m)]


def test_level_weights(oracle):
    lv = np.array([2, 3, 4, 4])
    p = np.array([1.0, 1.0, 1.0, 0.5])
    w = oracle.level_weights(lv, p, 0.5)
    assert w[0] / w[1] == pytest.approx(2 ** 0.5, rel=1e-15) and w[2] / w[3] == 2.0
    assert np.array_equal(oracle.level_weights(lv, p, 0.0), p)


def test_halton_extraction(oracle):
    tree = scenes.make_octree(3, 4096 + 7 * 500)
    w = oracle.level_weights(tree.levels, tree.weights, 0.5)
    n = 300_000
    leaf, pos = oracle.sample_halton(tree, w, 9, n)
    view_tree = scenes.Octree(centers=tree.centers, levels=tree.levels, weights=w, root_size=tree.root_size)
    leaf_s, _, counts = oracle.sample_octree(view_tree, 9, 0, n)
    assert np.array_equal(leaf, leaf_s)  # the same draws and leaf-grouped order
    edge = tree.root_size * 2.0 ** -tree.levels[leaf]
    assert np.all(np.abs(pos - tree.centers[leaf]) <= edge[:, None] / 2)
    # the first sample of every leaf with samples is Halton point 1: (1/2, 1/3, 1/5)
    start = np.concatenate([[0], np.cumsum(counts)])[:-1]
    has = counts > 0
    first = pos[start[has]]
    e = tree.root_size * 2.0 ** -tree.levels[has]
    expect = tree.centers[has].astype(np.float64) + np.array([0.0, 1 / 3 - 0.5, 0.2 - 0.5])[None, :] * e[:, None]
    np.testing.assert_allclose(first, expect, rtol=0, atol=1e-7)
