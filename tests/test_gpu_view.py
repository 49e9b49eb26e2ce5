"""GPU view-specific re-weighting (Eq. 4) and visibility re-sampling (App.
A.4) against the oracle: the weights bit-exact (FP64 with the same
operation order; the level factors from the same exp2), the re-sampled leaf
indices and positions bit-exact, and the count of samples left out of view
exact."""
import numpy as np
import pytest
import torch

from paper_2403_16862_gb300 import api, scenes
from tests.test_oracle_view import _straddling_scene

pytestmark = pytest.mark.gpu


def _gpu_tree(gpu, tree):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(gpu) for a in (tree.centers, tree.levels, tree.weights)]


def test_view_weights_bit_exact(gpu, oracle):
    tree, cam = _straddling_scene()
    c, l, p = _gpu_tree(gpu, tree)
    for lam in (0.5, 0.0, 1.25):
        w = api.view_weights(c, l, p, tree.root_size, cam, lambda_l=lam).cpu().numpy()
        ref = oracle.view_weights(tree, cam, lambda_l=lam)
        assert np.array_equal(w, ref)
    # the benchmark scene from an orbit camera (partly outside the cube)
    big = scenes.make_octree(0, 65536)
    cam2 = scenes.orbit_cameras([(640, 480)], radius=1.1)[0]
    c, l, p = _gpu_tree(gpu, big)
    w = api.view_weights(c, l, p, big.root_size, cam2).cpu().numpy()
    ref = oracle.view_weights(big, cam2)
    assert np.array_equal(w, ref) and (ref == 0).sum() > 0 and (ref > 0).sum() > 0


@pytest.mark.parametrize("rounds", [0, 1, 8, 32])
def test_view_sampling_bit_exact(gpu, oracle, rounds):
    tree, cam = _straddling_scene()
    w = oracle.view_weights(tree, cam)
    c, l, _ = _gpu_tree(gpu, tree)
    n = 200_000
    leaf, pos, left = api.sample_octree_view(c, l, torch.from_numpy(w).to(gpu), tree.root_size, cam, 11, 3, n,
                                             max_rounds=rounds)
    o_leaf, o_pos, o_left = oracle.sample_view(tree, w, cam, 11, 3, n, max_rounds=rounds)
    assert np.array_equal(leaf.cpu().numpy(), o_leaf)
    assert np.array_equal(pos.cpu().numpy(), o_pos)
    assert int(left.item()) == o_left
    if rounds >= 32:
        assert o_left == 0
