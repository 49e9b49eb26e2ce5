"""GPU sampling (inpc_sample_octree) against the oracle: leaf indices and
per-leaf counts bit-exact, positions bit-exact to the correctly rounded FP32
value of the oracle's exact FP64 position."""
import numpy as np
import pytest
import torch

from paper_2403_16862_gb300 import _binding as B
from paper_2403_16862_gb300 import api, scenes

pytestmark = pytest.mark.gpu


def _dev_tree(tree, dev):
    return (torch.from_numpy(tree.centers).to(dev), torch.from_numpy(tree.levels).to(dev),
            torch.from_numpy(tree.weights).to(dev))


def _check(tree, seed, view, n, dev, oracle):
    c, l, w = _dev_tree(tree, dev)
    leaf, pos, counts = api.sample_octree(c, l, w, tree.root_size, seed, view, n, with_counts=True)
    torch.cuda.synchronize()
    o_leaf, o_pos, o_counts = oracle.sample_octree(tree, seed, view, n)
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), o_counts), "per-leaf counts"
    assert np.array_equal(leaf.cpu().numpy(), o_leaf), "leaf indices"
    assert np.array_equal(pos.cpu().numpy(), o_pos.astype(np.float32)), "positions (single rounding of the exact value)"
    if n:
        assert np.max(np.abs(pos.cpu().numpy() - o_pos)) <= 1e-5 * tree.root_size


def test_small_trees(gpu, oracle):
    for seed, extra in [(0, 10), (1, 300), (2, 1000)]:
        t = scenes.make_octree(seed, 4096 + 7 * extra)
        _check(t, seed=7 + seed, view=seed, n=100_000 + 37 * seed, dev=gpu, oracle=oracle)


def test_count_paths(gpu, oracle):
    """Trees up to 4,096 leaves count their draws per CTA in shared memory,
    larger ones with warp-merged global additions: both sides of the
    threshold, and a 64-leaf tree whose counters take many draws each."""
    for n_leaves, start in ((64, 2), (4096, 4), (4096 + 7, 4)):
        t = scenes.make_octree(11, n_leaves, start_level=start)
        assert t.n_leaves == n_leaves
        _check(t, seed=13, view=2, n=300_001, dev=gpu, oracle=oracle)


def test_full_size_octree_4m_samples(gpu, oracle):
    """65,536-leaf octree, 4,194,304 samples: the sampling step of the
    full-size workload, in the launch configuration the benchmark times."""
    t = scenes.make_octree(0, 65536)
    _check(t, seed=0, view=0, n=4_194_304, dev=gpu, oracle=oracle)


def test_million_leaf_octree(gpu, oracle):
    t = scenes.make_octree(3, 1 << 20, start_level=6)
    _check(t, seed=3, view=5, n=1 << 21, dev=gpu, oracle=oracle)


def test_edge_cases(gpu, oracle):
    # one leaf; a tree with zero-weight leaves; non-power-of-two root size; tiny N
    one = scenes.Octree(centers=np.array([[0.3, 0.5, 0.7]], np.float32), levels=np.array([2], np.int32),
                        weights=np.array([0.25]), root_size=2.0)
    _check(one, 1, 0, 1000, gpu, oracle)
    t = scenes.make_octree(5, 4096 + 7 * 20)
    t.weights[::3] = 0.0
    _check(t, 2, 1, 50_000, gpu, oracle)
    t.root_size = 3.0  # positions scale; still exactly one rounding of the exact value
    _check(t, 4, 2, 20_000, gpu, oracle)
    for n in (0, 1, 2, 2049):
        _check(t, 5, 3, n, gpu, oracle)


def test_device_status_for_bad_weights(gpu):
    t = scenes.make_octree(6, 4096)
    c, l, w = _dev_tree(t, gpu)
    ws = api.workspace(B.inpc_sample_workspace_size(t.n_leaves, 1000), gpu)
    w_bad = w.clone()
    w_bad[17] = float("nan")
    api.sample_octree(c, l, w_bad, 1.0, 0, 0, 1000, ws=ws)
    assert api.read_device_status(ws) & B.INPC_DEV_BAD_WEIGHT
    leaf, pos = api.sample_octree(c, l, torch.zeros_like(w), 1.0, 0, 0, 1000, ws=ws)
    st = api.read_device_status(ws)
    assert st & B.INPC_DEV_NO_WEIGHT
    assert int(leaf.min()) >= 0 and int(leaf.max()) < t.n_leaves, "outputs stay in bounds"
    api.sample_octree(c, l, w, 1.0, 0, 0, 1000, ws=ws)
    assert api.read_device_status(ws) == 0


def test_stream_ordering_and_determinism(gpu):
    t = scenes.make_octree(8, 4096 + 700)
    c, l, w = _dev_tree(t, gpu)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = api.sample_octree(c, l, w, 1.0, 11, 2, 300_000)
    s.synchronize()
    b = api.sample_octree(c, l, w, 1.0, 11, 2, 300_000)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def _kat_cases():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")))
    return [([int(x, 16) for x in c["key"]], [int(x, 16) for x in c["ctr"]], [int(x, 16) for x in c["out"]])
            for c in g["cases"]]


def _device_philox(keys, ctrs, dev):
    # uint32 words carried in int64 on the host, int32 bit patterns on the device
    k = torch.from_numpy(np.asarray(keys, np.uint32).view(np.int32)).to(dev)
    c = torch.from_numpy(np.asarray(ctrs, np.uint32).view(np.int32)).to(dev)
    out = torch.empty(len(keys), 4, dtype=torch.int32, device=dev)
    B.inpc_philox4x32_10(k.data_ptr(), c.data_ptr(), len(keys), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def test_device_philox_known_answers(gpu):
    # the device generator (the one the sampler's kernels call) against the
    # published known-answer values of Philox4x32-10
    cases = _kat_cases()
    got = _device_philox([c[0] for c in cases], [c[1] for c in cases], gpu)
    for k, (_, _, want) in enumerate(cases):
        assert [int(x) for x in got[k]] == want


def test_sampler_positions_are_the_device_generator_words(gpu):
    # one level-0 leaf centred at 1/2, edge 1: position = (r_d >> 8) 2^-24 of
    # Philox(key = seed, counter = (slot, 0, view, 1)), exactly in FP32
    seed, view, n = 0x0123456789ABCDEF, 7, 4096 + 3
    c = torch.tensor([[0.5, 0.5, 0.5]], dtype=torch.float32, device=gpu)
    l = torch.zeros(1, dtype=torch.int32, device=gpu)
    w = torch.ones(1, dtype=torch.float64, device=gpu)
    leaf, pos = api.sample_octree(c, l, w, 1.0, seed, view, n)
    keys = [[seed & 0xFFFFFFFF, seed >> 32]] * n
    ctrs = [[k, 0, view, 1] for k in range(n)]
    r = _device_philox(keys, ctrs, gpu).astype(np.int64)
    want = ((r[:, :3] >> 8).astype(np.float64) * 2.0 ** -24).astype(np.float32)
    assert np.array_equal(pos.cpu().numpy(), want)
    assert int(leaf.abs().sum()) == 0
