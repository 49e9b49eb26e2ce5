"""The allocation-free sampler entry point (inpc_sample_octree_noalloc).

It serves callers that cannot allocate device memory: its scratch is a fixed
device array inside the library.  Called through the C ABI, it must give
exactly the outputs of inpc_sample_octree with a caller workspace, on two
calls in a row (the shared array keeps the previous call's contents, so the
second call checks that everything that must start at zero is cleared).
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2403_16862_gb300 import _binding as B
from paper_2403_16862_gb300 import scenes

pytestmark = pytest.mark.gpu


def _tree_struct(t, dev):
    c = torch.from_numpy(t.centers).to(dev)
    l = torch.from_numpy(t.levels).to(dev)
    w = torch.from_numpy(t.weights).to(dev)
    return (c, l, w), B.InpcOctree(c.data_ptr(), l.data_ptr(), w.data_ptr(), t.root_size, t.n_leaves)


def _run(entry, tree, seed, view, n, dev, ws=None):
    leaf = torch.empty(n, dtype=torch.int32, device=dev)
    pos = torch.empty(n, 3, dtype=torch.float32, device=dev)
    counts = torch.empty(tree.n_leaves, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    if entry == "noalloc":
        B.inpc_sample_octree_noalloc(tree, seed, view, n, leaf.data_ptr(), pos.data_ptr(), counts.data_ptr(), stream)
    else:
        B.inpc_sample_octree(tree, seed, view, n, leaf.data_ptr(), pos.data_ptr(), counts.data_ptr(), ws.data_ptr(),
                             ws.numel(), stream)
    torch.cuda.synchronize()
    return leaf.cpu().numpy(), pos.cpu().numpy(), counts.cpu().numpy()


def test_noalloc_matches_workspace_entry_twice(gpu):
    # two different trees and draws in a row: the second call reuses the
    # array the first one left behind
    cases = [(scenes.make_octree(0, 65536), 0, 0, 1_000_000), (scenes.make_octree(1, 4096 + 7 * 500), 5, 3, 300_000)]
    for octree, seed, view, n in cases:
        keep, tree = _tree_struct(octree, gpu)
        ws = torch.empty(B.inpc_sample_workspace_size(octree.n_leaves, n), dtype=torch.uint8, device=gpu)
        ref = _run("workspace", tree, seed, view, n, gpu, ws)
        got = _run("noalloc", tree, seed, view, n, gpu)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)


def test_noalloc_rejects_trees_beyond_the_static_array(gpu):
    octree = scenes.make_octree(2, 1 << 20, start_level=6)
    keep, tree = _tree_struct(octree, gpu)
    need = B.inpc_sample_workspace_size(octree.n_leaves, 10)
    assert need > B.INPC_SAMPLE_STATIC_SCRATCH_BYTES
    with pytest.raises(B.InpcError) as e:
        _run("noalloc", tree, 0, 0, 10, gpu)
    assert e.value.status == B.INPC_ERR_CAPACITY and "static" in str(e.value)


def test_noalloc_device_status_is_readable(gpu):
    # the sampler's device status word is the first word of the static array;
    # inpc_read_device_status with a null workspace reads it.  A NaN weight
    # and an all-zero tree are flagged, the outputs stay inside the tree, and
    # the next good call clears the word again.
    octree = scenes.make_octree(3, 4096 + 7 * 100)
    stream = torch.cuda.current_stream().cuda_stream
    keep, tree = _tree_struct(octree, gpu)
    _run("noalloc", tree, 0, 0, 10_000, gpu)
    assert B.inpc_read_device_status(None, stream) == 0
    w_bad = keep[2].clone()
    w_bad[17] = float("nan")
    bad = B.InpcOctree(keep[0].data_ptr(), keep[1].data_ptr(), w_bad.data_ptr(), octree.root_size, octree.n_leaves)
    _run("noalloc", bad, 0, 0, 10_000, gpu)
    assert B.inpc_read_device_status(None, stream) & B.INPC_DEV_BAD_WEIGHT
    w_zero = torch.zeros_like(keep[2])
    zero = B.InpcOctree(keep[0].data_ptr(), keep[1].data_ptr(), w_zero.data_ptr(), octree.root_size, octree.n_leaves)
    leaf, _, _ = _run("noalloc", zero, 0, 0, 10_000, gpu)
    assert B.inpc_read_device_status(None, stream) & B.INPC_DEV_NO_WEIGHT
    assert leaf.min() >= 0 and leaf.max() < octree.n_leaves, "outputs stay in bounds"
    _run("noalloc", tree, 0, 0, 10_000, gpu)
    assert B.inpc_read_device_status(None, stream) == 0
