"""The persistent front end of a batch (inpc_sample_query_batch): the
sampling and grid query of several views of uneven sample counts in one
work-queue launch must give bit-identical leaf indices, positions and
features to inpc_sample_octree + inpc_query_hashgrid of each view (which
the sampling and query tests compare with the oracle), on both count paths
of the sampler (trees up to 4,096 leaves and larger), FP32 and BF16, across
repeated calls on one workspace.  Its waits are bounded: an injected
dependency that never completes (host-side fault "queue_short") makes the
wait run out, the kernel returns with INPC_DEV_TIMEOUT in its status word,
and the next call is correct again.  The persistent batch form of
inpc_render_batch renders every view exactly as the stream-fork form."""
import numpy as np
import pytest
import torch

from paper_2403_16862_gb300 import _binding as B
from paper_2403_16862_gb300 import api, scenes
from paper_2403_16862_gb300.batch import ViewBatch

pytestmark = pytest.mark.gpu

RES16 = scenes.geometric_resolutions(16, 16, 4096)


def _tree(octree, dev):
    t = tuple(torch.from_numpy(x).to(dev) for x in (octree.centers, octree.levels, octree.weights))
    return t, B.InpcOctree(t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), octree.root_size, octree.n_leaves)


def _front(dev, tree_c, octree, desc, table, counts, view_ids, seed, ws, max_wait_us=2_000_000):
    hdt = torch.bfloat16 if desc.out_dtype == B.INPC_BF16 else torch.float32
    C = desc.n_levels * 4
    outs, views = [], []
    for n, vid in zip(counts, view_ids):
        o = dict(leaf=torch.full((max(n, 1),), -7, dtype=torch.int32, device=dev),
                 pos=torch.full((max(n, 1), 3), float("nan"), dtype=torch.float32, device=dev),
                 h=torch.full((max(n, 1), C), float("nan"), dtype=hdt, device=dev))
        outs.append(o)
        views.append(B.InpcFrontView(view_id=vid, n_samples=n, leaf_idx=o["leaf"].data_ptr(),
                                     pos=o["pos"].data_ptr(), h=o["h"].data_ptr()))
    B.inpc_sample_query_batch(tree_c, seed, desc, table.data_ptr(), views, max_wait_us, ws.data_ptr(), ws.numel(),
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return outs


def _alone(dev, tree_t, octree, desc, table, n, vid, seed):
    c, l, w = tree_t
    leaf, pos = api.sample_octree(c, l, w, octree.root_size, seed, vid, n)
    h = api.query_hashgrid(desc, table, pos)
    torch.cuda.synchronize()
    return leaf, pos, h


@pytest.mark.parametrize("n_leaves,start,bf16", [(4096, 4, False), (65536, 4, False), (65536, 4, True),
                                                 (4096 + 7 * 300, 4, True)])
def test_front_matches_per_view_calls(gpu, n_leaves, start, bf16):
    octree = scenes.make_octree(2, n_leaves, start_level=start)
    tree_t, tree_c = _tree(octree, gpu)
    grid = scenes.make_hashgrid(3, api.hashgrid_n_entries(RES16, 19), RES16, 19)
    t32 = torch.from_numpy(grid.table).to(gpu)
    if bf16:
        desc = api.hashgrid_desc(RES16, 19, table_dtype=torch.bfloat16, out_dtype=torch.bfloat16)
        table = t32.to(torch.bfloat16)
    else:
        desc, table = api.hashgrid_desc(RES16, 19), t32
    counts = [300_001, 0, 77_777, 1, 4096 * 3 + 5]
    vids = [5, 9, 0, 3, 11]
    ws = api.workspace(B.inpc_sample_query_batch_workspace_size(n_leaves, len(counts)), gpu)
    for rep in range(2):  # the second call reuses the workspace the first left behind
        outs = _front(gpu, tree_c, octree, desc, table, counts, vids, 17, ws)
        assert B.inpc_read_device_status(ws.data_ptr(), torch.cuda.current_stream().cuda_stream) == 0
        for o, n, vid in zip(outs, counts, vids):
            if n == 0:
                continue
            leaf, pos, h = _alone(gpu, tree_t, octree, desc, table, n, vid, 17)
            assert torch.equal(o["leaf"][:n], leaf), (rep, vid)
            assert torch.equal(o["pos"][:n], pos), (rep, vid)
            assert torch.equal(o["h"][:n], h), (rep, vid)


def test_front_flags_bad_weights(gpu):
    octree = scenes.make_octree(4, 4096 + 7 * 20)
    tree_t, _ = _tree(octree, gpu)
    w_bad = tree_t[2].clone()
    w_bad[5] = float("nan")
    bad = B.InpcOctree(tree_t[0].data_ptr(), tree_t[1].data_ptr(), w_bad.data_ptr(), octree.root_size,
                       octree.n_leaves)
    desc = api.hashgrid_desc(RES16, 16)
    table = torch.zeros(api.hashgrid_n_entries(RES16, 16), 4, dtype=torch.float32, device=gpu)
    ws = api.workspace(B.inpc_sample_query_batch_workspace_size(octree.n_leaves, 2), gpu)
    outs = _front(gpu, bad, octree, desc, table, [1000, 2000], [0, 1], 0, ws)
    st = B.inpc_read_device_status(ws.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st & B.INPC_DEV_BAD_WEIGHT and not st & B.INPC_DEV_TIMEOUT
    assert int(outs[1]["leaf"].min()) >= 0 and int(outs[1]["leaf"].max()) < octree.n_leaves


def test_front_wait_runs_out_and_returns(gpu):
    # the injected fault makes view 0's count scan wait for one draw tile
    # more than exists; with a 2 ms bound the wait gives up, the kernel
    # returns, the status says so, and the fault is disarmed by that launch
    octree = scenes.make_octree(5, 4096 + 7 * 40)
    tree_t, tree_c = _tree(octree, gpu)
    desc = api.hashgrid_desc(RES16, 16)
    grid = scenes.make_hashgrid(6, api.hashgrid_n_entries(RES16, 16), RES16, 16)
    table = torch.from_numpy(grid.table).to(gpu)
    ws = api.workspace(B.inpc_sample_query_batch_workspace_size(octree.n_leaves, 3), gpu)
    stream = torch.cuda.current_stream().cuda_stream
    B.inpc_set_fault("queue_short")
    try:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _front(gpu, tree_c, octree, desc, table, [50_000, 60_000, 70_000], [0, 1, 2], 3, ws, max_wait_us=2000)
        e1.record()
        torch.cuda.synchronize()
    finally:
        B.inpc_set_fault(None)
    st = B.inpc_read_device_status(ws.data_ptr(), stream)
    assert st & B.INPC_DEV_TIMEOUT
    assert e0.elapsed_time(e1) < 1000.0, "the bounded wait ended the launch"
    # the fault was taken by that launch: the next call completes and is exact
    outs = _front(gpu, tree_c, octree, desc, table, [50_000, 60_000, 70_000], [0, 1, 2], 3, ws)
    assert B.inpc_read_device_status(ws.data_ptr(), stream) == 0
    leaf, pos, h = _alone(gpu, tree_t, octree, desc, table, 50_000, 0, 3)
    assert torch.equal(outs[0]["leaf"][:50_000], leaf) and torch.equal(outs[0]["h"][:50_000], h)


def test_persistent_batch_renders_as_the_fork_form(gpu, tmp_path, monkeypatch):
    monkeypatch.setenv("INPC_TUNE_CACHE", str(tmp_path / "tune.json"))
    octree = scenes.make_octree(7, 4096 + 7 * 500)
    tree_t, _ = _tree(octree, gpu)
    grid = scenes.make_hashgrid(8, api.hashgrid_n_entries(RES16, 16), RES16, 16)
    table = torch.from_numpy(grid.table).to(gpu)
    desc = api.hashgrid_desc(RES16, 16)
    sizes = [(160, 120), (96, 64), (200, 100)]
    cams = scenes.orbit_cameras(sizes, focal_ref=160.0, ref_height=120)
    grads = [torch.from_numpy(scenes.upstream_grad(30 + v, (h, w, 64))).to(gpu) for v, (w, h) in enumerate(sizes)]
    a = ViewBatch(*tree_t, octree.root_size, desc, table, cams, 120_000, grads, seed=2, n_streams=2, tune=False)
    b = ViewBatch(*tree_t, octree.root_size, desc, table, cams, 120_000, grads, seed=2, n_streams=2, tune=False,
                  persistent=True)
    a.capture()
    b.capture()
    a.step()
    b.step()
    torch.cuda.synchronize()
    for va, vb in zip(a.views, b.views):
        assert torch.equal(va["img"], vb["img"]) and torch.equal(va["nc"], vb["nc"])
        assert torch.equal(va["h"], vb["h"]) and torch.equal(va["pos"], vb["pos"])
    e = (torch.linalg.norm(a.grad_table.double() - b.grad_table.double()) / torch.linalg.norm(a.grad_table.double()))
    assert float(e) < 1e-6
    st = B.inpc_read_device_status(b.front_ws.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0


def test_persistent_batch_beyond_one_front_launch(gpu, tmp_path, monkeypatch):
    # more than 64 views: inpc_render_batch_persistent runs its front end in
    # launches of 64 views; every view still renders as in the fork form
    monkeypatch.setenv("INPC_TUNE_CACHE", str(tmp_path / "tune.json"))
    octree = scenes.make_octree(9, 4096 + 7 * 50)
    tree_t, _ = _tree(octree, gpu)
    grid = scenes.make_hashgrid(10, api.hashgrid_n_entries(RES16, 14), RES16, 14)
    table = torch.from_numpy(grid.table).to(gpu)
    desc = api.hashgrid_desc(RES16, 14)
    sizes = [(48, 32)] * 70
    cams = scenes.orbit_cameras(sizes, focal_ref=48.0, ref_height=32)
    grads = [torch.from_numpy(scenes.upstream_grad(40 + v, (h, w, 64))).to(gpu) for v, (w, h) in enumerate(sizes)]
    a = ViewBatch(*tree_t, octree.root_size, desc, table, cams, 3000, grads, seed=4, n_streams=4, tune=False)
    b = ViewBatch(*tree_t, octree.root_size, desc, table, cams, 3000, grads, seed=4, n_streams=4, tune=False,
                  persistent=True)
    a.run_eager()
    b.run_eager()
    torch.cuda.synchronize()
    for v, (va, vb) in enumerate(zip(a.views, b.views)):
        assert torch.equal(va["pos"], vb["pos"]) and torch.equal(va["h"], vb["h"]), v
        assert torch.equal(va["img"], vb["img"]), v
    e = (torch.linalg.norm(a.grad_table.double() - b.grad_table.double()) / torch.linalg.norm(a.grad_table.double()))
    assert float(e) < 1e-6


def test_injected_argument_corruption_launches_nothing(gpu):
    # with real device buffers, a corrupted first array argument (host-side
    # fault "corrupt_args") is caught by each call's own validation: the call
    # returns INPC_ERR_INVALID_ARG and launches no kernel
    octree = scenes.make_octree(11, 4096 + 7 * 10)
    tree_t, tree_c = _tree(octree, gpu)
    desc = api.hashgrid_desc(RES16, 14)
    table = torch.zeros(api.hashgrid_n_entries(RES16, 14), 4, dtype=torch.float32, device=gpu)
    n = 5000
    leaf = torch.empty(n, dtype=torch.int32, device=gpu)
    pos = torch.rand(n, 3, device=gpu)
    h = torch.empty(n, 64, device=gpu)
    ws_s = api.workspace(B.inpc_sample_workspace_size(octree.n_leaves, n), gpu)
    fws = api.workspace(B.inpc_sample_query_batch_workspace_size(octree.n_leaves, 1), gpu)
    stream = torch.cuda.current_stream().cuda_stream
    fv = [B.InpcFrontView(view_id=0, n_samples=n, leaf_idx=leaf.data_ptr(), pos=pos.data_ptr(), h=h.data_ptr())]
    calls = [
        lambda: B.inpc_sample_octree(tree_c, 0, 0, n, leaf.data_ptr(), pos.data_ptr(), None, ws_s.data_ptr(),
                                     ws_s.numel(), stream),
        lambda: B.inpc_query_hashgrid(desc, table.data_ptr(), pos.data_ptr(), n, h.data_ptr(), stream),
        lambda: B.inpc_sample_query_batch(tree_c, 0, desc, table.data_ptr(), fv, 1000, fws.data_ptr(), fws.numel(),
                                          stream),
    ]
    torch.cuda.synchronize()
    before = B.inpc_kernel_launches()
    B.inpc_set_fault("corrupt_args")
    try:
        for call in calls:
            with pytest.raises(B.InpcError) as e:
                call()
            assert e.value.status == B.INPC_ERR_INVALID_ARG
    finally:
        B.inpc_set_fault(None)
    assert B.inpc_kernel_launches() == before
    calls[0]()  # disarmed: the same call runs
    torch.cuda.synchronize()
    assert B.inpc_kernel_launches() > before
