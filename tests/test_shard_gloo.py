"""The multi-GPU host logic on CPU ranks (gloo, world size 2): disjoint view
shards, the max-over-ranks timing, and the table-gradient sum a training loop
adds, checked against the oracle's gradient of both ranks' views."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2403_16862_gb300 import scenes, shard

RES = scenes.geometric_resolutions(6, 16, 256)
LOG2_T = 12
N = 3000


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _grads(oracle, tree, view):
    _, pos64, _ = oracle.sample_octree(tree, 0, view, N)
    dh = np.random.default_rng(50 + view).normal(size=(N, 4 * len(RES)))
    return oracle.hash_bwd(RES, LOG2_T, 4, pos64.astype(np.float32), dh)


def _rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle
        tree = scenes.make_octree(1, 4096 + 7 * 50)
        ids = [shard.view_ids(rank, world, step) for step in range(3)]
        every = [None] * world
        dist.all_gather_object(every, ids)
        flat = [v for r in every for step in r for v in step]
        assert len(flat) == len(set(flat)) == 3 * world
        assert sorted(flat) == list(range(3 * world))
        assert shard.max_over_ranks(1.5 + rank) == 1.5 + world - 1
        # each rank: its own view's table gradient, FP32, then the sum
        mine = _grads(oracle, tree, ids[0][0])
        g = torch.from_numpy(mine.astype(np.float32))
        shard.sum_table_grad(g)
        total = sum(_grads(oracle, tree, shard.view_ids(r, world, 0)[0]) for r in range(world))
        scale = sum(np.abs(_grads(oracle, tree, shard.view_ids(r, world, 0)[0])) for r in range(world))
        err = np.abs(g.numpy().astype(np.float64) - total)
        assert np.all(err <= 1e-6 * (scale + 1e-30) + 1e-7 * np.abs(total).max())
        np.save(os.path.join(out_dir, "rank%d.npy" % rank), g.numpy())

        # the overlapped exchange: each step's gradient accumulates into the
        # table GradExchange hands out, its sum starts asynchronously, and
        # the next step goes on; a table is summed before it is cleared and
        # written again two steps later
        gx = shard.GradExchange(mine.shape)
        for step in range(3):
            buf = gx.begin()
            buf += torch.from_numpy(_grads(oracle, tree, ids[step][0]).astype(np.float32))
            gx.launch()
            if step >= 1:
                prev = gx.result(step - 1).numpy().astype(np.float64)
                want = sum(_grads(oracle, tree, shard.view_ids(r, world, step - 1)[0]) for r in range(world))
                ab = sum(np.abs(_grads(oracle, tree, shard.view_ids(r, world, step - 1)[0])) for r in range(world))
                assert np.all(np.abs(prev - want) <= 1e-6 * (ab + 1e-30) + 1e-7 * np.abs(want).max()), step
        gx.finish()
        last = gx.result(2).numpy().astype(np.float64)
        want = sum(_grads(oracle, tree, shard.view_ids(r, world, 2)[0]) for r in range(world))
        assert np.allclose(last, want, rtol=0, atol=1e-6 * np.abs(want).max())
        with pytest.raises(ValueError):
            gx.result(0)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path, oracle):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    a, b = (np.load(tmp_path / ("rank%d.npy" % r)) for r in range(world))
    assert np.array_equal(a, b), "every rank holds the same summed gradient"


def test_view_ids_reject_bad_rank():
    with pytest.raises(ValueError):
        shard.view_ids(2, 2, 0)
    assert shard.view_ids(0, 1, 5) == [5]
    assert shard.max_over_ranks(3.25) == 3.25
