"""Batching form: several views of uneven size, forward and backward, spread
over streams and replayed from one CUDA graph (ViewBatch), and the tile
autotuner.  Each view's image and the shared table gradient are checked
against the oracle's own pipeline; the graph replay against the eager pass;
the BF16 batch against the FP32 batch (stated error)."""
import numpy as np
import pytest
import torch

from paper_2403_16862_gb300 import _binding as B
from paper_2403_16862_gb300 import api, autotune, scenes
from paper_2403_16862_gb300.batch import ViewBatch
from tests._parity import assert_cond_close
from tests.test_gpu_raster import _excluded_points

pytestmark = pytest.mark.gpu

RES16 = scenes.geometric_resolutions(16, 16, 4096)
SIZES = [(160, 120), (96, 64), (200, 150)]
N = 60_000
LOG2_T = 14


def _scene(oracle, seed=0):
    tree = scenes.make_octree(seed, 4096 + 7 * 300)
    grid = scenes.make_hashgrid(seed + 1, oracle.hash_entries(RES16, LOG2_T), RES16, LOG2_T)
    cams = scenes.orbit_cameras(SIZES, focal_ref=180.0, ref_height=120)
    grads = [scenes.upstream_grad(seed + 2 + v, (h, w, 64)) for v, (w, h) in enumerate(SIZES)]
    return tree, grid, cams, grads


def _batch(gpu, tree, grid, cams, grads, bf16=False, tune=False, n_streams=2):
    c, l, w = (torch.from_numpy(x).to(gpu) for x in (tree.centers, tree.levels, tree.weights))
    table = torch.from_numpy(grid.table).to(gpu)
    dt = torch.bfloat16 if bf16 else torch.float32
    desc = api.hashgrid_desc(RES16, LOG2_T, table_dtype=dt, out_dtype=dt)
    g = [torch.from_numpy(x).to(gpu) for x in grads]
    return ViewBatch(c, l, w, tree.root_size, desc, table.to(dt), cams, N, g, seed=5, n_streams=n_streams,
                     bf16=bf16, tune=tune)


def test_batch_matches_oracle_and_graph_replays(gpu, oracle, tmp_path, monkeypatch):
    monkeypatch.setenv("INPC_TUNE_CACHE", str(tmp_path / "tune.json"))
    tree, grid, cams, grads = _scene(oracle)
    vb = _batch(gpu, tree, grid, cams, grads, tune=True)
    vb.run_eager()
    torch.cuda.synchronize()
    eager_img = [d["img"].clone() for d in vb.views]
    eager_gt = vb.grad_table.clone()

    # oracle: every view samples its own points (view id = its index)
    o_gt = np.zeros(grid.table.shape)
    o_gab = np.zeros(grid.table.shape)
    excluded_rows = np.zeros(grid.table.shape)
    for v, cam in enumerate(cams):
        _, o_pos64, _ = oracle.sample_octree(tree, 5, v, N)
        o_pos = o_pos64.astype(np.float32)
        assert np.array_equal(vb.views[v]["pos"].cpu().numpy(), o_pos)
        o_h, o_hab = oracle.hash_fwd(RES16, LOG2_T, grid.table, o_pos, with_abs=True)
        ref = oracle.raster_fwd(cam, o_pos, o_h, head_mode=True, with_abs=True, feat_abs=o_hab)
        ok = ref["flags"] == 0
        assert (~ok).sum() <= max(2, 1e-4 * ok.size)
        assert_cond_close(eager_img[v].cpu().numpy(), ref["image"], ref["abs"], mask=ok[..., None],
                          what="view %d image" % v)
        rb = oracle.raster_bwd(cam, o_pos, o_h, grads[v], head_mode=True, with_abs=True, feat_abs=o_hab)
        gt, gab = oracle.hash_bwd(RES16, LOG2_T, 4, o_pos, rb["d_feat"], with_abs=True, dh_abs=rb["abs_feat"])
        o_gt += gt
        o_gab += gab
        keep = ~_excluded_points(oracle, cam, o_pos, ref["flags"])
        excluded_rows += oracle.hash_bwd(RES16, LOG2_T, 4, o_pos, np.repeat((~keep)[:, None], 64, 1).astype(np.float64))
    assert_cond_close(eager_gt.cpu().numpy(), o_gt, o_gab, mask=excluded_rows == 0, what="shared grad_table")

    # the tuner cached one of its candidates for every view shape
    for d in vb.views:
        assert (d["opts"].tile_w, d["opts"].tile_h) in autotune.CANDIDATES
    assert (tmp_path / "tune.json").exists()

    # graph replay: the forward is deterministic (bitwise), the table
    # gradient equal up to the order of its atomic additions
    vb.capture()
    launches0 = B.inpc_kernel_launches()
    for _ in range(2):
        vb.step()
    torch.cuda.synchronize()
    assert B.inpc_kernel_launches() == launches0, "a replay launches nothing through the library's host code"
    for v, d in enumerate(vb.views):
        assert torch.equal(d["img"], eager_img[v])
    assert_cond_close(vb.grad_table.cpu().numpy(), eager_gt.cpu().numpy(), o_gab, what="replayed grad_table")


def test_tiles_do_not_change_results(gpu, oracle, tmp_path, monkeypatch):
    """Every autotuner candidate gives bitwise the same image and, up to
    atomic order, the same table gradient."""
    monkeypatch.setenv("INPC_TUNE_CACHE", str(tmp_path / "tune.json"))
    tree, grid, cams, grads = _scene(oracle, seed=3)
    vb = _batch(gpu, tree, grid, cams[2:], grads[2:], tune=False, n_streams=1)
    vb.run_eager()
    torch.cuda.synchronize()
    d = vb.views[0]
    ref_img = d["img"].clone()
    ref_gt = vb.grad_table.clone()
    for tw, th in autotune.CANDIDATES:
        d["opts"].tile_w, d["opts"].tile_h = tw, th
        vb.run_eager()
        torch.cuda.synchronize()
        assert torch.equal(d["img"], ref_img), (tw, th)
        diff = (vb.grad_table - ref_gt).abs().max().item()
        assert diff <= 1e-5 * ref_gt.abs().max().item() + 1e-7, (tw, th, diff)
    best = autotune.tuned_tiles(d["cam"], d["opts"], vb.desc, d["pos"], d["h"], d["d_image"])
    assert best in autotune.CANDIDATES
    assert autotune.tuned_tiles(d["cam"], d["opts"], vb.desc, d["pos"], d["h"], d["d_image"]) == best


def test_bf16_batch_error_statement(gpu, oracle, tmp_path, monkeypatch):
    monkeypatch.setenv("INPC_TUNE_CACHE", str(tmp_path / "tune.json"))
    tree, grid, cams, grads = _scene(oracle, seed=7)
    f32 = _batch(gpu, tree, grid, cams, grads)
    b16 = _batch(gpu, tree, grid, cams, grads, bf16=True)
    f32.step()
    b16.step()
    torch.cuda.synchronize()
    for v in range(len(cams)):
        a, b = f32.views[v]["img"].double(), b16.views[v]["img"].double()
        e = (torch.linalg.norm(a - b) / torch.linalg.norm(a)).item()
        print("BF16 batch view %d image: norm-wise rel. difference to FP32 %.3e" % (v, e))
        assert e < 2.0 ** -6
    a, b = f32.grad_table.double(), b16.grad_table.double()
    e = (torch.linalg.norm(a - b) / torch.linalg.norm(a)).item()
    print("BF16 batch grad_table: norm-wise rel. difference to FP32 %.3e" % e)
    assert e < 2.0 ** -5
