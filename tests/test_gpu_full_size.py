"""Full-size checks of the precision and batching workloads, in the launch
configuration the benchmark times (sampling, query, rasterizer forward and
the fused backward).

* Precision workload: 1,048,576-leaf octree, 16,777,216 samples, 16-level
  2^21 x 4 grid, head mode, 1920x1080.  The FP32 path is compared with the
  oracle element by element (bit-exact samples, the 1e-5 rule elsewhere);
  the BF16 path (BF16 table, h and image; FP32 arithmetic, transmittance
  and gradients) against the same oracle run, its error stated per output
  and bounded as BF16 storage implies.
* Batching workload: 8 views of uneven size, 8,388,608 samples each, BF16,
  one CUDA graph over 4 streams with autotuned tiles.  Every view's image
  is bitwise the image of that view rendered on its own (a path the
  precision check compares with the oracle), and the shared table gradient
  is the sum of the views' own gradients up to the order of FP32 additions;
  the persistent front end renders the same images and features bitwise.

The oracle's FP64 arrays at 16M samples take about 40 GB of host memory;
the precision check skips on hosts with less available."""
import numpy as np
import pytest
import torch

from paper_2403_16862_gb300 import api, scenes
from paper_2403_16862_gb300.batch import ViewBatch
from tests._parity import assert_cond_close, cond_ratio
from tests.test_gpu_raster import _excluded_points, _product_widening

pytestmark = pytest.mark.gpu

RES16 = scenes.geometric_resolutions(16, 16, 4096)
LOG2_T = 21
ROWS = 1 << 20  # rows per host-side comparison chunk


def _mem_available_gb():
    with open("/proc/meminfo") as f:
        for line in f:
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 2 ** 20
    return 0.0


def _scene():
    tree = scenes.make_octree(0, 1 << 20, start_level=6)
    grid = scenes.make_hashgrid(1, api.hashgrid_n_entries(RES16, LOG2_T), RES16, LOG2_T)
    return tree, grid


def _close_rows(got, ref, scale, widen=None, mask=None, what=""):
    """The 1e-5 rule, row chunk by row chunk (GPU tensor against host
    arrays); ``widen`` [rows] scales a row's tolerance."""
    for r0 in range(0, ref.shape[0], ROWS):
        sl = slice(r0, r0 + ROWS)
        sc = scale[sl] if widen is None else scale[sl] * widen[sl, None]
        assert_cond_close(got[sl].float().cpu().numpy(), ref[sl], sc,
                          mask=None if mask is None else mask[sl], what="%s rows %d+" % (what, r0))


class _Err:
    """Norm-wise relative error and max |error| / max sum|terms|, accumulated
    over chunks."""
    def __init__(self):
        self.d2 = self.r2 = self.dmax = self.smax = 0.0

    def add(self, got, ref, scale, mask=None):
        d = got.astype(np.float64) - ref
        if mask is not None:
            d = np.where(mask, d, 0.0)
            ref = np.where(mask, ref, 0.0)
        self.d2 += float(np.square(d).sum())
        self.r2 += float(np.square(ref).sum())
        self.dmax = max(self.dmax, float(np.abs(d).max()) if d.size else 0.0)
        self.smax = max(self.smax, float(np.max(scale)) if np.size(scale) else 0.0)
        return self

    def add_rows(self, got, ref, scale, mask=None):
        for r0 in range(0, ref.shape[0], ROWS):
            sl = slice(r0, r0 + ROWS)
            self.add(got[sl].float().cpu().numpy(), ref[sl], scale[sl], None if mask is None else mask[sl])
        return self

    @property
    def normwise(self):
        return (self.d2 / max(self.r2, 1e-300)) ** 0.5

    @property
    def maxrel(self):
        return self.dmax / max(self.smax, 1e-300)


def _gpu_view(gpu, tree_t, table, desc, opts, cam, g, n, view_id=0):
    c, l, w, rs = tree_t
    leaf, pos = api.sample_octree(c, l, w, rs, 0, view_id, n)
    h = api.query_hashgrid(desc, table, pos)
    ws = api.workspace(api.rasterize_bwd_hashgrid_workspace_size(cam, opts, desc, n), gpu)
    img, T, nc, ws = api.rasterize_fwd(cam, opts, pos, h, ws=ws)
    gt = torch.zeros(table.shape, dtype=torch.float32, device=gpu)
    dh = torch.empty(n, 64, dtype=torch.float32, device=gpu)
    api.rasterize_bwd_hashgrid(cam, opts, desc, pos, h, T, nc, g, ws, gt, d_feat=dh)
    del ws
    return dict(leaf=leaf, pos=pos, h=h, img=img, T=T, nc=nc, gt=gt, dh=dh)


def test_precision_workload_full_size(gpu, oracle):
    if _mem_available_gb() < 64:
        pytest.skip("the FP64 oracle at 16M samples needs about 40 GB of host memory")
    n = 1 << 24
    f = 900.0 * 1080 / 832
    cam = scenes.make_camera((0.5, 0.5, -1.2), f, f, 960.0, 540.0, 1920, 1080)
    tree, grid = _scene()
    g_img = scenes.upstream_grad(11, (cam.height, cam.width, 64))

    # ---- GPU: FP32 and BF16 forms of the same view
    tree_t = tuple(torch.from_numpy(x).to(gpu) for x in (tree.centers, tree.levels, tree.weights)) + (tree.root_size,)
    t32 = torch.from_numpy(grid.table).to(gpu)
    g = torch.from_numpy(g_img).to(gpu)
    r32 = _gpu_view(gpu, tree_t, t32, api.hashgrid_desc(RES16, LOG2_T), api.RasterOptions(n_channels=64, head_mode=True),
                    cam, g, n)
    d16 = api.hashgrid_desc(RES16, LOG2_T, table_dtype=torch.bfloat16, out_dtype=torch.bfloat16)
    r16 = _gpu_view(gpu, tree_t, t32.to(torch.bfloat16), d16,
                    api.RasterOptions(n_channels=64, head_mode=True, bf16=True), cam, g, n)
    torch.cuda.synchronize()
    assert torch.equal(r16["pos"], r32["pos"])

    # ---- oracle, stage by stage, each output compared as soon as it exists
    o_leaf, o_pos64, _ = oracle.sample_octree(tree, 0, 0, n)
    o_pos = o_pos64.astype(np.float32)
    del o_pos64
    assert np.array_equal(r32["leaf"].cpu().numpy(), o_leaf), "leaf indices"
    assert np.array_equal(r32["pos"].cpu().numpy(), o_pos), "positions"
    del o_leaf
    o_h, o_hab = oracle.hash_fwd(RES16, LOG2_T, grid.table, o_pos, with_abs=True)
    _close_rows(r32["h"], o_h, o_hab, what="h")
    e_h = _Err().add_rows(r16["h"], o_h, o_hab)
    ref = oracle.raster_fwd(cam, o_pos, o_h, head_mode=True, with_abs=True, feat_abs=o_hab)
    rb = oracle.raster_bwd(cam, o_pos, o_h, g_img, head_mode=True, with_abs=True, feat_abs=o_hab)
    del o_h, o_hab
    ok = ref["flags"] == 0
    assert (~ok).sum() <= max(2, 1e-4 * ok.size)
    assert np.array_equal(r32["nc"].cpu().numpy()[ok], ref["n_contrib"][ok]), "blended counts"
    # pixels blending more than ~170 fragments widen the bound to n 2^-24
    wp, wpt = _product_widening(oracle, cam, o_pos, ref["n_contrib"])
    assert_cond_close(r32["img"].cpu().numpy(), ref["image"], ref["abs"] * wp[..., None], mask=ok[..., None],
                      what="image")
    assert_cond_close(r32["T"].cpu().numpy(), ref["T_final"], ref["T_final"] * wp, mask=ok, what="T_final")
    print("bound used without the long-blend widening: image %.3f, T_final %.3f"
          % (cond_ratio(r32["img"].cpu().numpy(), ref["image"], ref["abs"], mask=ok[..., None]),
             cond_ratio(r32["T"].cpu().numpy(), ref["T_final"], ref["T_final"], mask=ok)))
    e_img = _Err().add(r16["img"].float().cpu().numpy(), ref["image"], ref["abs"])
    e_T = _Err().add(r16["T"].cpu().numpy(), ref["T_final"], ref["T_final"])
    keep = ~_excluded_points(oracle, cam, o_pos, ref["flags"])
    del ref
    _close_rows(r32["dh"], rb["d_feat"], rb["abs_feat"], widen=wpt, mask=keep[:, None], what="dh")
    e_dh = _Err().add_rows(r16["dh"], rb["d_feat"], rb["abs_feat"])
    rb["abs_feat"] *= wpt[:, None]  # the table gradient's scale carries the widened dh scale
    o_gt, o_gab = oracle.hash_bwd(RES16, LOG2_T, 4, o_pos, rb["d_feat"], with_abs=True, dh_abs=rb["abs_feat"])
    del rb
    # table rows reached by a point with a fragment in a threshold-ambiguous pixel
    reach = np.zeros(o_gt.shape[0], bool)
    if (~keep).any():
        m = int((~keep).sum())
        reach = oracle.hash_bwd(RES16, LOG2_T, 4, o_pos[~keep], np.ones((m, 64))).any(axis=1)
    assert_cond_close(r32["gt"].cpu().numpy(), o_gt, o_gab, mask=~reach[:, None], what="grad_table")
    e_gt = _Err().add(r16["gt"].cpu().numpy(), o_gt, o_gab)

    stats = dict(h=e_h, image=e_img, T_final=e_T, dh=e_dh, grad_table=e_gt)
    for k, e in stats.items():
        print("BF16 form at full size, %-10s norm-wise rel. error %.3e  max|err| / max sum|terms| %.3e"
              % (k, e.normwise, e.maxrel))
    # the bounds BF16 storage implies (each stored value carries <= 2^-9
    # relative rounding; T and the gradients inherit that of h)
    assert e_h.normwise < 2.0 ** -7
    assert e_img.normwise < 2.0 ** -6
    assert e_dh.normwise < 2.0 ** -5 and e_gt.normwise < 2.0 ** -5


def test_batching_workload_full_size(gpu, tmp_path, monkeypatch):
    monkeypatch.setenv("INPC_TUNE_CACHE", str(tmp_path / "tune.json"))
    sizes = [(640, 480), (960, 540), (1024, 768), (1280, 832), (1280, 832), (1600, 900), (1920, 1080), (1920, 1080)]
    cams = scenes.orbit_cameras(sizes)
    n = 1 << 23
    tree, grid = _scene()
    tree_t = tuple(torch.from_numpy(x).to(gpu) for x in (tree.centers, tree.levels, tree.weights)) + (tree.root_size,)
    t16 = torch.from_numpy(grid.table).to(gpu).to(torch.bfloat16)
    d16 = api.hashgrid_desc(RES16, LOG2_T, table_dtype=torch.bfloat16, out_dtype=torch.bfloat16)
    grads = [torch.from_numpy(scenes.upstream_grad(100 + v, (h, w, 64))).to(gpu) for v, (w, h) in enumerate(sizes)]
    vb = ViewBatch(*tree_t, d16, t16, cams, n, grads, seed=0, n_streams=4, bf16=True, tune=True)
    vb.capture()
    vb.step()
    torch.cuda.synchronize()

    total = torch.zeros(t16.shape, dtype=torch.float64, device=gpu)
    for v, cam in enumerate(cams):
        alone = _gpu_view(gpu, tree_t, t16, d16, api.RasterOptions(n_channels=64, head_mode=True, bf16=True), cam,
                          grads[v], n, view_id=v)
        torch.cuda.synchronize()
        assert torch.equal(alone["img"], vb.views[v]["img"]), "view %d image" % v
        assert torch.equal(alone["nc"], vb.views[v]["nc"]), "view %d blended counts" % v
        total += alone["gt"].double()
        del alone
    e = (torch.linalg.norm(vb.grad_table.double() - total) / torch.linalg.norm(total)).item()
    print("batched table gradient against the sum of the views' own: norm-wise rel. difference %.3e" % e)
    assert e < 1e-5
    # the persistent front end (sampling of all views in one work-queue
    # launch, their query in one more) renders the same batch bitwise
    tiles = [(d["opts"].tile_w, d["opts"].tile_h) for d in vb.views]
    vp = ViewBatch(*tree_t, d16, t16, cams, n, grads, seed=0, n_streams=4, bf16=True, tune=False, persistent=True)
    for d, (tw, th) in zip(vp.views, tiles):
        d["opts"].tile_w, d["opts"].tile_h = tw, th
    vp.capture()
    vp.step()
    torch.cuda.synchronize()
    from paper_2403_16862_gb300 import _binding as B
    assert B.inpc_read_device_status(vp.front_ws.data_ptr(), torch.cuda.current_stream().cuda_stream) == 0
    for v in range(len(cams)):
        assert torch.equal(vp.views[v]["img"], vb.views[v]["img"]), "view %d image (persistent front end)" % v
        assert torch.equal(vp.views[v]["h"], vb.views[v]["h"]), "view %d features (persistent front end)" % v
    ep = (torch.linalg.norm(vp.grad_table.double() - total) / torch.linalg.norm(total)).item()
    assert ep < 1e-5
