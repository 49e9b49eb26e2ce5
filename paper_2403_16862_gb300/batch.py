"""Many views per launch: the forward and backward of a batch of views of
uneven size, recorded once into a CUDA graph and replayed as one launch per
step.  Views are spread over several streams so that their kernels overlap
(small images leave most of the GPU idle on their own); all views share the
octree, the grid table and one FP32 table gradient (accumulated with atomic
adds).  Tile sizes come from the autotuner.

With ``persistent=True`` the sampling and grid query of all views run first
as one persistent work-queue launch (the leaf CDF built once for the batch),
and only the rasterizer's forward and backward are spread over the streams.

Every computation runs in ``libinpc.so``; this module only owns buffers,
streams and the graph.
"""
from __future__ import annotations

import torch

from . import _binding as B
from . import api
from .autotune import tuned_tiles


class ViewBatch:
    def __init__(self, centers, levels, weights, root_size, desc, table, cams, n_samples, d_images, seed=0,
                 n_streams=4, bf16=False, tune=True, persistent=False, max_wait_us=2_000_000):
        self.dev = table.device
        self.tree = (centers, levels, weights, float(root_size))
        self.desc = desc
        self.table = table
        self.cams = list(cams)
        self.n = int(n_samples)
        self.seed = int(seed)
        self.bf16 = bool(bf16)
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(max(1, n_streams))]
        C = desc.n_levels * desc.n_feats
        hdt = torch.bfloat16 if bf16 else torch.float32
        self.grad_table = torch.zeros(table.shape, dtype=torch.float32, device=self.dev)
        self.views = []
        for v, cam in enumerate(self.cams):
            opts = api.RasterOptions(n_channels=C, head_mode=True, bf16=bf16)
            d = dict(cam=cam, d_image=d_images[v], view_id=v)
            d["ws_s"] = api.workspace(B.inpc_sample_workspace_size(levels.shape[0], self.n), self.dev)
            d["leaf"] = torch.empty(self.n, dtype=torch.int32, device=self.dev)
            d["pos"] = torch.empty(self.n, 3, dtype=torch.float32, device=self.dev)
            d["h"] = torch.empty(self.n, C, dtype=hdt, device=self.dev)
            d["img"] = torch.empty(cam.height, cam.width, C, dtype=hdt, device=self.dev)
            d["T"] = torch.empty(cam.height, cam.width, dtype=torch.float32, device=self.dev)
            d["nc"] = torch.empty(cam.height, cam.width, dtype=torch.int32, device=self.dev)
            d["opts"] = opts
            self.views.append(d)
        if tune:
            self._tune()
        for d in self.views:
            d["ws_r"] = api.workspace(api.rasterize_bwd_hashgrid_workspace_size(d["cam"], d["opts"], desc, self.n),
                                      self.dev)
        # persistent form: the sampling and query of every view in one
        # work-queue launch (inpc_render_batch_persistent)
        self.persistent = bool(persistent)
        self.max_wait_us = int(max_wait_us)
        self.front_ws = None
        if self.persistent:
            nv = min(len(self.cams), 64)
            self.front_ws = api.workspace(B.inpc_sample_query_batch_workspace_size(levels.shape[0], nv), self.dev)
        self.graph = None
        self._job_array = None

    def _tune(self):
        # one eager pass per view provides realistic inputs for the tile search
        c, l, w, rs = self.tree
        for d in self.views:
            api.sample_octree(c, l, w, rs, self.seed, d["view_id"], self.n, ws=d["ws_s"], out=(d["leaf"], d["pos"]))
            api.query_hashgrid(self.desc, self.table, d["pos"], out=d["h"])
            tw, th = tuned_tiles(d["cam"], d["opts"], self.desc, d["pos"], d["h"], d["d_image"])
            d["opts"].tile_w, d["opts"].tile_h = tw, th

    def _jobs(self):
        jobs = []
        for d in self.views:
            for k in ("d_image", "leaf", "pos", "h", "img", "T", "nc", "ws_s", "ws_r"):
                assert d[k].is_contiguous()
            jobs.append(B.InpcViewJob(
                cam=api.camera(d["cam"]), opts=d["opts"].c(), view_id=d["view_id"], n_samples=self.n,
                leaf_idx=d["leaf"].data_ptr(), pos=d["pos"].data_ptr(), h=d["h"].data_ptr(),
                image=d["img"].data_ptr(), T_final=d["T"].data_ptr(), n_contrib=d["nc"].data_ptr(),
                d_image=d["d_image"].data_ptr(), sample_ws=d["ws_s"].data_ptr(), sample_ws_bytes=d["ws_s"].numel(),
                raster_ws=d["ws_r"].data_ptr(), raster_ws_bytes=d["ws_r"].numel()))
        return (B.InpcViewJob * len(jobs))(*jobs)

    def _enqueue(self):
        """All views through inpc_render_batch: the current stream is the
        origin, the batch's own streams carry the other views."""
        c, l, w, rs = self.tree
        main = torch.cuda.current_stream()
        self.grad_table.zero_()
        if self._job_array is None:
            self._job_array = self._jobs()
        tree = B.InpcOctree(c.data_ptr(), l.data_ptr(), w.data_ptr(), rs, l.shape[0])
        # torch hands out streams from a fixed pool, so a batch created after
        # many others may get one twice (or the current stream): pass each once
        streams = [main.cuda_stream]
        for st in self.streams:
            if st.cuda_stream not in streams:
                streams.append(st.cuda_stream)
        if self.persistent:
            B.inpc_render_batch_persistent(tree, self.seed, self.desc, self.table.data_ptr(), self._job_array,
                                           self.grad_table.data_ptr(), streams, self.front_ws.data_ptr(),
                                           self.front_ws.numel(), self.max_wait_us)
        else:
            B.inpc_render_batch(tree, self.seed, self.desc, self.table.data_ptr(), self._job_array,
                                self.grad_table.data_ptr(), streams)

    def run_eager(self):
        """One pass without the graph (also creates the library's side streams)."""
        self._enqueue()

    def capture(self):
        self.run_eager()
        torch.cuda.synchronize(self.dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._enqueue()
        torch.cuda.synchronize(self.dev)
        return self

    def step(self):
        """All views, forward and backward, as one graph launch."""
        if self.graph is None:
            self.capture()
        self.graph.replay()

    @property
    def n_views(self):
        return len(self.views)
