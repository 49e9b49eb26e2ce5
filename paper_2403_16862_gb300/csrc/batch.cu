// batch.cu -- inpc_render_batch: a batch of views of one scene, each the
// per-view sequence sample -> query -> rasterize (-> fused backward), spread
// over several streams that fork from and join back into the first one.
//
// The views share the octree, the grid table and the FP32 table gradient
// (atomic additions), so they are independent and their kernels overlap on
// the GPU: small views leave most SMs idle on their own.  The fork and the
// join are event dependencies, which a stream capture on streams[0] turns
// into graph edges, so the whole batch can be recorded once and replayed as
// one graph launch per step.
#include <vector>

#include "common.cuh"

using namespace inpc;

namespace {

// Events for one call: created here, destroyed when the call returns (a
// recorded event is released once the device has completed it, and a
// captured one has become a graph edge by then).
struct Events {
  std::vector<cudaEvent_t> ev;
  ~Events() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  inpc_status make(cudaEvent_t* out) {
    INPC_CUDA(cudaEventCreateWithFlags(out, cudaEventDisableTiming), "cudaEventCreateWithFlags");
    ev.push_back(*out);
    return INPC_OK;
  }
};

inpc_status run_raster(const inpc_hashgrid_desc* grid, const inpc_view_job& v, float* grad_table, inpc_stream_t s) {
  INPC_TRY(inpc_rasterize_fwd(&v.cam, &v.opts, v.pos, nullptr, v.h, v.n_samples, v.image, v.T_final, v.n_contrib,
                              v.raster_ws, v.raster_ws_bytes, s));
  if (v.d_image)
    INPC_TRY(inpc_rasterize_bwd_hashgrid(&v.cam, &v.opts, grid, v.pos, v.h, v.n_samples, v.T_final, v.n_contrib,
                                         v.d_image, grad_table, nullptr, v.raster_ws, v.raster_ws_bytes, s));
  return INPC_OK;
}

inpc_status run_view(const inpc_octree* tree, uint64_t seed, const inpc_hashgrid_desc* grid, const void* table,
                     const inpc_view_job& v, float* grad_table, inpc_stream_t s) {
  INPC_TRY(inpc_sample_octree(tree, seed, v.view_id, v.n_samples, v.leaf_idx, v.pos, nullptr, v.sample_ws,
                              v.sample_ws_bytes, s));
  INPC_TRY(inpc_query_hashgrid(grid, table, v.pos, v.n_samples, v.h, s));
  return run_raster(grid, v, grad_table, s);
}

inpc_status check_batch(const inpc_octree* tree, const inpc_hashgrid_desc* grid, const void* table,
                        const inpc_view_job* views, int32_t n_views, float* grad_table, const inpc_stream_t* streams,
                        int32_t n_streams) {
  if (!tree || !grid || !table || !streams) return fail(INPC_ERR_INVALID_ARG, "inpc_render_batch: null pointer");
  if (n_views < 0 || (n_views > 0 && !views)) return fail(INPC_ERR_INVALID_ARG, "inpc_render_batch: bad views");
  if (n_streams < 1) return fail(INPC_ERR_INVALID_ARG, "inpc_render_batch: n_streams must be >= 1");
  for (int32_t i = 0; i < n_streams; ++i)
    for (int32_t j = 0; j < i; ++j)
      if (streams[i] == streams[j]) return fail(INPC_ERR_INVALID_ARG, "inpc_render_batch: stream %d repeats", i);
  for (int32_t v = 0; v < n_views; ++v) {
    if (views[v].d_image && !grad_table)
      return fail(INPC_ERR_INVALID_ARG, "inpc_render_batch: view %d has d_image but grad_table is null", v);
    if (views[v].opts.opacity_mode != INPC_OPACITY_FROM_CH0 || views[v].opts.feat_dtype != grid->out_dtype)
      return fail(INPC_ERR_INVALID_ARG, "inpc_render_batch: view %d needs head mode and feat_dtype = the grid's out_dtype",
                  v);
  }
  return INPC_OK;
}

// Fork the views' work over the streams (round robin from streams[0]), run
// `each` for every view, join every stream back into streams[0].
template <class F>
inpc_status fork_join(int32_t n_views, const inpc_stream_t* streams, int32_t n_streams, F each) {
  const int32_t used = n_views < n_streams ? n_views : n_streams;
  cudaStream_t origin = reinterpret_cast<cudaStream_t>(streams[0]);
  Events E;
  // fork: every other stream waits for what was enqueued on streams[0]
  if (used > 1) {
    cudaEvent_t start;
    INPC_TRY(E.make(&start));
    INPC_CUDA(cudaEventRecord(start, origin), "cudaEventRecord(fork)");
    for (int32_t i = 1; i < used; ++i)
      INPC_CUDA(cudaStreamWaitEvent(reinterpret_cast<cudaStream_t>(streams[i]), start, 0), "cudaStreamWaitEvent(fork)");
  }
  inpc_status st = INPC_OK;
  for (int32_t v = 0; v < n_views && st == INPC_OK; ++v) st = each(v, streams[v % used]);
  // join every forked stream, also after an error, so that a capture on
  // streams[0] can still be ended; the first error (the views' own, else
  // the join's) is what the call returns
  for (int32_t i = 1; i < used; ++i) {
    cudaEvent_t done = nullptr;
    const inpc_status mk = E.make(&done);
    cudaError_t e = cudaSuccess;
    if (mk == INPC_OK) {
      e = cudaEventRecord(done, reinterpret_cast<cudaStream_t>(streams[i]));
      if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, done, 0);
    }
    if (st == INPC_OK && mk != INPC_OK) st = mk;
    if (st == INPC_OK && e != cudaSuccess) st = fail(INPC_ERR_CUDA, "inpc_render_batch join: %s", cudaGetErrorString(e));
  }
  return st;
}

}  // namespace

extern "C" inpc_status inpc_render_batch(const inpc_octree* tree, uint64_t seed, const inpc_hashgrid_desc* grid,
                                         const void* table, const inpc_view_job* views, int32_t n_views,
                                         float* grad_table, const inpc_stream_t* streams, int32_t n_streams) {
  inpc::fault_arg(table);
  INPC_TRY(check_batch(tree, grid, table, views, n_views, grad_table, streams, n_streams));
  if (n_views == 0) return INPC_OK;
  return fork_join(n_views, streams, n_streams, [&](int32_t v, inpc_stream_t s) {
    return run_view(tree, seed, grid, table, views[v], grad_table, s);
  });
}

extern "C" inpc_status inpc_render_batch_persistent(const inpc_octree* tree, uint64_t seed,
                                                    const inpc_hashgrid_desc* grid, const void* table,
                                                    const inpc_view_job* views, int32_t n_views, float* grad_table,
                                                    const inpc_stream_t* streams, int32_t n_streams,
                                                    void* front_workspace, size_t front_workspace_bytes,
                                                    int64_t max_wait_us) {
  inpc::fault_arg(table);
  INPC_TRY(check_batch(tree, grid, table, views, n_views, grad_table, streams, n_streams));
  if (n_views == 0) return INPC_OK;
  // the sampling and query of every view: persistent launches of up to
  // kBatchFrontViews views each, one after another on streams[0]
  constexpr int32_t kBatchFrontViews = 64;
  for (int32_t v0 = 0; v0 < n_views; v0 += kBatchFrontViews) {
    const int32_t nv = n_views - v0 < kBatchFrontViews ? n_views - v0 : kBatchFrontViews;
    inpc_front_view fv[kBatchFrontViews];
    for (int32_t i = 0; i < nv; ++i) {
      const inpc_view_job& j = views[v0 + i];
      fv[i] = inpc_front_view{j.view_id, j.n_samples, j.leaf_idx, j.pos, j.h};
    }
    INPC_TRY(inpc_sample_query_batch(tree, seed, grid, table, fv, nv, max_wait_us, front_workspace,
                                     front_workspace_bytes, streams[0]));
  }
  return fork_join(n_views, streams, n_streams, [&](int32_t v, inpc_stream_t s) {
    return run_raster(grid, views[v], grad_table, s);
  });
}
