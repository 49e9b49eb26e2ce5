// octree.cu -- maintenance of the point-probability octree (Sec. 3.1:
// "Probability Updates" Eq. 2 / Eq. 3, "Subdivision", "Pruning"; App. A.4
// leaf layout) and the per-point blending weights it consumes (App. A.6).
//
// Blending weights: after a forward, every pixel's blended prefix (recorded
// by the forward in blending order) is walked once more with the forward's
// own product scan, so T_k alpha_k is bitwise the forward's; each splat's
// value lands at its bucket slot and a per-point pass combines a point's
// four splats with their bilinear weights.
//
// Updates: per-leaf max and min of the weights of the points drawn from the
// leaf (as FP32 bit patterns: non-negative floats order like their bits)
// with a warp-level reduction over runs of equal leaves first (the sampler
// emits points grouped by leaf), then one FP64 update per leaf.
//
// Subdivision and pruning: an exclusive scan of the per-leaf output counts
// (8 or 1; 1 or 0) gives every surviving leaf its place, so children
// replace their parent in place and the order of the list is kept.
#include "raster_impl.cuh"

namespace inpc {
namespace {

// ------------------------------------------------------ blending weights ---
__global__ void __launch_bounds__(256) k_pixel_splat_weights(RP P, const int32_t* __restrict__ n_contrib,
                                                            RasterWs ws) {
  const Group<32> G;
  const long long n_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < P.n_pix; q += n_warps) {
    const uint32_t s0 = ws.pix_start[q];
    const int m = (int)(ws.pix_start[q + 1] - s0);
    const int nb = m > 0 ? blended_count(n_contrib, q, m) : 0;
    float T = 1.0f;
    for (int b = 0; b < nb; b += 32) {
      const bool valid = b + G.lg < nb;
      uint32_t slot = 0;
      float a = 0.f;
      if (valid) {
        const uint2 o = order_at(P, ws, s0, m, b + G.lg);
        slot = o.x;
        a = ws.alpha[s0 + o.x];
      }
      const ChunkT<32> ct = chunk_transmittance<32>(G, P, a, valid, min(32, nb - b), T);
      if (G.lg < ct.take) reinterpret_cast<float*>(ws.fscal + s0 + slot)[0] = __fmul_rn(ct.Tk, a);
      T = G.bcast(ct.Tn, ct.take - 1);
      if (ct.stop) break;
    }
  }
}

__global__ void __launch_bounds__(256) k_point_blend_weights(RP P, const float* __restrict__ pos, RasterWs ws,
                                                            float* __restrict__ b_out) {
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < P.n;
       id += (long long)gridDim.x * blockDim.x) {
    const uint4 sl = __ldg(reinterpret_cast<const uint4*>(ws.pslot) + id);
    const uint32_t slots[4] = {sl.x, sl.y, sl.z, sl.w};
    float b = 0.f;
    if ((sl.x & sl.y & sl.z & sl.w) != kNoSlot) {
      Splat s;
      splat_point(P, pos, id, s);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (slots[k] != kNoSlot) b = __fmaf_rn(corner_weight(s.f, k & 1, k >> 1), ws.fscal[slots[k]].x, b);
    }
    b_out[id] = b;
  }
}

// --------------------------------------------------------------- updates ---
constexpr uint32_t kNoPoint = 0xFFFFFFFFu;  // min sentinel: above every non-negative float's bits

struct UpdateWs {
  uint32_t* status;
  uint32_t* bmax;  // [L] FP32 bits
  uint32_t* bmin;  // [L] FP32 bits, kNoPoint when no point was drawn from the leaf
  size_t bytes;
};

UpdateWs carve_update(void* base, int64_t L) {
  Carver c(base);
  UpdateWs w;
  w.status = static_cast<uint32_t*>(base);
  w.bmax = c.take<uint32_t>(std::max<int64_t>(L, 1));
  w.bmin = c.take<uint32_t>(std::max<int64_t>(L, 1));
  w.bytes = c.bytes();
  return w;
}

__global__ void __launch_bounds__(256) k_leaf_minmax(const int32_t* __restrict__ leaf_idx,
                                                    const float* __restrict__ b, long long n, long long L,
                                                    UpdateWs ws) {
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // the trip count is uniform per warp, so every lane takes part in the shuffles
  for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const long long id = base + lane;
    int leaf = -1;
    uint32_t bits = 0;
    if (id < n) {
      leaf = leaf_idx[id];
      const float v = b[id];
      bits = __float_as_uint(v);
      if (!(v >= 0.0f) || (bits & 0x80000000u)) {  // negative, -0 or NaN: counted as 0
        if (!(v == 0.0f)) raise_status(ws.status, INPC_DEV_BAD_BLEND_WEIGHT);
        bits = 0;
      }
      if (leaf < 0 || (long long)leaf >= L) {
        raise_status(ws.status, INPC_DEV_BAD_LEAF);
        leaf = -1;
      }
    }
    uint32_t mx = bits, mn = bits;
    // runs of equal leaves: lane i ends with the max / min over its run from i on
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ol = __shfl_down_sync(0xffffffffu, leaf, o);
      const uint32_t omx = __shfl_down_sync(0xffffffffu, mx, o);
      const uint32_t omn = __shfl_down_sync(0xffffffffu, mn, o);
      if (lane + o < 32 && ol == leaf) {
        mx = max(mx, omx);
        mn = min(mn, omn);
      }
    }
    const int prev = __shfl_up_sync(0xffffffffu, leaf, 1);
    if (leaf >= 0 && (lane == 0 || prev != leaf)) {
      atomicMax(ws.bmax + leaf, mx);
      atomicMin(ws.bmin + leaf, mn);
    }
  }
}

__global__ void k_leaf_update(double* __restrict__ p, double* __restrict__ q, long long L, double lambda_u,
                              UpdateWs ws) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L; i += (long long)gridDim.x * blockDim.x) {
    const double dp = __dmul_rn(lambda_u, p[i]), dq = __dmul_rn(lambda_u, q[i]);
    if (ws.bmin[i] == kNoPoint) {  // no point drawn from the leaf: decay only
      p[i] = dp;
      q[i] = dq;
    } else {
      const double mx = (double)__uint_as_float(ws.bmax[i]), mn = (double)__uint_as_float(ws.bmin[i]);
      const double spread = __dsub_rn(mx, mn);
      p[i] = mx > dp ? mx : dp;
      q[i] = spread > dq ? spread : dq;
    }
  }
}

// ---------------------------------------------------- subdivide / prune ---
struct RefineWs {
  uint32_t* offset;  // [L] exclusive scan of the output counts
  uint32_t* tops;    // scan block totals; grand total at the end
  size_t bytes;
};

RefineWs carve_refine(void* base, int64_t L) {
  Carver c(base);
  RefineWs w;
  w.offset = c.take<uint32_t>(std::max<int64_t>(L, 1));
  w.tops = c.take<uint32_t>(scan::n_tops(std::max<int64_t>(L, 1)));
  w.bytes = c.bytes();
  return w;
}

struct SplitCount {
  const double* q;
  double tau;
  __device__ uint32_t operator()(int64_t i) const { return q[i] > tau ? 8u : 1u; }
};

struct KeepCount {
  const double* p;
  double tau;
  __device__ uint32_t operator()(int64_t i) const { return p[i] < tau ? 0u : 1u; }
};

struct LeafOut {
  float* centers;
  int32_t* levels;
  double* p;
  double* q;
};

__device__ __forceinline__ void copy_leaf(const inpc_octree& t, const double* __restrict__ q, int64_t i, LeafOut out,
                                          int64_t o) {
  out.centers[3 * o + 0] = t.centers[3 * i + 0];
  out.centers[3 * o + 1] = t.centers[3 * i + 1];
  out.centers[3 * o + 2] = t.centers[3 * i + 2];
  out.levels[o] = t.levels[i];
  out.p[o] = t.weights[i];
  out.q[o] = q[i];
}

// split = 0: copy every leaf to its place (the leaf cap was reached).
__global__ void k_subdivide(inpc_octree t, const double* __restrict__ q, double tau, int split,
                            const uint32_t* __restrict__ offset, LeafOut out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < t.n_leaves;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!split) {
      copy_leaf(t, q, i, out, i);
      continue;
    }
    const int64_t o = offset[i];
    if (!(q[i] > tau)) {
      copy_leaf(t, q, i, out, o);
      continue;
    }
    const int l = t.levels[i];
    const double child = __dmul_rn((double)t.root_size, ldexp(1.0, -(l + 1)));  // child edge
    for (int k = 0; k < 8; ++k) {
      const int d[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
#pragma unroll
      for (int a = 0; a < 3; ++a)
        out.centers[3 * (o + k) + a] =
            (float)__dadd_rn((double)t.centers[3 * i + a], __dmul_rn((double)d[a] - 0.5, child));
      out.levels[o + k] = l + 1;
      out.p[o + k] = t.weights[i];
      out.q[o + k] = 0.0;
    }
  }
}

__global__ void k_prune(inpc_octree t, const double* __restrict__ q, double tau, const uint32_t* __restrict__ offset,
                        LeafOut out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < t.n_leaves;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!(t.weights[i] < tau)) copy_leaf(t, q, i, out, offset[i]);
}

inpc_status check_tree(const inpc_octree* t, const double* q) {
  if (!t || !t->centers || !t->levels || !t->weights || !q) return fail(INPC_ERR_INVALID_ARG, "null octree array");
  if (t->n_leaves < 1 || t->n_leaves > (int64_t(1) << 24))
    return fail(INPC_ERR_INVALID_ARG, "n_leaves must be in [1, 2^24]");
  if (!(t->root_size > 0.0f)) return fail(INPC_ERR_INVALID_ARG, "root_size must be positive");
  return INPC_OK;
}

inpc_status check_out(const LeafOut& o) {
  if (!o.centers || !o.levels || !o.p || !o.q) return fail(INPC_ERR_INVALID_ARG, "null output array");
  return INPC_OK;
}

unsigned grid_1d(int64_t n, int per_sm = 8) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)device_sm_count() * per_sm));
}

// Scan of the per-leaf output counts; returns the total on the host (the
// stream is synchronised).
template <class Load>
inpc_status count_outputs(Load ld, int64_t L, const RefineWs& ws, cudaStream_t s, int64_t* total) {
  INPC_TRY((scan::run<uint32_t, Load, false>(ld, L, ws.offset, ws.tops, s)));
  uint32_t t = 0;
  INPC_CUDA(cudaMemcpyAsync(&t, ws.tops + ceil_div(L, scan::kBlock), sizeof(t), cudaMemcpyDeviceToHost, s),
            "read output count");
  INPC_CUDA(cudaStreamSynchronize(s), "output count sync");
  *total = t;
  return INPC_OK;
}

}  // namespace
}  // namespace inpc

using namespace inpc;

extern "C" inpc_status inpc_rasterize_point_weights(const inpc_camera* cam, const inpc_raster_opts* opts,
                                                    const float* pos, int64_t n, const int32_t* n_contrib,
                                                    float* b_out, void* workspace, size_t workspace_bytes,
                                                    inpc_stream_t stream) {
  inpc::fault_arg(pos);
  RP P;
  INPC_TRY(make_rp(cam, opts, n, P));
  const RasterWs need = carve(nullptr, P.n_pix, n);
  if (!workspace || workspace_bytes < need.bytes || !aligned(workspace, 256))
    return fail(INPC_ERR_INVALID_ARG, "workspace null, unaligned or smaller than %zu bytes", need.bytes);
  if (n == 0) return INPC_OK;
  if (!pos || !n_contrib || !b_out) return fail(INPC_ERR_INVALID_ARG, "null pointer");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RasterWs ws = carve(workspace, P.n_pix, n);
  INPC_CUDA(cudaMemsetAsync(ws.fscal, 0, sizeof(float2) * std::max<long long>(4 * n, 1), s), "clear splat weights");
  INPC_TIMED("k_pixel_splat_weights", s,
             k_pixel_splat_weights<<<(unsigned)std::min<long long>(ceil_div(P.n_pix * 32, 256),
                                                                    (long long)device_sm_count() * 16),
                                     256, 0, s>>>(P, n_contrib, ws));
  INPC_TRY(check_launch("k_pixel_splat_weights"));
  INPC_TIMED("k_point_blend_weights", s,
             k_point_blend_weights<<<grid_1d(n, 16), 256, 0, s>>>(P, pos, ws, b_out));
  return check_launch("k_point_blend_weights");
}

extern "C" inpc_status inpc_octree_update_workspace_size(int64_t n_leaves, size_t* bytes) {
  if (inpc::fault_workspace_overflow())
    return inpc::fail(INPC_ERR_CAPACITY, "inpc_octree_update_workspace_size: size overflow (injected fault)");
  if (!bytes) return fail(INPC_ERR_INVALID_ARG, "bytes is null");
  if (n_leaves < 1 || n_leaves > (int64_t(1) << 24)) return fail(INPC_ERR_INVALID_ARG, "n_leaves must be in [1, 2^24]");
  *bytes = carve_update(nullptr, n_leaves).bytes;
  return INPC_OK;
}

extern "C" inpc_status inpc_octree_update(const int32_t* leaf_idx, const float* b, int64_t n, double* p, double* q,
                                          int64_t n_leaves, double lambda_u, void* workspace,
                                          size_t workspace_bytes, inpc_stream_t stream) {
  inpc::fault_arg(leaf_idx);
  if (n_leaves < 1 || n_leaves > (int64_t(1) << 24)) return fail(INPC_ERR_INVALID_ARG, "n_leaves must be in [1, 2^24]");
  if (n < 0 || n > INT32_MAX) return fail(INPC_ERR_CAPACITY, "n must be in [0, 2^31 - 1]");
  if (!p || !q || (n > 0 && (!leaf_idx || !b))) return fail(INPC_ERR_INVALID_ARG, "null pointer");
  if (!(lambda_u >= 0.0 && lambda_u <= 1.0)) return fail(INPC_ERR_INVALID_ARG, "lambda_u must be in [0, 1]");
  const UpdateWs need = carve_update(nullptr, n_leaves);
  if (!workspace || workspace_bytes < need.bytes || !aligned(workspace, 256))
    return fail(INPC_ERR_INVALID_ARG, "workspace null, unaligned or smaller than %zu bytes", need.bytes);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  UpdateWs ws = carve_update(workspace, n_leaves);
  INPC_CUDA(cudaMemsetAsync(workspace, 0, kHeaderBytes, s), "clear header");
  INPC_CUDA(cudaMemsetAsync(ws.bmax, 0, sizeof(uint32_t) * n_leaves, s), "clear max");
  INPC_CUDA(cudaMemsetAsync(ws.bmin, 0xFF, sizeof(uint32_t) * n_leaves, s), "clear min");
  if (n > 0) {
    INPC_TIMED("k_leaf_minmax", s, k_leaf_minmax<<<grid_1d(n, 16), 256, 0, s>>>(leaf_idx, b, n, n_leaves, ws));
    INPC_TRY(check_launch("k_leaf_minmax"));
  }
  INPC_TIMED("k_leaf_update", s, k_leaf_update<<<grid_1d(n_leaves), 256, 0, s>>>(p, q, n_leaves, lambda_u, ws));
  return check_launch("k_leaf_update");
}

extern "C" inpc_status inpc_octree_refine_workspace_size(int64_t n_leaves, size_t* bytes) {
  if (inpc::fault_workspace_overflow())
    return inpc::fail(INPC_ERR_CAPACITY, "inpc_octree_refine_workspace_size: size overflow (injected fault)");
  if (!bytes) return fail(INPC_ERR_INVALID_ARG, "bytes is null");
  if (n_leaves < 1 || n_leaves > (int64_t(1) << 24)) return fail(INPC_ERR_INVALID_ARG, "n_leaves must be in [1, 2^24]");
  *bytes = carve_refine(nullptr, n_leaves).bytes;
  return INPC_OK;
}

extern "C" inpc_status inpc_octree_subdivide(const inpc_octree* tree, const double* q, double tau_s,
                                             int64_t max_leaves, float* centers_out, int32_t* levels_out,
                                             double* p_out, double* q_out, int64_t out_capacity, int64_t* n_out,
                                             void* workspace, size_t workspace_bytes, inpc_stream_t stream) {
  inpc::fault_arg(tree);
  INPC_TRY(check_tree(tree, q));
  const LeafOut out{centers_out, levels_out, p_out, q_out};
  INPC_TRY(check_out(out));
  if (!n_out) return fail(INPC_ERR_INVALID_ARG, "n_out is null");
  const int64_t L = tree->n_leaves;
  const RefineWs need = carve_refine(nullptr, L);
  if (!workspace || workspace_bytes < need.bytes || !aligned(workspace, 256))
    return fail(INPC_ERR_INVALID_ARG, "workspace null, unaligned or smaller than %zu bytes", need.bytes);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const RefineWs ws = carve_refine(workspace, L);
  int64_t total = 0;
  INPC_TRY(count_outputs(SplitCount{q, tau_s}, L, ws, s, &total));
  const int split = total < max_leaves ? 1 : 0;
  const int64_t n_new = split ? total : L;
  if (n_new > out_capacity)
    return fail(INPC_ERR_CAPACITY, "subdivision yields %lld leaves, output capacity is %lld", (long long)n_new,
                (long long)out_capacity);
  INPC_TIMED("k_subdivide", s, k_subdivide<<<grid_1d(L), 256, 0, s>>>(*tree, q, tau_s, split, ws.offset, out));
  INPC_TRY(check_launch("k_subdivide"));
  *n_out = n_new;
  return INPC_OK;
}

extern "C" inpc_status inpc_octree_prune(const inpc_octree* tree, const double* q, double tau_p, float* centers_out,
                                         int32_t* levels_out, double* p_out, double* q_out, int64_t out_capacity,
                                         int64_t* n_out, void* workspace, size_t workspace_bytes,
                                         inpc_stream_t stream) {
  inpc::fault_arg(tree);
  INPC_TRY(check_tree(tree, q));
  const LeafOut out{centers_out, levels_out, p_out, q_out};
  INPC_TRY(check_out(out));
  if (!n_out) return fail(INPC_ERR_INVALID_ARG, "n_out is null");
  const int64_t L = tree->n_leaves;
  const RefineWs need = carve_refine(nullptr, L);
  if (!workspace || workspace_bytes < need.bytes || !aligned(workspace, 256))
    return fail(INPC_ERR_INVALID_ARG, "workspace null, unaligned or smaller than %zu bytes", need.bytes);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const RefineWs ws = carve_refine(workspace, L);
  int64_t total = 0;
  INPC_TRY(count_outputs(KeepCount{tree->weights, tau_p}, L, ws, s, &total));
  if (total > out_capacity)
    return fail(INPC_ERR_CAPACITY, "pruning keeps %lld leaves, output capacity is %lld", (long long)total,
                (long long)out_capacity);
  INPC_TIMED("k_prune", s, k_prune<<<grid_1d(L), 256, 0, s>>>(*tree, q, tau_p, ws.offset, out));
  INPC_TRY(check_launch("k_prune"));
  *n_out = total;
  return INPC_OK;
}
