// raster_bwd.cu -- C ABI of the rasterizer backward (App. A.6).
#include "hashgrid_impl.cuh"
#include "raster_impl.cuh"

namespace inpc {
namespace {

// Per point, one lane per grid level (its 4 features): the point's gradient
// row, gathered as in k_point_grad, then that level's eight corner
// contributions to the table gradient straight from registers (the adjoint
// of the query, as in k_hash_bwd), so the row never goes through memory.
// Coarse levels have few rows and receive millions of additions each, which
// serialise on the same L2 addresses.  Their contributions go to one of
// kReplicas copies (chosen by CTA) and k_fold_replicas sums the copies into
// the table gradient afterwards.
constexpr int kReplicas = 16;
constexpr int64_t kReplicaMaxRows = 1 << 17;  // levels up to this many rows are replicated

struct Replicas {
  int n_levels;      // leading levels that are replicated
  long long rows;    // table rows they span (level-aligned)
  float* base;       // [kReplicas][rows][4]
};

inline Replicas replica_plan(const GridParams& Gp, void* base) {
  Replicas r;
  r.n_levels = 0;
  while (r.n_levels < Gp.n_levels && r.n_levels + 1 < kMaxLevels &&
         (Gp.offset[r.n_levels + 1] - Gp.offset[r.n_levels]) <= kReplicaMaxRows)
    ++r.n_levels;
  r.rows = r.n_levels > 0 ? Gp.offset[r.n_levels] : 0;
  r.base = static_cast<float*>(base);
  return r;
}

inline size_t replica_bytes(const Replicas& r) { return (size_t)kReplicas * r.rows * 4 * sizeof(float); }

// Sum the replicas into the table gradient.  The add is atomic, so calls
// for several views may accumulate into one table concurrently.
__global__ void k_fold_replicas(const float4* __restrict__ rep, long long rows, float* __restrict__ grad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows; i += (long long)gridDim.x * blockDim.x) {
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kReplicas; ++k) {
      const float4 v = rep[k * rows + i];
      s.x += v.x;
      s.y += v.y;
      s.z += v.z;
      s.w += v.w;
    }
    if (s.x != 0.f || s.y != 0.f || s.z != 0.f || s.w != 0.f) red_add_v4(grad + 4 * i, s);
  }
}

template <int GA, class FT>
__global__ void __launch_bounds__(kThreads) k_point_grad_hash(RP P, GridParams Gp, const float* __restrict__ pos,
                                                               const FT* __restrict__ feat,
                                                               const float* __restrict__ d_image, RasterWs ws,
                                                               float* __restrict__ grad_table,
                                                               float* __restrict__ d_feat, Replicas rep) {
  constexpr int kGroups = kThreads / GA;
  const Group<GA> G;
  const int l = G.lg;
  const int ch = 4 * l;
  const bool active = l < Gp.n_levels;
  const long long g0 = (long long)blockIdx.x * kGroups + threadIdx.x / GA;
  const uint64_t keep = l2_evict_last(), stream = l2_evict_first();
  for (long long id = g0; id < P.n; id += (long long)gridDim.x * kGroups) {
    const uint4 sl = ld_hint_u4(reinterpret_cast<const uint4*>(ws.pslot) + id, stream);
    const uint32_t slots[4] = {sl.x, sl.y, sl.z, sl.w};
    float dc[4] = {0.f, 0.f, 0.f, 0.f};
    if ((sl.x & sl.y & sl.z & sl.w) != kNoSlot) {
      Splat s;
      splat_point(P, pos, id, s);
      float e_h0 = 0.f;
      const float ah = point_alpha_h(P, nullptr, feat, id, &e_h0);
      float2 sc[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) sc[k] = slots[k] == kNoSlot ? make_float2(0.f, 0.f) : ld_hint_f2(ws.fscal + slots[k], stream);
      float dah = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (slots[k] == kNoSlot) continue;
        const float w = corner_weight(s.f, k & 1, k >> 1);
        if (__fmul_rn(ah, w) <= P.alpha_max) dah = __fmaf_rn(w, sc[k].y, dah);
        if (active) {
          const long long pix = (long long)(s.f.j0 + (k >> 1)) * P.cam.W + (s.f.i0 + (k & 1));
          const float4 g = __ldg(reinterpret_cast<const float4*>(d_image + pix * P.F + ch));
          dc[0] = __fmaf_rn(sc[k].x, g.x, dc[0]);
          dc[1] = __fmaf_rn(sc[k].x, g.y, dc[1]);
          dc[2] = __fmaf_rn(sc[k].x, g.z, dc[2]);
          dc[3] = __fmaf_rn(sc[k].x, g.w, dc[3]);
        }
      }
      // channel 0 of the blended color is the constant 1; the opacity
      // gradient reaches h0 through alpha_h = 1 - exp(-exp(h0))
      if (l == 0) dc[0] = dah * (e_h0 * expf(-e_h0));
    }
    if (!active) continue;
    if (d_feat) *reinterpret_cast<float4*>(d_feat + id * P.F + ch) = make_float4(dc[0], dc[1], dc[2], dc[3]);
    if (dc[0] == 0.f && dc[1] == 0.f && dc[2] == 0.f && dc[3] == 0.f) continue;
    uint32_t cx, cy, cz;
    float gx[2], gy[2], gz[2];
    const int N = Gp.res[l];
    cell_frac(__ldg(pos + 3 * id + 0), N, cx, gx[0], gx[1]);
    cell_frac(__ldg(pos + 3 * id + 1), N, cy, gy[0], gy[1]);
    cell_frac(__ldg(pos + 3 * id + 2), N, cz, gz[0], gz[1]);
    float* gl = l < rep.n_levels
                    ? rep.base + 4 * ((long long)(blockIdx.x % kReplicas) * rep.rows + Gp.offset[l])
                    : grad_table + 4 * Gp.offset[l];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
      const float w = gx[bx] * gy[by] * gz[bz];
      const uint32_t row = vertex_row(Gp, l, cx + bx, cy + by, cz + bz);
      red_add_v4(gl + 4ull * row, make_float4(w * dc[0], w * dc[1], w * dc[2], w * dc[3]), keep);
    }
  }
}

template <int GA, class FT>
inpc_status launch_point_grad_hash(const RP& P, const GridParams& Gp, const float* pos, const FT* feat,
                                   const float* d_image, const RasterWs& ws, float* grad_table, float* d_feat,
                                   const Replicas& rep, cudaStream_t s) {
  constexpr int kGroups = kThreads / GA;
  if (rep.rows > 0) INPC_CUDA(cudaMemsetAsync(rep.base, 0, replica_bytes(rep), s), "clear replicas");
  const long long grid = std::min<long long>(ceil_div(P.n, kGroups), (long long)device_sm_count() * 32);
  INPC_TIMED("k_point_grad_hash", s,
             k_point_grad_hash<GA, FT><<<(unsigned)std::max<long long>(grid, 1), kThreads, 0, s>>>(
                 P, Gp, pos, feat, d_image, ws, grad_table, d_feat, rep));
  INPC_TRY(check_launch("k_point_grad_hash"));
  if (rep.rows > 0) {
    INPC_TIMED("k_fold_replicas", s,
               k_fold_replicas<<<(unsigned)std::min<long long>(ceil_div(rep.rows, 256), device_sm_count() * 8), 256,
                                 0, s>>>(reinterpret_cast<const float4*>(rep.base), rep.rows, grad_table));
    INPC_TRY(check_launch("k_fold_replicas"));
  }
  return INPC_OK;
}

}  // namespace
}  // namespace inpc

using namespace inpc;

extern "C" inpc_status inpc_rasterize_bwd(const inpc_camera* cam, const inpc_raster_opts* opts, const float* pos,
                                          const float* opacity, const void* feat, int64_t n, const float* T_final,
                                          const int32_t* n_contrib, const float* d_image, float* d_opacity,
                                          float* d_feat, void* workspace, size_t workspace_bytes,
                                          inpc_stream_t stream) {
  RP P;
  INPC_TRY(make_rp(cam, opts, n, P));
  const RasterWs need = carve(nullptr, P.n_pix, n);
  if (!workspace || workspace_bytes < need.bytes || !aligned(workspace, 256))
    return fail(INPC_ERR_INVALID_ARG, "workspace null, unaligned or smaller than %zu bytes", need.bytes);
  if (n == 0) return INPC_OK;
  if (!pos || !feat || !T_final || !n_contrib || !d_image || !d_feat)
    return fail(INPC_ERR_INVALID_ARG, "null pointer");
  if (!P.head && (!opacity || !d_opacity)) return fail(INPC_ERR_INVALID_ARG, "opacity and d_opacity required");
  const size_t va = P.F % 4 == 0 ? 16 : 4;
  const size_t vf = P.F % 4 == 0 ? (P.bf16 && P.F != 64 ? 8 : 16) : (P.bf16 ? 2 : 4);
  if (!aligned(feat, vf) || !aligned(d_image, va) || !aligned(d_feat, va))
    return fail(INPC_ERR_INVALID_ARG, "feat/d_image/d_feat misaligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RasterWs ws = carve(workspace, P.n_pix, n);
  return dispatch(P.F, [&](auto Vc, auto Gc) {
    constexpr int V = decltype(Vc)::value, GA = decltype(Gc)::value;
    if constexpr (GA != 32) {
      if (P.bf16) return fail(INPC_ERR_UNSUPPORTED, "BF16 features need n_channels = 32, 64 or 128");
    } else if (P.bf16)
      return launch_bwd<V, GA, __nv_bfloat16>(P, pos, opacity, static_cast<const __nv_bfloat16*>(feat), n_contrib,
                                              d_image, ws, P.head ? nullptr : d_opacity, d_feat, s);
    return launch_bwd<V, GA, float>(P, pos, opacity, static_cast<const float*>(feat), n_contrib, d_image, ws,
                                    P.head ? nullptr : d_opacity, d_feat, s);
  });
}

extern "C" inpc_status inpc_rasterize_bwd_hashgrid(const inpc_camera* cam, const inpc_raster_opts* opts,
                                                   const inpc_hashgrid_desc* grid, const float* pos, const void* feat,
                                                   int64_t n, const float* T_final, const int32_t* n_contrib,
                                                   const float* d_image, float* grad_table, float* d_feat,
                                                   void* workspace, size_t workspace_bytes, inpc_stream_t stream) {
  RP P;
  INPC_TRY(make_rp(cam, opts, n, P));
  GridParams Gp;
  int64_t n_entries = 0;
  INPC_TRY(make_params(grid, Gp, &n_entries));
  if (!P.head) return fail(INPC_ERR_UNSUPPORTED, "inpc_rasterize_bwd_hashgrid needs INPC_OPACITY_FROM_CH0");
  if (P.F != 4 * Gp.n_levels)
    return fail(INPC_ERR_INVALID_ARG, "n_channels (%d) must equal n_levels * n_feats (%d)", P.F, 4 * Gp.n_levels);
  const RasterWs need = carve(nullptr, P.n_pix, n);
  const Replicas rep_need = replica_plan(Gp, nullptr);
  const size_t total = need.bytes + replica_bytes(rep_need);
  if (!workspace || workspace_bytes < total || !aligned(workspace, 256))
    return fail(INPC_ERR_INVALID_ARG,
                "workspace null, unaligned or smaller than %zu bytes (inpc_rasterize_bwd_hashgrid_workspace_size)",
                total);
  if (n == 0) return INPC_OK;
  if (!pos || !feat || !T_final || !n_contrib || !d_image || !grad_table)
    return fail(INPC_ERR_INVALID_ARG, "null pointer");
  const size_t vf = P.bf16 && P.F != 64 ? 8 : 16;
  if (!aligned(feat, vf) || !aligned(d_image, 16) || !aligned(grad_table, 16) || (d_feat && !aligned(d_feat, 16)))
    return fail(INPC_ERR_INVALID_ARG, "feat/d_image/grad_table/d_feat misaligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RasterWs ws = carve(workspace, P.n_pix, n);
  const Replicas rep = replica_plan(Gp, static_cast<char*>(workspace) + need.bytes);
  return dispatch(P.F, [&](auto Vc, auto Gc) -> inpc_status {
    constexpr int V = decltype(Vc)::value, GA = decltype(Gc)::value;
    auto run = [&](auto ftag) -> inpc_status {
      using FT = decltype(ftag);
      const FT* f = static_cast<const FT*>(feat);
      INPC_TRY((launch_blend_bwd<V, GA, FT>(P, f, n_contrib, d_image, ws, s)));
      if (Gp.n_levels <= 8)
        return launch_point_grad_hash<8, FT>(P, Gp, pos, f, d_image, ws, grad_table, d_feat, rep, s);
      if (Gp.n_levels <= 16)
        return launch_point_grad_hash<16, FT>(P, Gp, pos, f, d_image, ws, grad_table, d_feat, rep, s);
      return launch_point_grad_hash<32, FT>(P, Gp, pos, f, d_image, ws, grad_table, d_feat, rep, s);
    };
    if constexpr (GA != 32) {
      if (P.bf16) return fail(INPC_ERR_UNSUPPORTED, "BF16 features need n_channels = 32, 64 or 128");
      return run(float());
    } else {
      if (P.bf16) return run(__nv_bfloat16());
      return run(float());
    }
  });
}

extern "C" inpc_status inpc_rasterize_bwd_hashgrid_workspace_size(const inpc_camera* cam, const inpc_raster_opts* opts,
                                                                  const inpc_hashgrid_desc* grid, int64_t n,
                                                                  size_t* bytes) {
  if (!bytes) return fail(INPC_ERR_INVALID_ARG, "bytes is null");
  RP P;
  INPC_TRY(make_rp(cam, opts, n, P));
  GridParams Gp;
  int64_t n_entries = 0;
  INPC_TRY(make_params(grid, Gp, &n_entries));
  *bytes = carve(nullptr, P.n_pix, n).bytes + replica_bytes(replica_plan(Gp, nullptr));
  return INPC_OK;
}
