// raster_bwd.cu -- C ABI of the rasterizer backward (App. A.6).
#include "hashgrid_impl.cuh"
#include "raster_impl.cuh"

namespace inpc {
namespace {

// Per point and grid level (its 4 features), two lanes: the point's gradient
// row for that level, gathered as in k_point_grad, then the level's corner
// contributions to the table gradient straight from registers (the adjoint
// of the query, as in k_hash_bwd), so the row never goes through memory.
// The two lanes own the cell's two x vertices, so each issues four of the
// eight corner reductions, and a pair's two reductions (x and x + 1 with
// the same y, z: rows differing in their low bits) usually share a 128-byte
// line, one L1 wavefront.  Values that depend on the point only (fragment
// scalars, footprint, position, the h0 term) are formed once per point, one
// lane per point, into shared-memory records that the level lanes read.
//
// The levels are split in halves over a pair of warps that share the same
// points: the even warp takes the coarse half, the odd warp the fine half.
// Each point slot of a CTA walks a run of points a few apart.  Points come
// grouped by octree leaf with the leaves in Morton order, so at the coarse
// levels such points fall in the same or a neighbouring cell, and a coarse
// lane keeps one float4 accumulator per cell corner (in shared memory),
// sending a corner's sum to memory only when the next point needs a
// different vertex in that slot.  The slot of vertex (X, Y, Z) is given by
// the parities of X, Y and Z: every cell has exactly one corner of each
// parity class, and a step of one cell along an axis keeps the four shared
// vertices in their slots, so neighbouring cells share accumulators as well.
// Coarse levels have few rows that would otherwise receive millions of
// additions each.  Fine levels change vertex at almost every point and
// reduce directly.
// A point's values shared by its level lanes.
struct __align__(16) PointRec {
  int pix0;        // pixel of footprint corner 0 (j0 W + i0)
  uint32_t mask;   // bit k: corner k's fragment has T_k alpha_k != 0
  float h0term;    // level-0 channel-0 gradient: the opacity path into h0
  float x;
  float4 sc;       // T_k alpha_k of the four fragments (0 without one)
  float y, z, pad0, pad1;
};

// The named barrier of warp pair `pair` (id 1 + pair, the pair's 64
// threads).  The warp first reconverges (a level loop may end early for
// half of its lanes at the end of a chunk), then meets the other warp.
__device__ __forceinline__ void pair_barrier(int pair) {
  __syncwarp();
  asm volatile("barrier.sync %0, 64;" ::"r"(1 + pair) : "memory");
}

// The record of point pid (< last; an empty record otherwise).
template <class FT>
__device__ __forceinline__ PointRec point_record(const RP& P, const float* __restrict__ pos,
                                                 const FT* __restrict__ feat, const RasterWs& ws, int pid, int last,
                                                 uint64_t stream) {
  PointRec R;
  R.mask = 0;
  R.pix0 = 0;
  R.h0term = 0.f;
  R.sc = make_float4(0.f, 0.f, 0.f, 0.f);
  R.x = R.y = R.z = 0.f;
  R.pad0 = R.pad1 = 0.f;
  if (pid >= last) return R;
  // the point's four (T_k alpha_k, dL/dalpha_k) pairs, one per footprint
  // corner (zero where no fragment blended), as one 32-byte sector
  const uint4 fa = ld_hint_u4(reinterpret_cast<const uint4*>(ws.fscal) + 2 * (long long)pid, stream);
  const uint4 fb = ld_hint_u4(reinterpret_cast<const uint4*>(ws.fscal) + 2 * (long long)pid + 1, stream);
  const float2 sc[4] = {make_float2(__uint_as_float(fa.x), __uint_as_float(fa.y)),
                        make_float2(__uint_as_float(fa.z), __uint_as_float(fa.w)),
                        make_float2(__uint_as_float(fb.x), __uint_as_float(fb.y)),
                        make_float2(__uint_as_float(fb.z), __uint_as_float(fb.w))};
  R.x = __ldg(pos + 3 * pid + 0);
  R.y = __ldg(pos + 3 * pid + 1);
  R.z = __ldg(pos + 3 * pid + 2);
  if (((fa.x | fa.y | fa.z | fa.w | fb.x | fb.y | fb.z | fb.w) & 0x7fffffffu) == 0u) return R;
  Splat sp;
  splat_xyz(P, R.x, R.y, R.z, sp);
  // exp(h0) as the forward's binning pass stored it (head mode), and
  // alpha_h = 1 - exp(-exp(h0)) from it with the same operations
  const float e_h0 = __ldg(ws.pexp + pid);
  const float ah = -expm1f(-e_h0);
  float dah = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    // a corner whose fragment has T_k alpha_k = 0 adds nothing to the
    // colour gradient: its image-gradient row is not gathered
    if (sc[k].x != 0.f) R.mask |= 1u << k;
    const float w = corner_weight(sp.f, k & 1, k >> 1);
    if (__fmul_rn(ah, w) <= P.alpha_max) dah = __fmaf_rn(w, sc[k].y, dah);
  }
  // channel 0 of the blended color is the constant 1; the opacity gradient
  // reaches h0 through alpha_h = 1 - exp(-exp(h0))
  R.h0term = dah * (e_h0 * expf(-e_h0));
  R.pix0 = sp.f.j0 * P.cam.W + sp.f.i0;
  R.sc = make_float4(sc[0].x, sc[1].x, sc[2].x, sc[3].x);
  return R;
}

template <int GA, class FT>
__global__ void __launch_bounds__(kThreads, 4) k_point_grad_hash(RP P, GridParams Gp, const float* __restrict__ pos,
                                                               const FT* __restrict__ feat,
                                                               const float* __restrict__ d_image, RasterWs ws,
                                                               float* __restrict__ grad_table,
                                                               float* __restrict__ d_feat, float* __restrict__ dfine,
                                                               int chunk) {
  constexpr int kH = GA / 2;                      // levels per half
  constexpr int kPW = 16 / kH;                    // points per warp (two lanes per level)
  constexpr int kGroups = (kThreads / 64) * kPW;  // points in flight per CTA
  constexpr int kBatch = 32 / kPW;                // iterations covered by one round of point records
  // warps come in pairs over the same kPW points: the even warp takes the
  // coarse half of the levels, the odd warp the fine half.  Each level has
  // two adjacent lanes, one per x vertex of the cell (bx = the vertex's x
  // parity): the pair's reductions usually fall in one 128-byte line and
  // cost one L1 wavefront instead of two.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool coarse = (warp & 1) == 0;
  const uint32_t bx = lane & 1u;
  const int lvl = (lane >> 1) % kH;
  const int l = (coarse ? 0 : kH) + lvl;
  const int ch = 4 * l;
  const bool active = l < Gp.n_levels;
  const int pw = lane / (2 * kH);
  const int slot = (warp >> 1) * kPW + pw;
  // the CTA takes `chunk` consecutive points; its point slots interleave
  // over them, so at any moment its warps work on neighbouring points
  // (shared image and fragment data in L1) while each slot's own sequence,
  // kGroups points apart, stays within a leaf or two
  // n <= 2^25 (the limit of the backward calls), so 32-bit point indices
  const int first = (int)blockIdx.x * chunk + slot;
  const int last = (int)min((long long)(blockIdx.x + 1) * chunk, P.n);
  const uint64_t keep = l2_evict_last(), stream = l2_evict_first();
  float* gl = active ? grad_table + 4 * Gp.offset[l] : nullptr;
  // this lane's level, hoisted: a row is x + y my + z mz (dense) or
  // (x ^ y my ^ z mz) & mask (hashed), as in vertex_row
  const bool dense = active && Gp.dense[active ? l : 0];
  const uint32_t side = active ? Gp.side[l] : 1u;
  const uint32_t my = dense ? side : 2654435761u, mz = dense ? side * side : 805459861u;
  const uint32_t rmask = dense ? 0xffffffffu : Gp.hash_mask;
  const int N = active ? Gp.res[l] : 1;
  // the coarse warps' corner accumulators, [y-z corner][point slot][level][x side]
  constexpr int kStride = kGroups * kH * 2;
  __shared__ float4 acc_s[4][kStride];
  float4* acc = &acc_s[0][(slot * kH + lvl) * 2 + bx];
  // the cell whose corners the accumulators hold (kFar: none yet)
  constexpr uint32_t kFar = 1u << 30;
  uint32_t hx = kFar, hy = kFar, hz = kFar;
  // Per-point values (fragment scalars, pixel, position, the h0 term) are
  // formed once per point: one lane per point computes them for the next
  // kBatch x kPW points of the warp pair into records, and the level lanes
  // of both warps then read the records, instead of every level lane
  // repeating the projection and the fragment gathers.  The fine warp, whose
  // level loop is the shorter one, forms the records of the next batch
  // before its level loop of the current batch, so the coarse warp never
  // waits for them; the records are double-buffered, so one barrier of the
  // pair per batch orders both the writes before the reads and the reads
  // of a buffer before its next writes.
  __shared__ PointRec rec_s[kThreads / 64][2][32];
  const int pair = warp >> 1;
  const int base = (int)blockIdx.x * chunk + pair * kPW;  // the pair's first point slot
  if (!coarse && base < last)
    rec_s[pair][0][lane] = point_record(P, pos, feat, ws, base + lane % kPW + (lane / kPW) * kGroups, last, stream);
  pair_barrier(pair);
  int buf = 0;
  for (int t0 = 0; base + t0 * kGroups < last; t0 += kBatch, buf ^= 1) {
    PointRec* rec = rec_s[pair][buf];
    if (!coarse && base + (t0 + kBatch) * kGroups < last)
      rec_s[pair][buf ^ 1][lane] =
          point_record(P, pos, feat, ws, base + lane % kPW + (t0 + kBatch + lane / kPW) * kGroups, last, stream);
    for (int t = 0; t < kBatch; ++t) {
      const int id = first + (t0 + t) * kGroups;
      if (id >= last) break;
      const PointRec R = rec[t * kPW + pw];
      float dc[4] = {0.f, 0.f, 0.f, 0.f};
      if (R.mask) {
        const float scx[4] = {R.sc.x, R.sc.y, R.sc.z, R.sc.w};
        if (active) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (!(R.mask & (1u << k))) continue;
            const int pix = R.pix0 + (k >> 1) * P.cam.W + (k & 1);
            const float4 g = __ldg(reinterpret_cast<const float4*>(d_image + (long long)pix * P.F + ch));
            dc[0] = __fmaf_rn(scx[k], g.x, dc[0]);
            dc[1] = __fmaf_rn(scx[k], g.y, dc[1]);
            dc[2] = __fmaf_rn(scx[k], g.z, dc[2]);
            dc[3] = __fmaf_rn(scx[k], g.w, dc[3]);
          }
        }
        if (l == 0) dc[0] = R.h0term;
      }
      if (!active) continue;
      if (d_feat && bx == 0)
        *reinterpret_cast<float4*>(d_feat + (long long)id * P.F + ch) = make_float4(dc[0], dc[1], dc[2], dc[3]);
      if (!coarse && dfine) {
        // deferred fine levels: the row goes to k_grad_fine (level-major, so
        // that pass reads a level's rows of consecutive points together)
        if (bx == 0) __stcs(reinterpret_cast<float4*>(dfine) + (long long)lvl * P.n + id, make_float4(dc[0], dc[1], dc[2], dc[3]));
        continue;
      }
      if (dc[0] == 0.f && dc[1] == 0.f && dc[2] == 0.f && dc[3] == 0.f) continue;
      uint32_t cx, cy, cz;
      float gx[2], gy[2], gz[2];
      cell_frac(R.x, N, cx, gx[0], gx[1]);
      cell_frac(R.y, N, cy, gy[0], gy[1]);
      cell_frac(R.z, N, cz, gz[0], gz[1]);
      // slot s holds the corner whose offsets are s's bits xor the cell's
      // parities; swapping the weight pairs of odd cells makes gy[sy] that
      // corner's weight.  Along x this lane owns the vertex of parity bx.
      const uint32_t px = cx & 1u, py = cy & 1u, pz = cz & 1u;
      const uint32_t qx = hx & 1u, qy = hy & 1u, qz = hz & 1u;
      const uint32_t X = cx + (bx ^ px);
      const float wx = (bx ^ px) ? gx[1] : gx[0];
      if (py) swap_f(gy[0], gy[1]);
      if (pz) swap_f(gz[0], gz[1]);
      if (coarse) {
        // does the slot keep its vertex?
        const uint32_t HX = hx + (bx ^ qx);
        const bool kx = X == HX;
        const bool ky[2] = {cy + py == hy + qy, cy + (py ^ 1u) == hy + (qy ^ 1u)};
        const bool kz[2] = {cz + pz == hz + qz, cz + (pz ^ 1u) == hz + (qz ^ 1u)};
        const bool held = hx != kFar;
        // the y and z terms of the held cell's rows of slots sy, sz
        const uint32_t hyb[2] = {(hy + qy) * my, (hy + (qy ^ 1u)) * my};
        const uint32_t hzb[2] = {(hz + qz) * mz, (hz + (qz ^ 1u)) * mz};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const uint32_t sy = s & 1, sz = s >> 1;
          const float w = wx * gy[sy] * gz[sz];
          const float4 a = acc[s * kStride];
          const bool same = kx && ky[sy] && kz[sz];
          // same vertex: add to the sum; otherwise start a new sum (fma onto 0)
          acc[s * kStride] = make_float4(__fmaf_rn(w, dc[0], same ? a.x : 0.f), __fmaf_rn(w, dc[1], same ? a.y : 0.f),
                                         __fmaf_rn(w, dc[2], same ? a.z : 0.f), __fmaf_rn(w, dc[3], same ? a.w : 0.f));
          // the slot moves to another vertex: send the old vertex its sum
          if (!same && held) {
            const uint32_t row = dense ? HX + hyb[sy] + hzb[sz] : ((HX ^ hyb[sy] ^ hzb[sz]) & rmask);
            red_add_v4(gl + 4ull * row, a, keep);
          }
        }
      } else {
        // the y and z terms of this cell's rows of slots sy, sz
        const uint32_t yb[2] = {(cy + py) * my, (cy + (py ^ 1u)) * my};
        const uint32_t zb[2] = {(cz + pz) * mz, (cz + (pz ^ 1u)) * mz};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const uint32_t sy = s & 1, sz = s >> 1;
          const float w = wx * gy[sy] * gz[sz];
          const uint32_t row = dense ? X + yb[sy] + zb[sz] : ((X ^ yb[sy] ^ zb[sz]) & rmask);
          red_add_v4(gl + 4ull * row, make_float4(w * dc[0], w * dc[1], w * dc[2], w * dc[3]), keep);
        }
      }
      hx = cx;
      hy = cy;
      hz = cz;
    }
    pair_barrier(pair);
  }
  if (!active || !coarse || hx == kFar) return;
  const uint32_t qx = hx & 1u, qy = hy & 1u, qz = hz & 1u;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const uint32_t sy = s & 1, sz = s >> 1;
    red_add_v4(gl + 4ull * vertex_row(Gp, l, hx + (bx ^ qx), hy + (sy ^ qy), hz + (sz ^ qz)), acc[s * kStride], keep);
  }
}

// The fine levels of the grid adjoint, deferred: for tables whose fine
// levels do not fit in L2, reductions into them from the fused kernel miss
// L2 and go to DRAM twice (a read before the add, a write-back later).  The
// fused kernel then stores each point's gradient row of every fine level
// (dL/dh of the level, 4 floats; level-major in dfine) instead of reducing
// it, and this pass adds the corner contributions level group after level
// group (plan_level_groups), so the rows receiving reductions at a time are
// one group's and stay in L2.  Two lanes per point, one per x vertex of the
// cell, 16 consecutive points per warp; the contributions are the fused
// kernel's own, (w_x w_y) w_z times the row.
__global__ void __launch_bounds__(256) k_grad_fine(GridParams Gp, LevelGroups LG, int l_first,
                                                   const float* __restrict__ pos, const float* __restrict__ dfine,
                                                   long long n, float* __restrict__ grad_table) {
  const int lb = LG.begin[blockIdx.y], le = LG.begin[blockIdx.y + 1];
  const uint64_t keep = l2_evict_last(), stream = l2_evict_first();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t bx = lane & 1u;
  // n <= 2^25 (the limit of the backward calls): 32-bit point indices
  const uint32_t n_groups = (uint32_t)((n + 15) >> 4);
  const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_groups; g += n_warps) {
    const uint32_t p = g * 16u + (lane >> 1);
    if (p >= (uint32_t)n) continue;  // nothing below is warp-collective
    const float x = __ldg(pos + 3 * p + 0), y = __ldg(pos + 3 * p + 1), z = __ldg(pos + 3 * p + 2);
    for (int l = lb; l < le; ++l) {
      const uint4 r = ld_hint_u4(reinterpret_cast<const uint4*>(dfine) + (long long)(l - l_first) * n + p, stream);
      const float4 d = make_float4(__uint_as_float(r.x), __uint_as_float(r.y), __uint_as_float(r.z),
                                   __uint_as_float(r.w));
      if (d.x == 0.f && d.y == 0.f && d.z == 0.f && d.w == 0.f) continue;
      uint32_t cx, cy, cz;
      float gx[2], gy[2], gz[2];
      const int N = Gp.res[l];
      cell_frac(x, N, cx, gx[0], gx[1]);
      cell_frac(y, N, cy, gy[0], gy[1]);
      cell_frac(z, N, cz, gz[0], gz[1]);
      float* gl = grad_table + 4 * Gp.offset[l];
      const float wx = gx[bx];
#pragma unroll
      for (int yz = 0; yz < 4; ++yz) {
        const int by = yz & 1, bz = yz >> 1;
        const float w = wx * gy[by] * gz[bz];
        const uint32_t row = vertex_row(Gp, l, cx + bx, cy + by, cz + bz);
        red_add_v4(gl + 4ull * row, make_float4(w * d.x, w * d.y, w * d.z, w * d.w), keep);
      }
    }
  }
}

// Levels per half of the fused kernel's warp pairs for a grid of n_levels
// levels (the template size it is launched with, halved).
inline int adjoint_half(int n_levels) { return n_levels <= 8 ? 4 : n_levels <= 16 ? 8 : 16; }

// Whether the fine half's gradient rows are deferred to k_grad_fine (they
// do not fit the L2 budget), and the bytes of its row buffer.
inline size_t fine_defer_bytes(const GridParams& Gp, long long n) {
  const int kH = adjoint_half(Gp.n_levels);
  if (Gp.n_levels <= kH) return 0;
  long long rows = 0;
  for (int l = kH; l < Gp.n_levels; ++l) rows += level_rows(Gp, l);
  if (rows * 16 <= kQueryL2Budget) return 0;
  return (size_t)std::max<long long>(n, 1) * (size_t)(Gp.n_levels - kH) * 16;
}

template <int GA, class FT>
inpc_status launch_point_grad_hash(const RP& P, const GridParams& Gp, const float* pos, const FT* feat,
                                   const float* d_image, const RasterWs& ws, float* grad_table, float* d_feat,
                                   float* dfine, cudaStream_t s) {
  constexpr int kGroups = (kThreads / 64) * (32 / GA);  // points in flight per CTA
  // kRun points per group and CTA chunk, as many CTAs as that needs up to
  // 32 per SM (longer runs beyond that)
  constexpr long long kRun = 48;
  const long long ctas_max = (long long)device_sm_count() * 32;
  const long long chunk = kGroups * std::max<long long>(kRun, ceil_div(P.n, ctas_max * kGroups));
  const long long grid = ceil_div(P.n, chunk);
  INPC_TIMED("k_point_grad_hash", s,
             k_point_grad_hash<GA, FT><<<(unsigned)std::max<long long>(grid, 1), kThreads, 0, s>>>(
                 P, Gp, pos, feat, d_image, ws, grad_table, d_feat, dfine, (int)chunk));
  INPC_TRY(check_launch("k_point_grad_hash"));
  if (!dfine) return INPC_OK;
  constexpr int kH = GA / 2;
  const LevelGroups LG = plan_level_groups(Gp, 16, kH);
  const long long cap = (long long)device_sm_count() * 16;
  const dim3 g2((unsigned)std::max<long long>(1, std::min<long long>((long long)ceil_div(2 * P.n, 256), cap)),
                (unsigned)LG.n);
  INPC_TIMED("k_grad_fine", s, k_grad_fine<<<g2, 256, 0, s>>>(Gp, LG, kH, pos, dfine, P.n, grad_table));
  return check_launch("k_grad_fine");
}

}  // namespace
}  // namespace inpc

using namespace inpc;

extern "C" inpc_status inpc_rasterize_bwd(const inpc_camera* cam, const inpc_raster_opts* opts, const float* pos,
                                          const float* opacity, const void* feat, int64_t n, const float* T_final,
                                          const int32_t* n_contrib, const float* d_image, float* d_opacity,
                                          float* d_feat, void* workspace, size_t workspace_bytes,
                                          inpc_stream_t stream) {
  inpc::fault_arg(pos);
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
  inpc::fault_arg(pos);
  RP P;
  INPC_TRY(make_rp(cam, opts, n, P));
  GridParams Gp;
  int64_t n_entries = 0;
  INPC_TRY(make_params(grid, Gp, &n_entries));
  if (!P.head) return fail(INPC_ERR_UNSUPPORTED, "inpc_rasterize_bwd_hashgrid needs INPC_OPACITY_FROM_CH0");
  if (P.F != 4 * Gp.n_levels)
    return fail(INPC_ERR_INVALID_ARG, "n_channels (%d) must equal n_levels * n_feats (%d)", P.F, 4 * Gp.n_levels);
  const RasterWs need = carve(nullptr, P.n_pix, n);
  // the deferred fine-level rows (large tables) follow the rasterizer's part
  const size_t fine_off = (need.bytes + 255) / 256 * 256;
  const size_t fine_bytes = fine_defer_bytes(Gp, n);
  const size_t total = fine_bytes ? fine_off + fine_bytes : need.bytes;
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
  float* dfine = fine_bytes ? reinterpret_cast<float*>(static_cast<char*>(workspace) + fine_off) : nullptr;
  return dispatch(P.F, [&](auto Vc, auto Gc) -> inpc_status {
    constexpr int V = decltype(Vc)::value, GA = decltype(Gc)::value;
    auto run = [&](auto ftag) -> inpc_status {
      using FT = decltype(ftag);
      const FT* f = static_cast<const FT*>(feat);
      INPC_TRY((launch_blend_bwd<V, GA, FT>(P, f, n_contrib, d_image, ws, s)));
      if (Gp.n_levels <= 8)
        return launch_point_grad_hash<8, FT>(P, Gp, pos, f, d_image, ws, grad_table, d_feat, dfine, s);
      if (Gp.n_levels <= 16)
        return launch_point_grad_hash<16, FT>(P, Gp, pos, f, d_image, ws, grad_table, d_feat, dfine, s);
      return launch_point_grad_hash<32, FT>(P, Gp, pos, f, d_image, ws, grad_table, d_feat, dfine, s);
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
  if (inpc::fault_workspace_overflow())
    return inpc::fail(INPC_ERR_CAPACITY, "inpc_rasterize_bwd_hashgrid_workspace_size: size overflow (injected fault)");
  if (!bytes) return fail(INPC_ERR_INVALID_ARG, "bytes is null");
  RP P;
  INPC_TRY(make_rp(cam, opts, n, P));
  GridParams Gp;
  int64_t n_entries = 0;
  INPC_TRY(make_params(grid, Gp, &n_entries));
  const size_t base = carve(nullptr, P.n_pix, n).bytes;
  const size_t fine_bytes = fine_defer_bytes(Gp, n);
  *bytes = fine_bytes ? (base + 255) / 256 * 256 + fine_bytes : base;
  return INPC_OK;
}
