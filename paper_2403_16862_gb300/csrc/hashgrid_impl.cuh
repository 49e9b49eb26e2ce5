// hashgrid_impl.cuh -- multi-resolution grid layout and per-level cell
// arithmetic (Sec. 3.3, App. A.5), shared by the query kernels and the
// fused rasterizer backward.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace inpc {
namespace {

constexpr int kMaxLevels = 32;
// Every level starts on a multiple of 16 rows (256 bytes of FP32 rows), so
// row parity is the same within a level and in the whole table and aligned
// row pairs can be fetched with one vector load.
constexpr int64_t kLevelAlignRows = 16;

struct GridParams {
  int n_levels;
  uint32_t hash_mask;
  int res[kMaxLevels];
  uint32_t side[kMaxLevels];  // res + 1
  uint32_t dense[kMaxLevels];
  long long offset[kMaxLevels];
};

inpc_status make_params(const inpc_hashgrid_desc* g, GridParams& p, int64_t* total) {
  if (!g) return fail(INPC_ERR_INVALID_ARG, "hash grid descriptor is null");
  if (g->n_levels < 1 || g->n_levels > kMaxLevels)
    return fail(INPC_ERR_INVALID_ARG, "n_levels must be in [1, 32], got %d", g->n_levels);
  if (g->n_feats != 4) return fail(INPC_ERR_UNSUPPORTED, "n_feats must be 4, got %d", g->n_feats);
  if (g->log2_T < 4 || g->log2_T > 24) return fail(INPC_ERR_INVALID_ARG, "log2_T must be in [4, 24]");
  if ((g->table_dtype != INPC_F32 && g->table_dtype != INPC_BF16) ||
      (g->out_dtype != INPC_F32 && g->out_dtype != INPC_BF16))
    return fail(INPC_ERR_UNSUPPORTED, "dtype must be INPC_F32 or INPC_BF16");
  const int64_t T = int64_t(1) << g->log2_T;
  p.n_levels = g->n_levels;
  p.hash_mask = (uint32_t)(T - 1);
  int64_t off = 0;
  for (int l = 0; l < g->n_levels; ++l) {
    const int64_t r = g->res[l];
    if (r < 1 || r > (1 << 24)) return fail(INPC_ERR_INVALID_ARG, "res[%d] = %lld out of range", l, (long long)r);
    const int64_t side = r + 1;
    const bool dense = side <= 4096 && side * side * side <= T;
    p.res[l] = (int)r;
    p.side[l] = (uint32_t)side;
    p.dense[l] = dense ? 1u : 0u;
    off = (off + kLevelAlignRows - 1) / kLevelAlignRows * kLevelAlignRows;
    p.offset[l] = off;
    off += dense ? side * side * side : T;
  }
  off = (off + kLevelAlignRows - 1) / kLevelAlignRows * kLevelAlignRows;
  for (int l = g->n_levels; l < kMaxLevels; ++l) {
    p.res[l] = 1; p.side[l] = 2; p.dense[l] = 1; p.offset[l] = off;
  }
  *total = off;
  return INPC_OK;
}

// The query's level groups: a launch covers one group per grid y index,
// every point going through the group's levels before the next group
// starts, so the rows in use at a time are one group's.  Groups hold an
// even number of levels (pairs, so that a point's output for a pair is
// one 32-byte sector), as many pairs as keep the group's rows within
// kQueryL2Budget bytes: a table that fits in L2 beside the streamed
// positions and outputs is one group (each point's position read once),
// a larger one is split so that a group's rows stay resident.
#ifndef INPC_QUERY_L2_BUDGET_MB
#define INPC_QUERY_L2_BUDGET_MB 64
#endif
constexpr long long kQueryL2Budget = (long long)INPC_QUERY_L2_BUDGET_MB << 20;

struct LevelGroups {
  int n;
  int begin[kMaxLevels + 1];  // group j covers levels begin[j] .. begin[j + 1] - 1
};

// Rows of level l.
inline long long level_rows(const GridParams& P, int l) {
  const long long side = P.side[l];
  return P.dense[l] ? side * side * side : (long long)P.hash_mask + 1;
}

// Level groups of the levels l_first .. n_levels - 1.
inline LevelGroups plan_level_groups(const GridParams& P, int row_bytes, int l_first = 0) {
  LevelGroups g;
  g.n = 0;
  long long bytes = 0;
  for (int l = l_first; l < P.n_levels; l += 2) {
    long long pair = 0;
    for (int k = l; k < l + 2 && k < P.n_levels; ++k) pair += level_rows(P, k) * row_bytes;
    if (g.n == 0 || bytes + pair > kQueryL2Budget) {
      g.begin[g.n++] = l;
      bytes = 0;
    }
    bytes += pair;
  }
  g.begin[g.n] = P.n_levels;
  return g;
}

// Cell of x in [0, 1] at resolution N and both linear weights of that cell:
// with s = fl(x N) and e = x N - s exactly (FMA), the upper-corner weight
// f1 = x N - cell and the lower-corner weight f0 = cell + 1 - x N are each
// formed from exact terms and rounded once, so each keeps full relative
// accuracy even when the other is close to 1; the cell is the floor of the
// exact product.
__device__ __forceinline__ void cell_frac(float x, int N, uint32_t& cell, float& f0, float& f1) {
  x = fminf(fmaxf(x, 0.0f), 1.0f);
  const float Nf = (float)N;
  const float s = __fmul_rn(x, Nf);
  const float e = __fmaf_rn(x, Nf, -s);
  float c = floorf(s);
  if (__fadd_rn(__fsub_rn(s, c), e) < 0.0f) c -= 1.0f;  // exact product just below the integer s
  if (c > Nf - 1.0f) c = Nf - 1.0f;
  cell = (uint32_t)c;
  f1 = __fadd_rn(__fsub_rn(s, c), e);
  f0 = __fsub_rn(__fsub_rn(c + 1.0f, s), e);
}

__device__ __forceinline__ void swap_f(float& a, float& b) {
  const float t = a;
  a = b;
  b = t;
}

__device__ __forceinline__ uint32_t vertex_row(const GridParams& P, int l, uint32_t x, uint32_t y, uint32_t z) {
  if (P.dense[l]) return x + P.side[l] * (y + P.side[l] * z);
  return (x ^ (y * 2654435761u) ^ (z * 805459861u)) & P.hash_mask;
}

// L2 eviction priorities: the table gradient (and the table in the query)
// is kept with evict_last while data read once streams through with
// evict_first, so the rows that receive reductions or gathers stay resident.
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

template <class TT>
__device__ __forceinline__ float4 load_row(const TT* __restrict__ table, long long row, uint64_t pol);

template <>
__device__ __forceinline__ float4 load_row<float>(const float* __restrict__ table, long long row, uint64_t pol) {
  float4 r;
  asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "l"(table + 4 * row), "l"(pol));
  return r;
}

template <>
__device__ __forceinline__ float4 load_row<__nv_bfloat16>(const __nv_bfloat16* __restrict__ table, long long row,
                                                          uint64_t pol) {
  uint32_t x, y;
  asm("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(x), "=r"(y)
               : "l"(table + 4 * row), "l"(pol));
  return make_float4(__uint_as_float(x << 16), __uint_as_float(x & 0xFFFF0000u), __uint_as_float(y << 16),
                     __uint_as_float(y & 0xFFFF0000u));
}

template <class OT>
__device__ __forceinline__ void store_out(OT* __restrict__ out, long long idx4, float4 v);

template <>
__device__ __forceinline__ void store_out<float>(float* __restrict__ out, long long idx4, float4 v) {
  __stcs(reinterpret_cast<float4*>(out) + idx4, v);
}

template <>
__device__ __forceinline__ void store_out<__nv_bfloat16>(__nv_bfloat16* __restrict__ out, long long idx4, float4 v) {
  __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
  __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
  uint2 raw;
  raw.x = *reinterpret_cast<uint32_t*>(&a);
  raw.y = *reinterpret_cast<uint32_t*>(&b);
  __stcs(reinterpret_cast<uint2*>(out) + idx4, raw);
}

// Half of a 4-feature output row: features 2 half .. 2 half + 1.
template <class OT>
__device__ __forceinline__ void store_half(OT* __restrict__ out, long long idx4, uint32_t half, float2 v);

template <>
__device__ __forceinline__ void store_half<float>(float* __restrict__ out, long long idx4, uint32_t half, float2 v) {
  __stcs(reinterpret_cast<float2*>(out) + 2 * idx4 + half, v);
}

template <>
__device__ __forceinline__ void store_half<__nv_bfloat16>(__nv_bfloat16* __restrict__ out, long long idx4,
                                                          uint32_t half, float2 v) {
  __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
  __stcs(reinterpret_cast<unsigned int*>(out) + 2 * idx4 + half, *reinterpret_cast<unsigned int*>(&a));
}

// One lane of the query's lane pair for a point at (x, y, z) and level l:
// lane bx gathers the four corners at x + bx of the point's cell and
// weights them; the pair adds its partial sums with one exchange (a warp
// shuffle, so the whole warp calls this together) and the lane returns
// features 2 bx and 2 bx + 1 of the level.
template <class TT>
__device__ __forceinline__ float2 query_half(const GridParams& P, const TT* __restrict__ table, float x, float y,
                                             float z, int l, uint32_t bx, uint64_t keep) {
  uint32_t cx, cy, cz;
  float gx[2], gy[2], gz[2];
  const int N = P.res[l];
  cell_frac(x, N, cx, gx[0], gx[1]);
  cell_frac(y, N, cy, gy[0], gy[1]);
  cell_frac(z, N, cz, gz[0], gz[1]);
  const TT* tab = table + 4 * P.offset[l];
  const float wx = bx ? gx[1] : gx[0];
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int yz = 0; yz < 4; ++yz) {
    const int by = yz & 1, bz = yz >> 1;
    const float4 t = load_row<TT>(tab, vertex_row(P, l, cx + bx, cy + by, cz + bz), keep);
    const float w = wx * (gy[by] * gz[bz]);
    acc.x = fmaf(w, t.x, acc.x);
    acc.y = fmaf(w, t.y, acc.y);
    acc.z = fmaf(w, t.z, acc.z);
    acc.w = fmaf(w, t.w, acc.w);
  }
  // lane 0 keeps features 0-1, lane 1 features 2-3
  const float s0 = bx ? acc.x : acc.z, s1 = bx ? acc.y : acc.w;
  const float r0 = __shfl_xor_sync(0xffffffffu, s0, 1), r1 = __shfl_xor_sync(0xffffffffu, s1, 1);
  return bx ? make_float2(acc.z + r0, acc.w + r1) : make_float2(acc.x + r0, acc.y + r1);
}

__device__ __forceinline__ void red_add_v4(float* addr, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}

__device__ __forceinline__ void red_add_v4(float* addr, float4 v, uint64_t pol) {
  asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(addr), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ uint4 ld_hint_u4(const void* p, uint64_t pol) {
  uint4 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ float2 ld_hint_f2(const void* p, uint64_t pol) {
  float2 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(r.x), "=f"(r.y)
               : "l"(p), "l"(pol));
  return r;
}

}  // namespace
}  // namespace inpc
