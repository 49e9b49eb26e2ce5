// hashgrid.cu -- multi-resolution hash-grid query (Sec. 3.3, App. A.5) and
// its adjoint (the table gradient).
//
// One thread per (point, level); levels go in groups of two along grid y so
// that the rows in use at any time fit in L2, and within a group a warp
// covers 16 points x 2 levels (32-byte output pieces, one sector each).  The 8 corner rows of a level are
// gathered as 16-byte vectors (FP32) or 8-byte vectors (BF16); for the x
// neighbours the hash (multiplier 1 on x) keeps rows adjacent, so a corner
// pair usually shares one 32-byte sector.  The output is written with
// streaming stores so that it does not evict the table from L2.
//
// The backward uses red.global.add.v4.f32 (one 16-byte vector reduction per
// corner and level), accumulating into an FP32 gradient table.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace inpc {
namespace {

constexpr int kMaxLevels = 32;

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
    p.offset[l] = off;
    off += dense ? side * side * side : T;
  }
  for (int l = g->n_levels; l < kMaxLevels; ++l) {
    p.res[l] = 1; p.side[l] = 2; p.dense[l] = 1; p.offset[l] = off;
  }
  *total = off;
  return INPC_OK;
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

__device__ __forceinline__ uint32_t vertex_row(const GridParams& P, int l, uint32_t x, uint32_t y, uint32_t z) {
  if (P.dense[l]) return x + P.side[l] * (y + P.side[l] * z);
  return (x ^ (y * 2654435761u) ^ (z * 805459861u)) & P.hash_mask;
}

template <class TT>
__device__ __forceinline__ float4 load_row(const TT* __restrict__ table, long long row);

template <>
__device__ __forceinline__ float4 load_row<float>(const float* __restrict__ table, long long row) {
  return __ldg(reinterpret_cast<const float4*>(table) + row);
}

template <>
__device__ __forceinline__ float4 load_row<__nv_bfloat16>(const __nv_bfloat16* __restrict__ table, long long row) {
  const uint2 raw = __ldg(reinterpret_cast<const uint2*>(table) + row);
  float4 r;
  r.x = __uint_as_float(raw.x << 16);
  r.y = __uint_as_float(raw.x & 0xFFFF0000u);
  r.z = __uint_as_float(raw.y << 16);
  r.w = __uint_as_float(raw.y & 0xFFFF0000u);
  return r;
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

// Levels are processed in groups of kLevelGroup along grid y: blocks are
// dispatched in linear order, so all points visit one group of levels
// before the next, and the rows touched at a time (one or two 8 MB levels)
// stay resident in L2 instead of the whole table.
constexpr int kLevelGroup = 2;

template <class TT, class OT>
__global__ void __launch_bounds__(256) k_hash_fwd(GridParams P, const TT* __restrict__ table,
                                                  const float* __restrict__ pos, long long n, OT* __restrict__ h) {
  const int l0 = blockIdx.y * kLevelGroup;
  const int gl = min(kLevelGroup, P.n_levels - l0);
  const long long total = n * gl;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / gl;
    const int l = l0 + (int)(i - p * gl);
    uint32_t cx, cy, cz;
    float gx[2], gy[2], gz[2];
    const int N = P.res[l];
    cell_frac(__ldg(pos + 3 * p + 0), N, cx, gx[0], gx[1]);
    cell_frac(__ldg(pos + 3 * p + 1), N, cy, gy[0], gy[1]);
    cell_frac(__ldg(pos + 3 * p + 2), N, cz, gz[0], gz[1]);
    const TT* tab = table + 4 * P.offset[l];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
      const float w = gx[bx] * gy[by] * gz[bz];
      const float4 t = load_row<TT>(tab, vertex_row(P, l, cx + bx, cy + by, cz + bz));
      acc.x = fmaf(w, t.x, acc.x);
      acc.y = fmaf(w, t.y, acc.y);
      acc.z = fmaf(w, t.z, acc.z);
      acc.w = fmaf(w, t.w, acc.w);
    }
    store_out<OT>(h, p * P.n_levels + l, acc);
  }
}

__device__ __forceinline__ void red_add_v4(float* addr, float4 v) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}

__global__ void __launch_bounds__(256) k_hash_bwd(GridParams P, const float* __restrict__ pos,
                                                  const float* __restrict__ dh, long long n,
                                                  float* __restrict__ grad) {
  const int l0 = blockIdx.y * kLevelGroup;
  const int gl = min(kLevelGroup, P.n_levels - l0);
  const long long total = n * gl;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = i / gl;
    const int l = l0 + (int)(i - p * gl);
    const float4 g = __ldcs(reinterpret_cast<const float4*>(dh) + p * P.n_levels + l);
    if (g.x == 0.f && g.y == 0.f && g.z == 0.f && g.w == 0.f) continue;
    uint32_t cx, cy, cz;
    float gx[2], gy[2], gz[2];
    const int N = P.res[l];
    cell_frac(__ldg(pos + 3 * p + 0), N, cx, gx[0], gx[1]);
    cell_frac(__ldg(pos + 3 * p + 1), N, cy, gy[0], gy[1]);
    cell_frac(__ldg(pos + 3 * p + 2), N, cz, gz[0], gz[1]);
    float* gl_ = grad + 4 * P.offset[l];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
      const float w = gx[bx] * gy[by] * gz[bz];
      const uint32_t row = vertex_row(P, l, cx + bx, cy + by, cz + bz);
      red_add_v4(gl_ + 4ull * row, make_float4(w * g.x, w * g.y, w * g.z, w * g.w));
    }
  }
}

dim3 grid_for(long long n, int n_levels, int threads) {
  const int groups = (n_levels + kLevelGroup - 1) / kLevelGroup;
  const long long work = n * std::min(kLevelGroup, n_levels);
  const long long cap = (long long)device_sm_count() * 16;
  long long g = ceil_div(work, threads);
  return dim3((unsigned)std::max<long long>(1, std::min(g, cap)), (unsigned)groups, 1);
}

}  // namespace
}  // namespace inpc

using namespace inpc;

extern "C" inpc_status inpc_hashgrid_n_entries(const inpc_hashgrid_desc* g, int64_t* n_entries) {
  if (!n_entries) return fail(INPC_ERR_INVALID_ARG, "n_entries is null");
  GridParams P;
  INPC_TRY(make_params(g, P, n_entries));
  return INPC_OK;
}

extern "C" inpc_status inpc_query_hashgrid(const inpc_hashgrid_desc* g, const void* table, const float* pos,
                                           int64_t n, void* h_out, inpc_stream_t stream) {
  GridParams P;
  int64_t total = 0;
  INPC_TRY(make_params(g, P, &total));
  if (n < 0 || n > INT32_MAX) return fail(INPC_ERR_CAPACITY, "n out of range");
  if (n == 0) return INPC_OK;
  if (!table || !pos || !h_out) return fail(INPC_ERR_INVALID_ARG, "inpc_query_hashgrid: null pointer");
  const size_t ta = g->table_dtype == INPC_F32 ? 16 : 8, oa = g->out_dtype == INPC_F32 ? 16 : 8;
  if (!aligned(table, ta) || !aligned(h_out, oa) || !aligned(pos, 4))
    return fail(INPC_ERR_INVALID_ARG, "inpc_query_hashgrid: misaligned table/output/pos");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const dim3 grid = grid_for(n, P.n_levels, 256);
  if (g->table_dtype == INPC_F32 && g->out_dtype == INPC_F32)
    k_hash_fwd<float, float><<<grid, 256, 0, s>>>(P, (const float*)table, pos, n, (float*)h_out);
  else if (g->table_dtype == INPC_F32)
    k_hash_fwd<float, __nv_bfloat16><<<grid, 256, 0, s>>>(P, (const float*)table, pos, n, (__nv_bfloat16*)h_out);
  else if (g->out_dtype == INPC_F32)
    k_hash_fwd<__nv_bfloat16, float><<<grid, 256, 0, s>>>(P, (const __nv_bfloat16*)table, pos, n, (float*)h_out);
  else
    k_hash_fwd<__nv_bfloat16, __nv_bfloat16>
        <<<grid, 256, 0, s>>>(P, (const __nv_bfloat16*)table, pos, n, (__nv_bfloat16*)h_out);
  return check_launch("k_hash_fwd");
}

extern "C" inpc_status inpc_query_hashgrid_bwd(const inpc_hashgrid_desc* g, const float* pos, const float* dh,
                                               int64_t n, float* grad_table, inpc_stream_t stream) {
  GridParams P;
  int64_t total = 0;
  INPC_TRY(make_params(g, P, &total));
  if (n < 0 || n > INT32_MAX) return fail(INPC_ERR_CAPACITY, "n out of range");
  if (n == 0) return INPC_OK;
  if (!pos || !dh || !grad_table) return fail(INPC_ERR_INVALID_ARG, "inpc_query_hashgrid_bwd: null pointer");
  if (!aligned(grad_table, 16) || !aligned(dh, 16) || !aligned(pos, 4))
    return fail(INPC_ERR_INVALID_ARG, "inpc_query_hashgrid_bwd: misaligned buffer");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_hash_bwd<<<grid_for(n, P.n_levels, 256), 256, 0, s>>>(P, pos, dh, n, grad_table);
  return check_launch("k_hash_bwd");
}
