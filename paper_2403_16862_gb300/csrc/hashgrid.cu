// hashgrid.cu -- multi-resolution hash-grid query (Sec. 3.3, App. A.5) and
// its adjoint (the table gradient).
//
// The query runs two threads per (point, level), each gathering the four
// corners on one side of the cell along x; levels go in groups of two along
// grid y so that the rows in use at any time fit in L2, and within a group
// a warp covers 8 points x 2 levels.  Corner rows are gathered as 16-byte
// vectors (FP32) or 8-byte vectors (BF16).  The output is written with
// streaming stores so that it does not evict the table from L2.
//
// The backward uses red.global.add.v4.f32 (one 16-byte vector reduction per
// corner and level), accumulating into an FP32 gradient table.
#include <algorithm>

#include "hashgrid_impl.cuh"

namespace inpc {
namespace {

// Levels are processed in groups of kLevelGroup along grid y: blocks are
// dispatched in linear order, so all points visit one group of levels
// before the next, and the rows touched at a time (one or two 8 MB levels)
// stay resident in L2 instead of the whole table.
constexpr int kLevelGroup = 2;

// Two lanes per (point, level): lane bx gathers the four corners at x + bx.
// The x neighbours' rows differ only in their lowest bits (hashed: x is
// multiplied by 1 before the XOR; dense: consecutive rows), so they share
// one 128-byte line unless the carry of x + 1 reaches bit 3 (FP32) or bit 4
// (BF16).  Loading both from one instruction then costs one L1 wavefront
// instead of two, and the L1 wavefront rate bounds this kernel.  The pair
// adds its partial sums with one exchange, and each lane stores half of
// the four features.
template <class TT, class OT>
__global__ void __launch_bounds__(256) k_hash_fwd(GridParams P, const TT* __restrict__ table,
                                                  const float* __restrict__ pos, long long n, OT* __restrict__ h) {
  const int l0 = blockIdx.y * kLevelGroup;
  const int gl = min(kLevelGroup, P.n_levels - l0);
  // n <= 2^29 (checked by the caller): 32-bit indices do not overflow
  const uint32_t total = 2u * (uint32_t)n * (uint32_t)gl;
  const uint64_t keep = l2_evict_last();
  const int lane = threadIdx.x & 31;
  const uint32_t bx = lane & 1u;
  // warp-uniform trip count: the pair exchange is a warp shuffle
  for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x - lane); base < total; base += gridDim.x * blockDim.x) {
    const uint32_t i = base + lane;
    const bool valid = i < total;
    const uint32_t item = (valid ? i : total - 1) >> 1;  // spare lanes redo the last item
    const uint32_t p = item / (uint32_t)gl;
    const int l = l0 + (int)(item - p * gl);
    query_pair<TT, OT>(P, table, __ldg(pos + 3 * p + 0), __ldg(pos + 3 * p + 1), __ldg(pos + 3 * p + 2), p, l, bx,
                       valid, h, keep);
  }
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
  inpc::fault_arg(table);
  GridParams P;
  int64_t total = 0;
  INPC_TRY(make_params(g, P, &total));
  if (n < 0 || n > (int64_t(1) << 29)) return fail(INPC_ERR_CAPACITY, "n must be in [0, 2^29]");
  if (n == 0) return INPC_OK;
  if (!table || !pos || !h_out) return fail(INPC_ERR_INVALID_ARG, "inpc_query_hashgrid: null pointer");
  const size_t ta = g->table_dtype == INPC_F32 ? 16 : 8, oa = g->out_dtype == INPC_F32 ? 16 : 8;
  if (!aligned(table, ta) || !aligned(h_out, oa) || !aligned(pos, 4))
    return fail(INPC_ERR_INVALID_ARG, "inpc_query_hashgrid: misaligned table/output/pos");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const dim3 grid = grid_for(2 * n, P.n_levels, 256);
  TimedLaunch timed("k_hash_fwd", s);
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
  inpc::fault_arg(pos);
  GridParams P;
  int64_t total = 0;
  INPC_TRY(make_params(g, P, &total));
  if (n < 0 || n > INT32_MAX) return fail(INPC_ERR_CAPACITY, "n out of range");
  if (n == 0) return INPC_OK;
  if (!pos || !dh || !grad_table) return fail(INPC_ERR_INVALID_ARG, "inpc_query_hashgrid_bwd: null pointer");
  if (!aligned(grad_table, 16) || !aligned(dh, 16) || !aligned(pos, 4))
    return fail(INPC_ERR_INVALID_ARG, "inpc_query_hashgrid_bwd: misaligned buffer");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  TimedLaunch timed("k_hash_bwd", s);
  k_hash_bwd<<<grid_for(n, P.n_levels, 256), 256, 0, s>>>(P, pos, dh, n, grad_table);
  return check_launch("k_hash_bwd");
}
