// hashgrid.cu -- multi-resolution hash-grid query (Sec. 3.3, App. A.5) and
// its adjoint (the table gradient).
//
// The query runs two threads per point, each gathering the four corners on
// one side of the cell along x; a warp takes 16 consecutive points through
// all levels.  Corner rows are gathered as 16-byte vectors (FP32) or 8-byte
// vectors (BF16).  The output is written with streaming stores so that it
// does not evict the table from L2.
//
// The backward uses red.global.add.v4.f32 (one 16-byte vector reduction per
// corner and level), accumulating into an FP32 gradient table.
#include <algorithm>

#include "hashgrid_impl.cuh"

namespace inpc {
namespace {

// The adjoint processes levels in groups of kLevelGroup along grid y: blocks are
// dispatched in linear order, so all points visit one group of levels
// before the next, and the rows touched at a time (one or two 8 MB levels)
// stay resident in L2 instead of the whole table.
constexpr int kLevelGroup = 2;

// A warp takes 16 consecutive points, two lanes per point, through the
// levels of one level group (grid y, plan_level_groups), two levels at a
// time: lane bx gathers the four corners at x + bx
// of the point's cell.  The x neighbours' rows differ only in their lowest
// bits (hashed: x is multiplied by 1 before the XOR; dense: consecutive
// rows), so they share one 128-byte line unless the carry of x + 1 reaches
// bit 3 (FP32) or bit 4 (BF16): loading both from one instruction costs one
// L1 wavefront instead of two, and the L1 wavefront rate bounds this
// kernel.  Consecutive points come from the same octree leaf, so at the
// coarse levels the 16 points of an instruction mostly fall in a few cells
// and share their lines as well (about 2.6 distinct lines per point and
// level on average over the benchmark's 16 levels, against 2.9 with 8
// points of two levels per instruction).  A group's rows stay in L2 under
// evict_last while positions and outputs stream past them.  After each pair of levels the two lanes swap halves so that each stores
// one level's whole 16-byte row: the warp writes each point's two levels
// as one full 32-byte sector.
template <class TT, class OT>
__global__ void __launch_bounds__(256) k_hash_fwd(GridParams P, LevelGroups LG, const TT* __restrict__ table,
                                                  const float* __restrict__ pos, long long n, OT* __restrict__ h) {
  const int lb = LG.begin[blockIdx.y], le = LG.begin[blockIdx.y + 1];
  const uint64_t keep = l2_evict_last();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t bx = lane & 1u;
  // n <= 2^29 (checked by the caller): 32-bit indices do not overflow
  const uint32_t n_groups = (uint32_t)((n + 15) >> 4);
  const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
  // warp-uniform trip counts: the pair exchanges are warp shuffles
  for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_groups; g += n_warps) {
    const uint32_t pr = g * 16u + (lane >> 1);
    const bool valid = pr < (uint32_t)n;
    const uint32_t p = valid ? pr : (uint32_t)n - 1u;  // spare lanes redo the last point
    const float x = __ldg(pos + 3 * p + 0), y = __ldg(pos + 3 * p + 1), z = __ldg(pos + 3 * p + 2);
    OT* hp = h + (long long)p * P.n_levels * 4;
    for (int l = lb; l < le; l += 2) {
      const float2 a = query_half<TT>(P, table, x, y, z, l, bx, keep);
      if (l + 1 < le) {
        const float2 b = query_half<TT>(P, table, x, y, z, l + 1, bx, keep);
        // lane 0 holds features 0-1 of both levels, lane 1 features 2-3:
        // lane 0 gives level l + 1's half away and takes level l's, lane 1
        // the other way round
        const float2 give = bx ? a : b;
        const float r0 = __shfl_xor_sync(0xffffffffu, give.x, 1), r1 = __shfl_xor_sync(0xffffffffu, give.y, 1);
        const float4 row = bx ? make_float4(r0, r1, b.x, b.y) : make_float4(a.x, a.y, r0, r1);
        if (valid) store_out<OT>(hp, l + (int)bx, row);
      } else if (valid) {
        store_half<OT>(hp, l, bx, a);
      }
    }
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
  // two lanes per point; grid y: the level groups
  const LevelGroups LG = plan_level_groups(P, g->table_dtype == INPC_F32 ? 16 : 8);
  const long long cap = (long long)device_sm_count() * 16;
  const dim3 grid((unsigned)std::max<long long>(1, std::min<long long>((long long)ceil_div(2 * n, 256), cap)),
                  (unsigned)LG.n);
  TimedLaunch timed("k_hash_fwd", s);
  if (g->table_dtype == INPC_F32 && g->out_dtype == INPC_F32)
    k_hash_fwd<float, float><<<grid, 256, 0, s>>>(P, LG, (const float*)table, pos, n, (float*)h_out);
  else if (g->table_dtype == INPC_F32)
    k_hash_fwd<float, __nv_bfloat16><<<grid, 256, 0, s>>>(P, LG, (const float*)table, pos, n, (__nv_bfloat16*)h_out);
  else if (g->out_dtype == INPC_F32)
    k_hash_fwd<__nv_bfloat16, float><<<grid, 256, 0, s>>>(P, LG, (const __nv_bfloat16*)table, pos, n, (float*)h_out);
  else
    k_hash_fwd<__nv_bfloat16, __nv_bfloat16>
        <<<grid, 256, 0, s>>>(P, LG, (const __nv_bfloat16*)table, pos, n, (__nv_bfloat16*)h_out);
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
