// calibrate.cu -- the L2 reduction rate of this GPU, the ceiling of the grid
// adjoint's table-gradient additions (inpc_l2_reduction_rate).  Measurement
// support for roofline reporting; not part of the method.
#include "common.cuh"

namespace inpc {
namespace {

constexpr int kCalThreads = 256;
constexpr int kCalIters = 128;

// Each lane draws rows from a linear congruential sequence of its own
// (uniform over the region) and adds (1, 1, 1, 1) there with one 16-byte
// vector reduction, under the evict_last policy the adjoint uses.  Paired:
// lane 2j + 1 takes lane 2j's row with the lowest bit flipped, so the pair
// covers one aligned 32-byte sector.
__global__ void __launch_bounds__(kCalThreads) k_l2_reduce(float* __restrict__ buf, uint32_t row_mask, int paired,
                                                           uint32_t seed) {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t h = (tid ^ seed) * 2654435761u + 12345u;
  for (int i = 0; i < kCalIters; ++i) {
    h = h * 1664525u + 1013904223u;
    uint32_t row = (h >> 7) & row_mask;
    if (paired) row = (__shfl_sync(0xffffffffu, row, lane & ~1u) & ~1u) | (lane & 1u);
    float* a = buf + 4ull * row;
    asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(1.f), "f"(1.f),
                 "f"(1.f), "f"(1.f), "l"(pol)
                 : "memory");
  }
}

}  // namespace
}  // namespace inpc

using namespace inpc;

extern "C" inpc_status inpc_l2_reduction_rate(float* buf, int64_t rows, int32_t paired, double* gops,
                                              inpc_stream_t stream) {
  inpc::fault_arg(buf);
  if (!buf || !gops) return fail(INPC_ERR_INVALID_ARG, "inpc_l2_reduction_rate: null pointer");
  if (!aligned(buf, 16)) return fail(INPC_ERR_INVALID_ARG, "inpc_l2_reduction_rate: buf must be 16-byte aligned");
  if (rows < (int64_t(1) << 10) || rows > (int64_t(1) << 26) || (rows & (rows - 1)) != 0)
    return fail(INPC_ERR_INVALID_ARG, "inpc_l2_reduction_rate: rows must be a power of two in [2^10, 2^26]");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int blocks = device_sm_count() * 8;
  const uint32_t mask = (uint32_t)(rows - 1);
  const int pr = paired ? 1 : 0;
  for (int w = 0; w < 2; ++w) k_l2_reduce<<<blocks, kCalThreads, 0, s>>>(buf, mask, pr, 7u + (uint32_t)w);
  INPC_TRY(check_launch("k_l2_reduce"));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(INPC_ERR_CUDA, "inpc_l2_reduction_rate: cudaEventCreate failed");
  }
  constexpr int kReps = 5;
  cudaEventRecord(e0, s);
  for (int r = 0; r < kReps; ++r) k_l2_reduce<<<blocks, kCalThreads, 0, s>>>(buf, mask, pr, 100u + (uint32_t)r);
  cudaEventRecord(e1, s);
  const cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return fail(INPC_ERR_CUDA, "inpc_l2_reduction_rate: %s", cudaGetErrorString(err));
  INPC_TRY(check_launch("k_l2_reduce"));
  const double lanes = (double)blocks * kCalThreads * kCalIters * kReps;
  *gops = ms > 0.f ? lanes / (ms * 1e-3) / 1e9 : 0.0;
  return INPC_OK;
}
