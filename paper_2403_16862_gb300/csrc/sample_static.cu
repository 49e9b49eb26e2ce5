// sample_static.cu -- inpc_sample_octree_noalloc: the octree sampler with its
// scratch in a fixed, file-scope device array instead of a caller-provided
// workspace, for callers that must not allocate device memory.
//
// The array is INPC_SAMPLE_STATIC_SCRATCH_BYTES long; every GPU that loads
// this library keeps it until the process exits.  In host code the array's
// name is only a host-side stand-in, so its device address is looked up once
// per device (with that device current) and cached.  All calls on a device
// share the array: the sampler clears what must start at zero on every call,
// and calls whose GPU work overlaps (other streams or host threads) race.
#include <mutex>

#include "common.cuh"

namespace inpc {
namespace {

static __device__ __align__(256) unsigned char g_sample_scratch[INPC_SAMPLE_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of g_sample_scratch on the current device (looked up on the
// first call for that device).
inpc_status scratch_address(void** out) {
  int dev = -1;
  INPC_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(INPC_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_sample_scratch);
    if (e != cudaSuccess || !p)
      return fail(INPC_ERR_CUDA, "cudaGetSymbolAddress(static sampler scratch): %s", cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return INPC_OK;
}

}  // namespace
}  // namespace inpc

extern "C" inpc_status inpc_sample_octree_noalloc(const inpc_octree* tree, uint64_t seed, uint32_t view_id,
                                                  int64_t n_samples, int32_t* leaf_idx_out, float* pos_out,
                                                  int32_t* leaf_counts_out, inpc_stream_t stream) {
  if (!tree) return inpc::fail(INPC_ERR_INVALID_ARG, "inpc_sample_octree_noalloc: tree is null");
  size_t need = 0;
  INPC_TRY(inpc_sample_workspace_size(tree->n_leaves, n_samples, &need));
  if (need > (size_t)INPC_SAMPLE_STATIC_SCRATCH_BYTES)
    return inpc::fail(INPC_ERR_CAPACITY,
                      "inpc_sample_octree_noalloc: %lld leaves need %zu bytes of scratch, the static array holds %zu "
                      "(use inpc_sample_octree with a workspace)",
                      (long long)tree->n_leaves, need, (size_t)INPC_SAMPLE_STATIC_SCRATCH_BYTES);
  void* scratch = nullptr;
  INPC_TRY(inpc::scratch_address(&scratch));
  return inpc_sample_octree(tree, seed, view_id, n_samples, leaf_idx_out, pos_out, leaf_counts_out, scratch,
                            (size_t)INPC_SAMPLE_STATIC_SCRATCH_BYTES, stream);
}
