// sample_static.cu -- inpc_sample_octree_noalloc: the octree sampler with its
// scratch in a fixed, file-scope device array instead of a caller-provided
// workspace, for callers that must not allocate device memory.
//
// The array is INPC_SAMPLE_STATIC_SCRATCH_BYTES long; every GPU that loads
// this library keeps it until the process exits.  In host code the array's
// name is only a host-side stand-in, so its device address is looked up
// (with the device current) on the first call in each CUDA context and
// cached per device together with that context's id; a call in another
// context of the same device (after cudaDeviceReset, for instance) looks it
// up again.  All calls on a device share the array: the sampler clears what
// must start at zero on every call, and calls whose GPU work overlaps (other
// streams or host threads) race.  The array's first word is the sampler's
// device status word, read by inpc_read_device_status with a null workspace.
#include <mutex>

#include "common.cuh"

namespace inpc {
namespace {

static __device__ __align__(256) unsigned char g_sample_scratch[INPC_SAMPLE_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct Cached {
  unsigned long long ctx_id;  // id of the CUDA context the address belongs to
  void* addr;
};
Cached g_addr[kMaxDevices] = {};

// The driver's cuCtxGetCurrent / cuCtxGetId, fetched through the runtime so
// that the library does not link libcuda directly.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

// Id of the current CUDA context (0 if the driver cannot tell).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

}  // namespace

// Device address of g_sample_scratch on the current device, looked up on the
// first call in the device's current context.
inpc_status noalloc_scratch_address(void** out) {
  int dev = -1;
  INPC_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(INPC_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  const unsigned long long id = current_context_id();  // 0 before the device's first runtime call
  if (!g_addr[dev].addr || id == 0 || id != g_addr[dev].ctx_id) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_sample_scratch);
    if (e != cudaSuccess || !p)
      return fail(INPC_ERR_CUDA, "cudaGetSymbolAddress(static sampler scratch): %s", cudaGetErrorString(e));
    // the lookup initialises the runtime's context if nothing had yet
    g_addr[dev] = Cached{id ? id : current_context_id(), p};
  }
  *out = g_addr[dev].addr;
  return INPC_OK;
}

}  // namespace inpc

extern "C" inpc_status inpc_sample_octree_noalloc(const inpc_octree* tree, uint64_t seed, uint32_t view_id,
                                                  int64_t n_samples, int32_t* leaf_idx_out, float* pos_out,
                                                  int32_t* leaf_counts_out, inpc_stream_t stream) {
  inpc::fault_arg(tree);
  if (!tree) return inpc::fail(INPC_ERR_INVALID_ARG, "inpc_sample_octree_noalloc: tree is null");
  size_t need = 0;
  INPC_TRY(inpc_sample_workspace_size(tree->n_leaves, n_samples, &need));
  if (need > (size_t)INPC_SAMPLE_STATIC_SCRATCH_BYTES)
    return inpc::fail(INPC_ERR_CAPACITY,
                      "inpc_sample_octree_noalloc: %lld leaves need %zu bytes of scratch, the static array holds %zu "
                      "(use inpc_sample_octree with a workspace)",
                      (long long)tree->n_leaves, need, (size_t)INPC_SAMPLE_STATIC_SCRATCH_BYTES);
  void* scratch = nullptr;
  INPC_TRY(inpc::noalloc_scratch_address(&scratch));
  return inpc_sample_octree(tree, seed, view_id, n_samples, leaf_idx_out, pos_out, leaf_counts_out, scratch,
                            (size_t)INPC_SAMPLE_STATIC_SCRATCH_BYTES, stream);
}
