// capi.cu -- library-wide C ABI entry points: error text, version, device
// status readback.
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace inpc {

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

void count_launches(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

void set_last_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

int device_sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  static std::mutex mu;
  static int cache[64] = {0};
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 0 || dev >= 64) return 148;
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    cache[dev] = n;
  }
  return cache[dev];
}

}  // namespace inpc

extern "C" const char* inpc_last_error(void) { return inpc::g_last_error.c_str(); }

extern "C" const char* inpc_version(void) { return "inpc-gb300 0.1 (sm_103a)"; }

extern "C" uint64_t inpc_kernel_launches(void) { return inpc::g_launches.load(); }

extern "C" inpc_status inpc_read_device_status(const void* workspace, inpc_stream_t stream, uint32_t* status_out) {
  if (!workspace || !status_out) return inpc::fail(INPC_ERR_INVALID_ARG, "inpc_read_device_status: null pointer");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  INPC_CUDA(cudaMemcpyAsync(&v, workspace, sizeof(v), cudaMemcpyDeviceToHost, s), "read status");
  INPC_CUDA(cudaStreamSynchronize(s), "read status sync");
  *status_out = v;
  return INPC_OK;
}
