// capi.cu -- library-wide C ABI entry points: error text, version, device
// status readback.
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

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

// ---------------------------------------------------------- kernel timer ---
namespace {
struct TimerRec {
  const char* kernel;  // a string literal at the launch site
  cudaEvent_t a, b;
  bool done;           // timer_end recorded b
};
std::atomic<bool> g_timer_on{false};
std::mutex g_timer_mu;
std::vector<TimerRec> g_timer_recs;
std::vector<cudaEvent_t> g_timer_pool;

cudaEvent_t pooled_event() {
  if (!g_timer_pool.empty()) {
    cudaEvent_t e = g_timer_pool.back();
    g_timer_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

bool timer_enabled() { return g_timer_on.load(std::memory_order_relaxed); }

int timer_begin(const char* kernel, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return -1;
  std::lock_guard<std::mutex> lk(g_timer_mu);
  if (g_timer_recs.size() >= (1u << 20)) return -1;  // bounded: unread records are dropped
  TimerRec r{kernel, pooled_event(), pooled_event(), false};
  if (!r.a || !r.b || cudaEventRecord(r.a, s) != cudaSuccess) {
    if (r.a) g_timer_pool.push_back(r.a);
    if (r.b) g_timer_pool.push_back(r.b);
    return -1;
  }
  g_timer_recs.push_back(r);
  return (int)g_timer_recs.size() - 1;
}

void timer_end(int rec, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_timer_mu);
  if (rec < 0 || rec >= (int)g_timer_recs.size()) return;
  TimerRec& r = g_timer_recs[rec];
  r.done = cudaEventRecord(r.b, s) == cudaSuccess;
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
  if (!status_out) return inpc::fail(INPC_ERR_INVALID_ARG, "inpc_read_device_status: status_out is null");
  if (!workspace) {
    // the allocation-free sampler's status word: the first word of its static
    // scratch array on the current device
    void* p = nullptr;
    INPC_TRY(inpc::noalloc_scratch_address(&p));
    workspace = p;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  INPC_CUDA(cudaMemcpyAsync(&v, workspace, sizeof(v), cudaMemcpyDeviceToHost, s), "read status");
  INPC_CUDA(cudaStreamSynchronize(s), "read status sync");
  *status_out = v;
  return INPC_OK;
}

extern "C" int inpc_kernel_timer_enable(int on) {
  return inpc::g_timer_on.exchange(on != 0) ? 1 : 0;
}

extern "C" inpc_status inpc_kernel_timer_read(const char* kernel, double* total_ms, int64_t* launches) {
  using namespace inpc;
  if (!total_ms || !launches) return fail(INPC_ERR_INVALID_ARG, "inpc_kernel_timer_read: null pointer");
  std::lock_guard<std::mutex> lk(g_timer_mu);
  double ms_sum = 0.0;
  int64_t count = 0;
  std::vector<TimerRec> keep;
  for (TimerRec& r : g_timer_recs) {
    const bool match = !kernel || std::strcmp(kernel, r.kernel) == 0;
    if (!match) {
      keep.push_back(r);
      continue;
    }
    if (r.done) {
      float ms = 0.f;
      if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
        return fail(INPC_ERR_CUDA, "inpc_kernel_timer_read: %s", cudaGetErrorString(cudaGetLastError()));
      ms_sum += ms;
      ++count;
    }
    g_timer_pool.push_back(r.a);
    g_timer_pool.push_back(r.b);
  }
  // records handed out by timer_begin index this vector; read only between
  // launches (no TimedLaunch scope open), as the header states
  g_timer_recs.swap(keep);
  *total_ms = ms_sum;
  *launches = count;
  return INPC_OK;
}
