// common.cuh -- helpers shared by the sm_103a kernels of the INPC hot path:
// error reporting, workspace carving, the Philox counter RNG and the FP32
// pinhole projection.  Nothing here is shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <cstdarg>
#include <string>

#include "../../include/inpc.h"

namespace inpc {

// ---------------------------------------------------------------- errors ---
void set_last_error(const char* fmt, ...);

inline inpc_status fail(inpc_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error("%s", buf);
  return st;
}

void count_launches(int k);

// Call once after each group of k kernel launches (k counted toward
// inpc_kernel_launches); reports a launch failure as INPC_ERR_CUDA.
inline inpc_status check_launch(const char* what, int k = 1) {
  count_launches(k);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(INPC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return INPC_OK;
}

// Per-kernel device timing (inpc_kernel_timer_enable/_read): while enabled,
// every launch made inside a TimedLaunch scope is bracketed by two CUDA
// events recorded on its stream.  Launches recorded into a CUDA graph are
// not timed.  Disabled, a scope costs one relaxed atomic load.
bool timer_enabled();
int timer_begin(const char* kernel, cudaStream_t s);
void timer_end(int rec, cudaStream_t s);

struct TimedLaunch {
  int rec = -1;
  cudaStream_t s;
  TimedLaunch(const char* kernel, cudaStream_t st) : s(st) {
    if (timer_enabled()) rec = timer_begin(kernel, st);
  }
  ~TimedLaunch() {
    if (rec >= 0) timer_end(rec, s);
  }
  TimedLaunch(const TimedLaunch&) = delete;
  TimedLaunch& operator=(const TimedLaunch&) = delete;
};

// Launch statement(s) under a TimedLaunch named `kernel`.
#define INPC_TIMED(kernel, stream, ...)               \
  do {                                                \
    ::inpc::TimedLaunch _timed_launch(kernel, stream); \
    __VA_ARGS__;                                      \
  } while (0)

#define INPC_TRY(expr)                 \
  do {                                 \
    inpc_status _st = (expr);          \
    if (_st != INPC_OK) return _st;    \
  } while (0)

#define INPC_CUDA(expr, what)                                                              \
  do {                                                                                     \
    cudaError_t _e = (expr);                                                               \
    if (_e != cudaSuccess) return ::inpc::fail(INPC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(_e)); \
  } while (0)

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// ------------------------------------------------------------- workspace ---
// Every workspace starts with a 256-byte header; word 0 is the device status.
constexpr size_t kHeaderBytes = 256;

struct Carver {
  char* base;
  size_t off = kHeaderBytes;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  size_t bytes() const { return (off + 255) & ~size_t(255); }
};

__device__ __forceinline__ void raise_status(uint32_t* status, uint32_t bits) { atomicOr(status, bits); }

// ------------------------------------------------------------------ RNG ---
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications; the high halves are xored with the other two
// counter words and the round key, and the key advances by the Weyl
// increments between rounds.
struct U32x4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                               uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo_a = 0xD2511F53u * c0;
    const uint32_t hi_a = __umulhi(0xD2511F53u, c0);
    const uint32_t lo_b = 0xCD9E8D57u * c2;
    const uint32_t hi_b = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi_b ^ c1 ^ k0;
    const uint32_t n2 = hi_a ^ c3 ^ k1;
    c0 = n0;
    c1 = lo_b;
    c2 = n2;
    c3 = lo_a;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U32x4{c0, c1, c2, c3};
}

// ------------------------------------------------------------ projection ---
struct Cam {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int W, H;
  float near_plane, far_plane;
};

inline Cam to_cam(const inpc_camera& c) {
  Cam k;
  for (int i = 0; i < 9; ++i) k.R[i] = c.R[i];
  for (int i = 0; i < 3; ++i) k.t[i] = c.t[i];
  k.fx = c.fx; k.fy = c.fy; k.cx = c.cx; k.cy = c.cy;
  k.W = c.width; k.H = c.height;
  k.near_plane = c.near_plane; k.far_plane = c.far_plane;
  return k;
}

// Eq. 5 in FP32 with the operation order fixed by the ABI (explicit
// round-to-nearest intrinsics so the compiler cannot contract or reorder).
// Returns false for culled points (outside the near/far slab or NaN).
__device__ __forceinline__ bool project_point(const Cam& c, float x, float y, float z, float& u, float& v,
                                              float& d) {
  const float xc = __fmaf_rn(c.R[2], z, __fmaf_rn(c.R[1], y, __fmaf_rn(c.R[0], x, c.t[0])));
  const float yc = __fmaf_rn(c.R[5], z, __fmaf_rn(c.R[4], y, __fmaf_rn(c.R[3], x, c.t[1])));
  const float zc = __fmaf_rn(c.R[8], z, __fmaf_rn(c.R[7], y, __fmaf_rn(c.R[6], x, c.t[2])));
  d = zc;
  if (!(zc > c.near_plane && zc < c.far_plane)) return false;
  u = __fmaf_rn(c.fx, __fdiv_rn(xc, zc), c.cx);
  v = __fmaf_rn(c.fy, __fdiv_rn(yc, zc), c.cy);
  return true;
}

// Bilinear footprint of a projected point (Eq. 6): top-left pixel (i0, j0)
// of the 2x2 nearest centers and the fractional offsets fu, fv in [0, 1);
// the corner (i0 + a, j0 + b) has weight (a ? fu : 1 - fu) * (b ? fv : 1 - fv).
// Returns false if no corner can touch the image.
struct Footprint {
  int i0, j0;
  float fu, fv;
};

__device__ __forceinline__ bool footprint(const Cam& c, float u, float v, Footprint& f) {
  if (!(u >= -0.5f && u < (float)c.W + 0.5f && v >= -0.5f && v < (float)c.H + 0.5f)) return false;
  const float su = __fsub_rn(u, 0.5f);
  const float sv = __fsub_rn(v, 0.5f);
  const float fi = floorf(su);
  const float fj = floorf(sv);
  f.i0 = (int)fi;
  f.j0 = (int)fj;
  f.fu = __fsub_rn(su, fi);
  f.fv = __fsub_rn(sv, fj);
  return true;
}

__device__ __forceinline__ float corner_weight(const Footprint& f, int a, int b) {
  const float wu = a ? f.fu : __fsub_rn(1.0f, f.fu);
  const float wv = b ? f.fv : __fsub_rn(1.0f, f.fv);
  return __fmul_rn(wu, wv);
}

// ----------------------------------------------------------- small utils ---
__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

int device_sm_count();

// Host-side fault injection (faults.cu, inpc_set_fault): size queries that
// report an overflow, and a first array argument corrupted to NULL at the
// entry of every compute call, which the call's own validation must catch.
bool fault_workspace_overflow();
bool fault_corrupt_args();
template <class T>
inline void fault_arg(T*& p) {
  if (fault_corrupt_args()) p = nullptr;
}

// Device address of the allocation-free sampler's static scratch array on the
// current device (sample_static.cu); its first word is that sampler's status.
inpc_status noalloc_scratch_address(void** out);

}  // namespace inpc
