// head.cu -- the view-dependent appearance head (Sec. 3.3): spherical
// contraction of the query positions into [0, 1]^3 (mip-NeRF 360), and per
// point the opacity alpha_h = 1 - exp(-exp(h0)) with a 4D color from degree-2
// real spherical harmonics of the viewing direction on the next 36 features
// (channel c uses h[1 + 9 c + k], k < 9), plus its derivative.
//
// The head is evaluated once per point before the rasterizer (which then
// blends 4 channels with given opacities) instead of once per splat inside
// the blend: the point's 37 features are read once, not four times.
#include <cmath>

#include <cuda_bf16.h>

#include "common.cuh"

namespace inpc {
namespace {

struct ShConsts {
  float c0, c1, c2, c20, c22;  // sqrt(1/4pi), sqrt(3/4pi), sqrt(15/4pi), sqrt(5/16pi), sqrt(15/16pi)
  double o[3];                 // camera center -R^T t
};

ShConsts make_consts(const inpc_camera& cam) {
  const double pi = std::acos(-1.0);
  ShConsts k;
  k.c0 = (float)std::sqrt(1.0 / (4.0 * pi));
  k.c1 = (float)std::sqrt(3.0 / (4.0 * pi));
  k.c2 = (float)std::sqrt(15.0 / (4.0 * pi));
  k.c20 = (float)std::sqrt(5.0 / (16.0 * pi));
  k.c22 = (float)std::sqrt(15.0 / (16.0 * pi));
  for (int a = 0; a < 3; ++a)
    k.o[a] = -((double)cam.R[a] * cam.t[0] + (double)cam.R[3 + a] * cam.t[1] + (double)cam.R[6 + a] * cam.t[2]);
  return k;
}

// The direction is formed in FP64: x - o cancels for points near a
// coordinate plane through the camera, and FP32 would lose the small
// component's relative accuracy there.
__device__ __forceinline__ void sh9(const ShConsts& k, const float* p, float Y[9]) {
  const double vx = (double)p[0] - k.o[0], vy = (double)p[1] - k.o[1], vz = (double)p[2] - k.o[2];
  const double len = sqrt(vx * vx + vy * vy + vz * vz);
  float x = 0.f, y = 0.f, z = 1.f;
  if (len > 0.0) {
    x = (float)(vx / len);
    y = (float)(vy / len);
    z = (float)(vz / len);
  }
  Y[0] = k.c0;
  Y[1] = k.c1 * y;
  Y[2] = k.c1 * z;
  Y[3] = k.c1 * x;
  Y[4] = k.c2 * x * y;
  Y[5] = k.c2 * y * z;
  Y[6] = k.c20 * fmaf(3.f * z, z, -1.f);
  Y[7] = k.c2 * x * z;
  Y[8] = k.c22 * (x * x - y * y);
}

__device__ __forceinline__ float ldf(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) {
  return __uint_as_float(((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p))) << 16);
}

__global__ void k_contract(const float* __restrict__ pos, int64_t n, float cx, float cy, float cz, float radius,
                           float* __restrict__ out) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const float y0 = __fdiv_rn(__fsub_rn(pos[3 * p + 0], cx), radius);
    const float y1 = __fdiv_rn(__fsub_rn(pos[3 * p + 1], cy), radius);
    const float y2 = __fdiv_rn(__fsub_rn(pos[3 * p + 2], cz), radius);
    const float r = __fsqrt_rn(__fmaf_rn(y2, y2, __fmaf_rn(y1, y1, __fmul_rn(y0, y0))));
    float sc = 1.0f;
    if (r > 1.0f) sc = __fdiv_rn(__fsub_rn(2.0f, __fdiv_rn(1.0f, r)), r);
    out[3 * p + 0] = __fmaf_rn(__fmul_rn(y0, sc), 0.25f, 0.5f);
    out[3 * p + 1] = __fmaf_rn(__fmul_rn(y1, sc), 0.25f, 0.5f);
    out[3 * p + 2] = __fmaf_rn(__fmul_rn(y2, sc), 0.25f, 0.5f);
  }
}

template <class HT>
__global__ void k_sh_head_fwd(ShConsts k, const float* __restrict__ pos, const HT* __restrict__ h, int64_t n, int F,
                              float* __restrict__ alpha, float* __restrict__ color) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    float Y[9];
    sh9(k, pos + 3 * p, Y);
    const HT* row = h + (int64_t)F * p;
    alpha[p] = -expm1f(-expf(ldf(row)));
    float c[4];
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      float s = 0.f;
#pragma unroll
      for (int b = 0; b < 9; ++b) s = fmaf(Y[b], ldf(row + 1 + 9 * ch + b), s);
      c[ch] = s;
    }
    reinterpret_cast<float4*>(color)[p] = make_float4(c[0], c[1], c[2], c[3]);
  }
}

template <class HT>
__global__ void k_sh_head_bwd(ShConsts k, const float* __restrict__ pos, const HT* __restrict__ h, int64_t n, int F,
                              const float* __restrict__ d_alpha, const float* __restrict__ d_color,
                              float* __restrict__ dh) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    float Y[9];
    sh9(k, pos + 3 * p, Y);
    float* out = dh + (int64_t)F * p;
    const float e = expf(ldf(h + (int64_t)F * p));
    out[0] = d_alpha[p] * (e * expf(-e));
    const float4 g = reinterpret_cast<const float4*>(d_color)[p];
    const float gc[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
    for (int ch = 0; ch < 4; ++ch)
#pragma unroll
      for (int b = 0; b < 9; ++b) out[1 + 9 * ch + b] = Y[b] * gc[ch];
    for (int f = 37; f < F; ++f) out[f] = 0.f;
  }
}

unsigned grid_for_points(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)device_sm_count() * 16));
}

inpc_status check_head(const inpc_camera* cam, const float* pos, const void* h, int32_t dtype, int64_t n, int32_t F) {
  if (!cam) return fail(INPC_ERR_INVALID_ARG, "camera is null");
  if (n < 0) return fail(INPC_ERR_INVALID_ARG, "n < 0");
  if (F < 37) return fail(INPC_ERR_INVALID_ARG, "the SH head needs n_channels >= 37 (1 opacity + 36 SH)");
  if (dtype != INPC_F32 && dtype != INPC_BF16) return fail(INPC_ERR_UNSUPPORTED, "dtype must be INPC_F32 or INPC_BF16");
  if (n > 0 && (!pos || !h)) return fail(INPC_ERR_INVALID_ARG, "null pointer");
  return INPC_OK;
}

}  // namespace
}  // namespace inpc

using namespace inpc;

extern "C" inpc_status inpc_contract_positions(const float* pos, int64_t n, const float* center, float radius,
                                               float* out, inpc_stream_t stream) {
  inpc::fault_arg(pos);
  if (n < 0) return fail(INPC_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return INPC_OK;
  if (!pos || !center || !out) return fail(INPC_ERR_INVALID_ARG, "null pointer");
  if (!(radius > 0.0f)) return fail(INPC_ERR_INVALID_ARG, "radius must be positive");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_contract<<<grid_for_points(n), 256, 0, s>>>(pos, n, center[0], center[1], center[2], radius, out);
  return check_launch("k_contract");
}

extern "C" inpc_status inpc_sh_head_fwd(const inpc_camera* cam, const float* pos, const void* h, int32_t h_dtype,
                                        int64_t n, int32_t n_channels, float* alpha_out, float* color_out,
                                        inpc_stream_t stream) {
  inpc::fault_arg(pos);
  INPC_TRY(check_head(cam, pos, h, h_dtype, n, n_channels));
  if (n == 0) return INPC_OK;
  if (!alpha_out || !color_out || !aligned(color_out, 16)) return fail(INPC_ERR_INVALID_ARG, "bad output pointer");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const ShConsts k = make_consts(*cam);
  if (h_dtype == INPC_F32)
    k_sh_head_fwd<float><<<grid_for_points(n), 256, 0, s>>>(k, pos, static_cast<const float*>(h), n, n_channels,
                                                             alpha_out, color_out);
  else
    k_sh_head_fwd<__nv_bfloat16><<<grid_for_points(n), 256, 0, s>>>(k, pos, static_cast<const __nv_bfloat16*>(h), n,
                                                                     n_channels, alpha_out, color_out);
  return check_launch("k_sh_head_fwd");
}

extern "C" inpc_status inpc_sh_head_bwd(const inpc_camera* cam, const float* pos, const void* h, int32_t h_dtype,
                                        int64_t n, int32_t n_channels, const float* d_alpha, const float* d_color,
                                        float* dh_out, inpc_stream_t stream) {
  inpc::fault_arg(pos);
  INPC_TRY(check_head(cam, pos, h, h_dtype, n, n_channels));
  if (n == 0) return INPC_OK;
  if (!d_alpha || !d_color || !dh_out || !aligned(d_color, 16)) return fail(INPC_ERR_INVALID_ARG, "bad pointer");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const ShConsts k = make_consts(*cam);
  if (h_dtype == INPC_F32)
    k_sh_head_bwd<float><<<grid_for_points(n), 256, 0, s>>>(k, pos, static_cast<const float*>(h), n, n_channels,
                                                             d_alpha, d_color, dh_out);
  else
    k_sh_head_bwd<__nv_bfloat16><<<grid_for_points(n), 256, 0, s>>>(k, pos, static_cast<const __nv_bfloat16*>(h), n,
                                                                     n_channels, d_alpha, d_color, dh_out);
  return check_launch("k_sh_head_bwd");
}
