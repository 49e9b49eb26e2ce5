// raster_bwd.cu -- C ABI of the rasterizer backward (App. A.6).
#include "raster_impl.cuh"

using namespace inpc;

extern "C" inpc_status inpc_rasterize_bwd(const inpc_camera* cam, const inpc_raster_opts* opts, const float* pos,
                                          const float* opacity, const void* feat, int64_t n, const float* T_final,
                                          const int32_t* n_contrib, const float* d_image, float* d_opacity,
                                          float* d_feat, void* workspace, size_t workspace_bytes,
                                          inpc_stream_t stream) {
  RP P;
  INPC_TRY(make_rp(cam, opts, n, P));
  const RasterWs need = carve(nullptr, P.n_pix, n);
  if (!workspace || workspace_bytes < need.bytes || !aligned(workspace, 256))
    return fail(INPC_ERR_INVALID_ARG, "workspace null, unaligned or smaller than %zu bytes", need.bytes);
  if (n == 0) return INPC_OK;
  if (!pos || !feat || !T_final || !n_contrib || !d_image || !d_feat)
    return fail(INPC_ERR_INVALID_ARG, "null pointer");
  if (!P.head && (!opacity || !d_opacity)) return fail(INPC_ERR_INVALID_ARG, "opacity and d_opacity required");
  const size_t va = P.F % 4 == 0 ? 16 : 4;
  const size_t vf = P.F % 4 == 0 ? (P.bf16 ? 8 : 16) : (P.bf16 ? 2 : 4);
  if (!aligned(feat, vf) || !aligned(d_image, va) || !aligned(d_feat, va))
    return fail(INPC_ERR_INVALID_ARG, "feat/d_image/d_feat misaligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RasterWs ws = carve(workspace, P.n_pix, n);
  return dispatch(P.F, [&](auto Vc, auto Gc) {
    constexpr int V = decltype(Vc)::value, GA = decltype(Gc)::value;
    if constexpr (GA != 32) {
      if (P.bf16) return fail(INPC_ERR_UNSUPPORTED, "BF16 features need n_channels = 32, 64 or 128");
    } else if (P.bf16)
      return launch_bwd<V, GA, __nv_bfloat16>(P, pos, opacity, static_cast<const __nv_bfloat16*>(feat), n_contrib,
                                              d_image, ws, P.head ? nullptr : d_opacity, d_feat, s);
    return launch_bwd<V, GA, float>(P, pos, opacity, static_cast<const float*>(feat), n_contrib, d_image, ws,
                                    P.head ? nullptr : d_opacity, d_feat, s);
  });
}
