// raster_fwd.cu -- C ABI of the rasterizer forward (Sec. 3.4, Algorithm 1).
#include "raster_impl.cuh"

using namespace inpc;

extern "C" inpc_status inpc_rasterize_workspace_size(const inpc_camera* cam, const inpc_raster_opts* opts, int64_t n,
                                                     size_t* bytes) {
  if (inpc::fault_workspace_overflow())
    return inpc::fail(INPC_ERR_CAPACITY, "inpc_rasterize_workspace_size: size overflow (injected fault)");
  if (!bytes) return fail(INPC_ERR_INVALID_ARG, "bytes is null");
  RP P;
  INPC_TRY(make_rp(cam, opts, n, P, kMaxFwdPoints));
  *bytes = carve(nullptr, P.n_pix, n).bytes;
  return INPC_OK;
}

extern "C" inpc_status inpc_rasterize_fwd(const inpc_camera* cam, const inpc_raster_opts* opts, const float* pos,
                                          const float* opacity, const void* feat, int64_t n, void* image,
                                          float* T_final, int32_t* n_contrib, void* workspace,
                                          size_t workspace_bytes, inpc_stream_t stream) {
  inpc::fault_arg(pos);
  RP P;
  INPC_TRY(make_rp(cam, opts, n, P, kMaxFwdPoints));
  const RasterWs need = carve(nullptr, P.n_pix, n);
  if (!workspace || workspace_bytes < need.bytes || !aligned(workspace, 256))
    return fail(INPC_ERR_INVALID_ARG, "workspace null, unaligned or smaller than %zu bytes", need.bytes);
  if (!image || !T_final || !n_contrib) return fail(INPC_ERR_INVALID_ARG, "null output");
  if (n > 0 && (!pos || !feat)) return fail(INPC_ERR_INVALID_ARG, "null pos or feat");
  if (n > 0 && !P.head && !opacity) return fail(INPC_ERR_INVALID_ARG, "opacity required in INPC_OPACITY_GIVEN mode");
  const size_t va = P.F % 4 == 0 ? (P.bf16 && P.F != 64 ? 8 : 16) : (P.bf16 ? 2 : 4);
  if (!aligned(feat, va) || !aligned(image, va) || !aligned(pos, 4))
    return fail(INPC_ERR_INVALID_ARG, "feat/image must be %zu-byte aligned", va);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RasterWs ws = carve(workspace, P.n_pix, n);
  INPC_CUDA(cudaMemsetAsync(workspace, 0, kHeaderBytes, s), "clear header");
  return dispatch(P.F, [&](auto Vc, auto Gc) {
    constexpr int V = decltype(Vc)::value, GA = decltype(Gc)::value;
    if constexpr (GA != 32) {
      if (P.bf16) return fail(INPC_ERR_UNSUPPORTED, "BF16 features need n_channels = 32, 64 or 128");
    } else if (P.bf16)
      return launch_fwd<V, GA, __nv_bfloat16>(P, pos, opacity, static_cast<const __nv_bfloat16*>(feat), ws,
                                              static_cast<__nv_bfloat16*>(image), T_final, n_contrib, s);
    return launch_fwd<V, GA, float>(P, pos, opacity, static_cast<const float*>(feat), ws, static_cast<float*>(image),
                                    T_final, n_contrib, s);
  });
}

