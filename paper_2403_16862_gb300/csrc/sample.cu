// sample.cu -- octree point sampling (Sec. 3.2): exact quantised FP64 CDF,
// Philox4x32-10 draws with a guide-table CDF search, per-leaf counts, and
// leaf-grouped output slots with uniform in-leaf positions.
//
// Kernel sequence per call (one stream, no host synchronisation):
//   k_wmax        max weight + validation (atomicMax on the FP64 bit pattern)
//   k_scan_local  per-block inclusive scan of q_i = rint(w_i / wmax * 2^29)
//   k_scan_tops   exclusive scan of the block totals (one CTA)
//   k_scan_add    add block offsets -> cdf (exact integers in FP64)
//   k_guide       first leaf of every bucket of draw values
//   k_draw_count  draws -> leaf (search between two guide entries) -> counts
//   k_scan_*      exclusive scan of counts -> first output slot of each leaf
//   k_place       slot -> leaf (two-level search), Philox position
#include <algorithm>
#include <cmath>

#include <cuda_bf16.h>

#include "sample_impl.cuh"

namespace inpc {
namespace {

struct SampleWs {
  uint32_t* status;          // header word 0
  unsigned long long* wmax;  // header word 1 (FP64 bit pattern)
  double* cdf;               // [L]
  double* cdf_tops;          // [nb]
  uint32_t* counts;          // [L]
  uint32_t* starts;          // [L]
  uint32_t* count_tops;      // [nb]
  uint32_t* guide;           // [2^guide_log2(L) + 1]
  size_t bytes;
};

SampleWs carve(void* base, int64_t L) {
  Carver c(base);
  SampleWs w;
  w.status = reinterpret_cast<uint32_t*>(base);
  w.wmax = base ? reinterpret_cast<unsigned long long*>(static_cast<char*>(base) + 8) : nullptr;
  const int64_t nb = ceil_div(L, kScanBlock);
  w.cdf = c.take<double>(L);
  w.cdf_tops = c.take<double>(nb);
  w.counts = c.take<uint32_t>(L);
  w.starts = c.take<uint32_t>(L);
  w.count_tops = c.take<uint32_t>(nb);
  w.guide = c.take<uint32_t>((int64_t(1) << guide_log2(L)) + 1);
  w.bytes = c.bytes();
  return w;
}

__global__ void k_wmax(const double* __restrict__ w, int64_t L, unsigned long long* wmax, uint32_t* status) {
  double m = 0.0;
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = w[i];
    if (!(x >= 0.0) || isinf(x)) bad = true;
    else m = fmax(m, x);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_status(status, INPC_DEV_BAD_WEIGHT);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(wmax, (unsigned long long)__double_as_longlong(m));
}

// Loaders for the block scan: quantised weights, or plain counts.
struct QuantLoad {
  const double* w;
  const unsigned long long* wmax;
  __device__ double operator()(int64_t i) const {
    return quantised_weight(w[i], __longlong_as_double((long long)*wmax));
  }
};

struct CountLoad {
  const uint32_t* c;
  __device__ uint32_t operator()(int64_t i) const { return c[i]; }
};

template <class T>
__device__ T block_exclusive_scan(T v, T* warp_sums, T* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const T n = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += n;
  }
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    T s = lane < nw ? warp_sums[lane] : T(0);
    T si = s;
    for (int o = 1; o < 32; o <<= 1) {
      const T n = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += n;
    }
    if (lane < nw) warp_sums[lane] = si - s;
    if (lane == nw - 1) *total = si;
  }
  __syncthreads();
  const T r = warp_sums[wid] + incl - v;
  __syncthreads();
  return r;
}

// Per-block scan (inclusive or exclusive) of loader values into out[],
// block totals into tops[].
template <class T, class Load, bool kInclusive>
__global__ void __launch_bounds__(kScanThreads) k_scan_local(Load ld, int64_t L, T* __restrict__ out,
                                                             T* __restrict__ tops) {
  __shared__ T warp_sums[32];
  __shared__ T total;
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T run = T(0);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < L) ? ld(base + k) : T(0);
    run += v[k];
  }
  const T pre = block_exclusive_scan<T>(run, warp_sums, &total);
  T acc = pre;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (kInclusive) acc += v[k];
    if (base + k < L) out[base + k] = acc;
    if (!kInclusive) acc += v[k];
  }
  if (threadIdx.x == 0) tops[blockIdx.x] = total;
}

// Exclusive scan of the (at most kScanBlock * kScanBlock / kScanBlock) block totals in one CTA.
template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_tops(T* tops, int64_t nb) {
  __shared__ T warp_sums[32];
  __shared__ T total;
  T carry = T(0);
  for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
    const int64_t i = b0 + threadIdx.x;
    const T v = i < nb ? tops[i] : T(0);
    const T ex = block_exclusive_scan<T>(v, warp_sums, &total);
    if (i < nb) tops[i] = carry + ex;
    carry += total;
    __syncthreads();
  }
}

template <class T>
__global__ void k_scan_add(T* __restrict__ out, const T* __restrict__ tops, int64_t L) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < L) out[i] += tops[i / kScanBlock];
}

template <class T, class Load, bool kInclusive>
inpc_status scan(Load ld, int64_t L, T* out, T* tops, cudaStream_t s) {
  const int64_t nb = ceil_div(L, kScanBlock);
  k_scan_local<T, Load, kInclusive><<<(unsigned)nb, kScanThreads, 0, s>>>(ld, L, out, tops);
  k_scan_tops<T><<<1, kScanThreads, 0, s>>>(tops, nb);
  if (nb > 1) k_scan_add<T><<<(unsigned)ceil_div(L, 256), 256, 0, s>>>(out, tops, L);
  return check_launch("sample scan", nb > 1 ? 3 : 2);
}

// First leaf of every bucket of draw values (guide_entry).
__global__ void k_guide(const double* __restrict__ cdf, int64_t L, int Gl, uint32_t* __restrict__ guide) {
  const uint64_t Q = (uint64_t)cdf[L - 1];
  const int64_t G = int64_t(1) << Gl;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= G; j += (int64_t)gridDim.x * blockDim.x)
    guide[j] = guide_entry(LdPlain(), cdf, L, Gl, Q, j);
}

// Draws land on leaves at random, so a CTA's draws only repeat leaves when
// the tree is small: then they are counted in shared memory (one counter
// per leaf) and flushed once; otherwise each warp merges its equal leaves
// and adds to the global counts directly.
template <bool kSmem>
__global__ void __launch_bounds__(kDrawThreads) k_draw_count(const double* __restrict__ cdf, int64_t L,
                                                             const uint32_t* __restrict__ guide, int Gl,
                                                             int64_t n_draws, uint32_t k0, uint32_t k1,
                                                             uint32_t view_id, uint32_t* __restrict__ counts) {
  __shared__ uint32_t vals[kSmem ? kSmemLeaves : 1];
  if (kSmem) {
    for (int j = threadIdx.x; j < L; j += blockDim.x) vals[j] = 0;
    __syncthreads();
  }
  const uint64_t Qi = (uint64_t)cdf[L - 1];
  const int64_t base = (int64_t)blockIdx.x * kDrawPerCta;
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < kDrawPerThread; ++k) {
    const int64_t s = base + (int64_t)k * kDrawThreads + threadIdx.x;
    int leaf = -1;
    if (s < n_draws) leaf = (int)draw_leaf(LdPlain(), cdf, L, guide, Gl, Qi, s, view_id, k0, k1);
    const unsigned peers = __match_any_sync(0xffffffffu, leaf);
    if (leaf >= 0 && lane == __ffs(peers) - 1) {
      if (kSmem) atomicAdd(&vals[leaf], (uint32_t)__popc(peers));
      else atomicAdd(&counts[leaf], (uint32_t)__popc(peers));
    }
  }
  if (kSmem) {
    __syncthreads();
    for (int j = threadIdx.x; j < L; j += blockDim.x)
      if (vals[j]) atomicAdd(&counts[j], vals[j]);
  }
}

__global__ void __launch_bounds__(256) k_place(const uint32_t* __restrict__ starts, int64_t L, int stride_log2,
                                               int64_t n, uint32_t k0, uint32_t k1, uint32_t view_id,
                                               const float* __restrict__ centers,
                                               const int32_t* __restrict__ levels, float root_size,
                                               int32_t* __restrict__ leaf_out, float* __restrict__ pos_out) {
  __shared__ uint32_t coarse[kCoarse];
  int n_coarse;
  load_coarse(LdPlain(), starts, L, stride_log2, coarse, n_coarse);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    // leaf = (number of leaves whose first slot is <= k) - 1
    int64_t leaf = upper_bound2<uint32_t>(LdPlain(), starts, L, coarse, n_coarse, stride_log2, (uint32_t)k) - 1;
    if (leaf < 0) leaf = 0;
    place_slot(k, leaf, view_id, k0, k1, centers, levels, root_size, leaf_out, pos_out);
  }
}

__global__ void k_check_total(const double* cdf, int64_t L, uint32_t* status) {
  if (threadIdx.x == 0 && !(cdf[L - 1] > 0.0)) raise_status(status, INPC_DEV_NO_WEIGHT);
}

// ------------------------------------------------ view-specific sampling ---
// Eq. 4 per leaf: frustum culling of the leaf cube (all 8 corners outside
// one plane), view depth d = max(|z - near| / far, tau_d) of the center and
// the level factor 2^(l lambda_l) from a host table; FP64 with explicit
// round-to-nearest operations in a fixed order.
constexpr int kMaxViewLevel = 63;

struct LevelFactors {
  double f[kMaxViewLevel + 1];  // 2^(l lambda_l)
};

__device__ __forceinline__ double dmad(double a, double b, double c) { return __dadd_rn(__dmul_rn(a, b), c); }

__device__ __forceinline__ void cam_space_d(const Cam& c, const double x[3], double xc[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k)
    xc[k] = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn((double)c.R[3 * k], x[0]), __dmul_rn((double)c.R[3 * k + 1], x[1])),
                                __dmul_rn((double)c.R[3 * k + 2], x[2])),
                      (double)c.t[k]);
}

__global__ void k_view_weights(inpc_octree t, Cam cam, LevelFactors lf, double tau_d, double* __restrict__ w_out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < t.n_leaves;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int l = t.levels[i];
    if (l < 0 || l > kMaxViewLevel) {
      w_out[i] = 0.0;
      continue;
    }
    const double e = ldexp((double)t.root_size, -l);
    const double c[3] = {(double)t.centers[3 * i], (double)t.centers[3 * i + 1], (double)t.centers[3 * i + 2]};
    bool out[6] = {true, true, true, true, true, true};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double x[3] = {dmad((k & 1) ? 0.5 : -0.5, e, c[0]), dmad((k & 2) ? 0.5 : -0.5, e, c[1]),
                           dmad((k & 4) ? 0.5 : -0.5, e, c[2])};
      double xc[3];
      cam_space_d(cam, x, xc);
      if (!(xc[2] <= (double)cam.near_plane)) out[0] = false;
      if (!(xc[2] >= (double)cam.far_plane)) out[1] = false;
      if (!(__dadd_rn(__dmul_rn((double)cam.fx, xc[0]), __dmul_rn((double)cam.cx, xc[2])) < 0.0)) out[2] = false;
      if (!(__dadd_rn(__dmul_rn((double)cam.fx, xc[0]), __dmul_rn(__dsub_rn((double)cam.cx, (double)cam.W), xc[2])) >= 0.0))
        out[3] = false;
      if (!(__dadd_rn(__dmul_rn((double)cam.fy, xc[1]), __dmul_rn((double)cam.cy, xc[2])) < 0.0)) out[4] = false;
      if (!(__dadd_rn(__dmul_rn((double)cam.fy, xc[1]), __dmul_rn(__dsub_rn((double)cam.cy, (double)cam.H), xc[2])) >= 0.0))
        out[5] = false;
    }
    if (out[0] || out[1] || out[2] || out[3] || out[4] || out[5]) {
      w_out[i] = 0.0;
      continue;
    }
    double xc[3];
    cam_space_d(cam, c, xc);
    double d = __ddiv_rn(fabs(__dsub_rn(xc[2], (double)cam.near_plane)), (double)cam.far_plane);
    if (d < tau_d) d = tau_d;
    w_out[i] = __ddiv_rn(t.weights[i], __dmul_rn(d, lf.f[l]));
  }
}

// A sample is in view when the rasterizer's FP32 projection keeps it and it
// lands in [0, W) x [0, H).
__device__ __forceinline__ bool in_view(const Cam& c, const float* p) {
  float u, v, d;
  if (!project_point(c, p[0], p[1], p[2], u, v, d)) return false;
  return u >= 0.0f && u < (float)c.W && v >= 0.0f && v < (float)c.H;
}

// One re-sampling round: every sample not in view draws a new leaf from the
// CDF (Philox purpose 2 + 2 round) and a new position in it (3 + 2 round).
__global__ void k_resample_round(const double* __restrict__ cdf, int64_t L, const uint32_t* __restrict__ guide,
                                 int Gl, Cam cam, int64_t n, uint32_t k0,
                                 uint32_t k1, uint32_t view_id, uint32_t round, const float* __restrict__ centers,
                                 const int32_t* __restrict__ levels, float root_size, int32_t* __restrict__ leaf_out,
                                 float* __restrict__ pos_out) {
  const uint64_t Qi = (uint64_t)cdf[L - 1];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    if (in_view(cam, pos_out + 3 * k)) continue;
    const U32x4 r = philox4x32_10((uint32_t)k, (uint32_t)((uint64_t)k >> 32), view_id, 2u + 2u * round, k0, k1);
    const int64_t leaf = leaf_of_words(LdPlain(), cdf, L, guide, Gl, Qi, r);
    const U32x4 r2 = philox4x32_10((uint32_t)k, (uint32_t)((uint64_t)k >> 32), view_id, 3u + 2u * round, k0, k1);
    leaf_out[k] = (int32_t)leaf;
    leaf_position(r2, leaf, centers, levels, root_size, pos_out + 3 * k);
  }
}

__global__ void k_count_out_of_view(Cam cam, int64_t n, const float* __restrict__ pos, uint32_t* n_left) {
  uint32_t c = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    c += in_view(cam, pos + 3 * k) ? 0u : 1u;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(n_left, c);
}

// --------------------------------------------------------- pre-extraction ---
// Radical inverse of i in base b: the digits of i mirrored behind the radix
// point, as the exact fraction num / b^m (both below 2^53 for i < 2^31 and
// b <= 5), divided once.
__device__ __forceinline__ double radical_inverse(uint32_t b, uint64_t i) {
  uint64_t num = 0, den = 1;
  while (i > 0) {
    num = num * b + i % b;
    den *= b;
    i /= b;
  }
  return __ddiv_rn((double)num, (double)den);
}

// Slot k -> leaf (as k_place), then the Halton point of index (k - first
// slot of the leaf) + 1 in bases (2, 3, 5) inside the leaf, rounded once
// from FP64 to FP32.
__global__ void __launch_bounds__(256) k_place_halton(const uint32_t* __restrict__ starts, int64_t L,
                                                      int stride_log2, int64_t n, const float* __restrict__ centers,
                                                      const int32_t* __restrict__ levels, float root_size,
                                                      int32_t* __restrict__ leaf_out, float* __restrict__ pos_out) {
  __shared__ uint32_t coarse[kCoarse];
  int n_coarse;
  load_coarse(LdPlain(), starts, L, stride_log2, coarse, n_coarse);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t leaf = upper_bound2<uint32_t>(LdPlain(), starts, L, coarse, n_coarse, stride_log2, (uint32_t)k) - 1;
    if (leaf < 0) leaf = 0;
    const uint64_t j = (uint64_t)(k - (int64_t)starts[leaf]) + 1;
    const double edge = ldexp((double)root_size, -levels[leaf]);
    const uint32_t bases[3] = {2u, 3u, 5u};
    leaf_out[k] = (int32_t)leaf;
#pragma unroll
    for (int d = 0; d < 3; ++d)
      pos_out[3 * k + d] = __double2float_rn(
          __dadd_rn((double)centers[3 * leaf + d], __dmul_rn(__dsub_rn(radical_inverse(bases[d], j), 0.5), edge)));
  }
}

__global__ void k_level_weights(const int32_t* __restrict__ levels, const double* __restrict__ p, int64_t L,
                                LevelFactors lf, double* __restrict__ w_out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x) {
    const int l = levels[i];
    w_out[i] = (l < 0 || l > kMaxViewLevel) ? 0.0 : __ddiv_rn(p[i], lf.f[l]);
  }
}

// acc += scale * image (the per-pixel average of several feature images).
template <class T>
__global__ void k_accumulate(const T* __restrict__ img, float* __restrict__ acc, int64_t n, float scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc[i] = __fmaf_rn(scale, (float)img[i], acc[i]);
}


}  // namespace
}  // namespace inpc

using namespace inpc;

extern "C" inpc_status inpc_sample_workspace_size(int64_t n_leaves, int64_t n_samples, size_t* bytes) {
  if (inpc::fault_workspace_overflow())
    return inpc::fail(INPC_ERR_CAPACITY, "inpc_sample_workspace_size: size overflow (injected fault)");
  if (!bytes) return fail(INPC_ERR_INVALID_ARG, "inpc_sample_workspace_size: bytes is null");
  if (n_leaves < 1 || n_leaves > (int64_t(1) << 24))
    return fail(INPC_ERR_CAPACITY, "n_leaves must be in [1, 2^24], got %lld", (long long)n_leaves);
  if (n_samples < 0 || n_samples > INT32_MAX) return fail(INPC_ERR_CAPACITY, "n_samples out of range");
  *bytes = carve(nullptr, n_leaves).bytes;
  return INPC_OK;
}

namespace inpc {
namespace {
inpc_status sample_impl(const inpc_octree* tree, uint64_t seed, uint32_t view_id, int64_t n_samples,
                        int32_t* leaf_idx_out, float* pos_out, int32_t* leaf_counts_out, void* workspace,
                        size_t workspace_bytes, inpc_stream_t stream, bool halton);
}  // namespace
}  // namespace inpc

extern "C" inpc_status inpc_sample_octree(const inpc_octree* tree, uint64_t seed, uint32_t view_id,
                                          int64_t n_samples, int32_t* leaf_idx_out, float* pos_out,
                                          int32_t* leaf_counts_out, void* workspace, size_t workspace_bytes,
                                          inpc_stream_t stream) {
  inpc::fault_arg(tree);
  return sample_impl(tree, seed, view_id, n_samples, leaf_idx_out, pos_out, leaf_counts_out, workspace,
                     workspace_bytes, stream, false);
}

extern "C" inpc_status inpc_sample_octree_halton(const inpc_octree* tree, uint64_t seed, int64_t n_samples,
                                                 int32_t* leaf_idx_out, float* pos_out, int32_t* leaf_counts_out,
                                                 void* workspace, size_t workspace_bytes, inpc_stream_t stream) {
  inpc::fault_arg(tree);
  return sample_impl(tree, seed, 0u, n_samples, leaf_idx_out, pos_out, leaf_counts_out, workspace, workspace_bytes,
                     stream, true);
}

extern "C" inpc_status inpc_level_weights(const inpc_octree* tree, double lambda_l, double* w_out,
                                          inpc_stream_t stream) {
  inpc::fault_arg(tree);
  if (!tree || !tree->levels || !tree->weights || !w_out) return fail(INPC_ERR_INVALID_ARG, "null pointer");
  if (tree->n_leaves < 1 || tree->n_leaves > (int64_t(1) << 24))
    return fail(INPC_ERR_INVALID_ARG, "n_leaves must be in [1, 2^24]");
  if (!std::isfinite(lambda_l)) return fail(INPC_ERR_INVALID_ARG, "lambda_l must be finite");
  LevelFactors lf;
  for (int l = 0; l <= kMaxViewLevel; ++l) lf.f[l] = std::exp2((double)l * lambda_l);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t grid = std::min<int64_t>(ceil_div(tree->n_leaves, 256), (int64_t)device_sm_count() * 8);
  k_level_weights<<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(tree->levels, tree->weights, tree->n_leaves,
                                                                       lf, w_out);
  return check_launch("k_level_weights");
}

namespace inpc {
namespace {
__global__ void k_philox(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ ctrs, int64_t n,
                         uint32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const U32x4 r = philox4x32_10(ctrs[4 * i], ctrs[4 * i + 1], ctrs[4 * i + 2], ctrs[4 * i + 3], keys[2 * i],
                                  keys[2 * i + 1]);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
  }
}
}  // namespace
}  // namespace inpc

extern "C" inpc_status inpc_philox4x32_10(const uint32_t* keys, const uint32_t* ctrs, int64_t n, uint32_t* out,
                                          inpc_stream_t stream) {
  inpc::fault_arg(keys);
  if (n < 0) return fail(INPC_ERR_INVALID_ARG, "inpc_philox4x32_10: n < 0");
  if (n == 0) return INPC_OK;
  if (!keys || !ctrs || !out) return fail(INPC_ERR_INVALID_ARG, "inpc_philox4x32_10: null pointer");
  if (!aligned(keys, 4) || !aligned(ctrs, 4) || !aligned(out, 4))
    return fail(INPC_ERR_INVALID_ARG, "inpc_philox4x32_10: misaligned array");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t grid = std::min<int64_t>(ceil_div(n, 256), (int64_t)device_sm_count() * 8);
  k_philox<<<(unsigned)grid, 256, 0, s>>>(keys, ctrs, n, out);
  return check_launch("k_philox");
}

extern "C" inpc_status inpc_accumulate_image(const void* image, int32_t dtype, int64_t n_elems, float scale,
                                             float* acc, inpc_stream_t stream) {
  inpc::fault_arg(image);
  if (n_elems < 0) return fail(INPC_ERR_INVALID_ARG, "n_elems < 0");
  if (n_elems == 0) return INPC_OK;
  if (!image || !acc) return fail(INPC_ERR_INVALID_ARG, "null pointer");
  if (dtype != INPC_F32 && dtype != INPC_BF16) return fail(INPC_ERR_UNSUPPORTED, "dtype must be INPC_F32 or INPC_BF16");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const unsigned grid =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n_elems, 256), (int64_t)device_sm_count() * 16));
  if (dtype == INPC_F32) k_accumulate<float><<<grid, 256, 0, s>>>(static_cast<const float*>(image), acc, n_elems, scale);
  else
    k_accumulate<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(image), acc, n_elems, scale);
  return check_launch("k_accumulate");
}

namespace inpc {
namespace {
inpc_status sample_impl(const inpc_octree* tree, uint64_t seed, uint32_t view_id, int64_t n_samples,
                        int32_t* leaf_idx_out, float* pos_out, int32_t* leaf_counts_out, void* workspace,
                        size_t workspace_bytes, inpc_stream_t stream, bool halton) {
  if (!tree) return fail(INPC_ERR_INVALID_ARG, "inpc_sample_octree: tree is null");
  const int64_t L = tree->n_leaves;
  size_t need = 0;
  INPC_TRY(inpc_sample_workspace_size(L, n_samples, &need));
  if (!tree->centers || !tree->levels || !tree->weights)
    return fail(INPC_ERR_INVALID_ARG, "inpc_sample_octree: null octree array");
  if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
    return fail(INPC_ERR_INVALID_ARG, "inpc_sample_octree: workspace null, unaligned or smaller than %zu bytes", need);
  if (n_samples > 0 && (!leaf_idx_out || !pos_out))
    return fail(INPC_ERR_INVALID_ARG, "inpc_sample_octree: null output");
  if (!(tree->root_size > 0.0f)) return fail(INPC_ERR_INVALID_ARG, "root_size must be positive");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SampleWs ws = carve(workspace, L);
  INPC_CUDA(cudaMemsetAsync(workspace, 0, kHeaderBytes, s), "clear header");
  INPC_CUDA(cudaMemsetAsync(ws.counts, 0, sizeof(uint32_t) * L, s), "clear counts");
  const int sms = device_sm_count();
  k_wmax<<<(unsigned)std::min<int64_t>(ceil_div(L, 256), sms * 4), 256, 0, s>>>(tree->weights, L, ws.wmax, ws.status);
  INPC_TRY(check_launch("k_wmax"));
  INPC_TRY((scan<double, QuantLoad, true>(QuantLoad{tree->weights, ws.wmax}, L, ws.cdf, ws.cdf_tops, s)));
  k_check_total<<<1, 32, 0, s>>>(ws.cdf, L, ws.status);
  INPC_TRY(check_launch("k_check_total"));
  const int Gl = guide_log2(L);
  k_guide<<<(unsigned)std::min<int64_t>(ceil_div((int64_t(1) << Gl) + 1, 256), sms * 8), 256, 0, s>>>(ws.cdf, L, Gl,
                                                                                                     ws.guide);
  INPC_TRY(check_launch("k_guide"));
  const int sl = coarse_stride_log2(L);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  if (n_samples > 0) {
    const unsigned grid = (unsigned)ceil_div(n_samples, kDrawPerCta);
    if (L <= kSmemLeaves)
      INPC_TIMED("k_draw_count", s,
                 k_draw_count<true><<<grid, kDrawThreads, 0, s>>>(ws.cdf, L, ws.guide, Gl, n_samples, k0, k1, view_id,
                                                                  ws.counts));
    else
      INPC_TIMED("k_draw_count", s,
                 k_draw_count<false><<<grid, kDrawThreads, 0, s>>>(ws.cdf, L, ws.guide, Gl, n_samples, k0, k1,
                                                                   view_id, ws.counts));
    INPC_TRY(check_launch("k_draw_count"));
  }
  INPC_TRY((scan<uint32_t, CountLoad, false>(CountLoad{ws.counts}, L, ws.starts, ws.count_tops, s)));
  if (n_samples > 0) {
    const int64_t grid = std::min<int64_t>(ceil_div(n_samples, 256), (int64_t)sms * 16);
    if (halton) {
      INPC_TIMED("k_place_halton", s,
                 k_place_halton<<<(unsigned)grid, 256, 0, s>>>(ws.starts, L, sl, n_samples, tree->centers,
                                                               tree->levels, tree->root_size, leaf_idx_out, pos_out));
      INPC_TRY(check_launch("k_place_halton"));
    } else {
      INPC_TIMED("k_place", s,
                 k_place<<<(unsigned)grid, 256, 0, s>>>(ws.starts, L, sl, n_samples, k0, k1, view_id, tree->centers,
                                                        tree->levels, tree->root_size, leaf_idx_out, pos_out));
      INPC_TRY(check_launch("k_place"));
    }
  }
  if (leaf_counts_out)
    INPC_CUDA(cudaMemcpyAsync(leaf_counts_out, ws.counts, sizeof(uint32_t) * L, cudaMemcpyDeviceToDevice, s),
              "copy counts");
  return INPC_OK;
}
}  // namespace
}  // namespace inpc

extern "C" inpc_status inpc_view_weights(const inpc_octree* tree, const inpc_camera* cam, double lambda_l,
                                         double tau_d, double* w_out, inpc_stream_t stream) {
  inpc::fault_arg(tree);
  if (!tree || !cam || !w_out) return fail(INPC_ERR_INVALID_ARG, "inpc_view_weights: null pointer");
  if (!tree->centers || !tree->levels || !tree->weights)
    return fail(INPC_ERR_INVALID_ARG, "inpc_view_weights: null octree array");
  if (tree->n_leaves < 1 || tree->n_leaves > (int64_t(1) << 24))
    return fail(INPC_ERR_INVALID_ARG, "n_leaves must be in [1, 2^24]");
  if (!(tree->root_size > 0.0f)) return fail(INPC_ERR_INVALID_ARG, "root_size must be positive");
  if (!(cam->near_plane > 0.0f) || !(cam->far_plane > cam->near_plane) || cam->width < 1 || cam->height < 1)
    return fail(INPC_ERR_INVALID_ARG, "bad camera");
  if (!(tau_d > 0.0) || !std::isfinite(lambda_l)) return fail(INPC_ERR_INVALID_ARG, "need tau_d > 0, finite lambda_l");
  LevelFactors lf;
  for (int l = 0; l <= kMaxViewLevel; ++l) lf.f[l] = std::exp2((double)l * lambda_l);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t grid = std::min<int64_t>(ceil_div(tree->n_leaves, 256), (int64_t)device_sm_count() * 8);
  INPC_TIMED("k_view_weights", s,
             k_view_weights<<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(*tree, to_cam(*cam), lf, tau_d,
                                                                                w_out));
  return check_launch("k_view_weights");
}

extern "C" inpc_status inpc_sample_octree_view(const inpc_octree* tree, const inpc_camera* cam, uint64_t seed,
                                               uint32_t view_id, int64_t n_samples, int32_t max_rounds,
                                               int32_t* leaf_idx_out, float* pos_out, uint32_t* n_left,
                                               void* workspace, size_t workspace_bytes, inpc_stream_t stream) {
  inpc::fault_arg(tree);
  if (!cam) return fail(INPC_ERR_INVALID_ARG, "inpc_sample_octree_view: camera is null");
  if (max_rounds < 0 || max_rounds > 64) return fail(INPC_ERR_INVALID_ARG, "max_rounds must be in [0, 64]");
  if (!(cam->near_plane > 0.0f) || !(cam->far_plane > cam->near_plane) || cam->width < 1 || cam->height < 1)
    return fail(INPC_ERR_INVALID_ARG, "bad camera");
  INPC_TRY(inpc_sample_octree(tree, seed, view_id, n_samples, leaf_idx_out, pos_out, nullptr, workspace,
                              workspace_bytes, stream));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const SampleWs ws = carve(workspace, tree->n_leaves);
  const Cam c = to_cam(*cam);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ceil_div(n_samples, 256), (int64_t)device_sm_count() * 16));
  if (n_samples > 0)
    for (int32_t r = 0; r < max_rounds; ++r) {
      INPC_TIMED("k_resample_round", s,
                 k_resample_round<<<(unsigned)grid, 256, 0, s>>>(ws.cdf, tree->n_leaves, ws.guide,
                                                                guide_log2(tree->n_leaves), c, n_samples, k0, k1, view_id,
                                                                (uint32_t)r, tree->centers, tree->levels,
                                                                tree->root_size, leaf_idx_out, pos_out));
      INPC_TRY(check_launch("k_resample_round"));
    }
  if (n_left) {
    INPC_CUDA(cudaMemsetAsync(n_left, 0, sizeof(uint32_t), s), "clear n_left");
    if (n_samples > 0) {
      k_count_out_of_view<<<(unsigned)grid, 256, 0, s>>>(c, n_samples, pos_out, n_left);
      INPC_TRY(check_launch("k_count_out_of_view"));
    }
  }
  return INPC_OK;
}
