// sample_impl.cuh -- the octree sampler's per-item arithmetic (Sec. 3.2),
// shared by the per-view sampling kernels (sample.cu) and the persistent
// multi-view kernel (batch_front.cu), so that both give bit-identical
// draws, counts and positions.
//
//   q_i  = rint(w_i / max w * 2^29), cdf = their exact prefix sum (FP64)
//   draw s: Philox(counter = (s lo, s hi, view, 0)) -> 53-bit b -> value
//           floor(b Q / 2^53) -> leaf = smallest i with cdf_i > value,
//           searched between two guide-table entries
//   slot k: leaf = last leaf whose first slot is <= k; position from
//           Philox(counter = (k lo, k hi, view, 1)), rounded once to FP32
#pragma once

#include "common.cuh"

namespace inpc {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanBlock = kScanThreads * kScanItems;  // 2048 items per CTA
constexpr int kCoarse = 2048;                          // coarse search table entries (shared memory)
constexpr int kDrawThreads = 256;
constexpr int kDrawPerThread = 16;
constexpr int kDrawPerCta = kDrawThreads * kDrawPerThread;
constexpr int kSmemLeaves = 4096;  // trees up to this many leaves count their draws in shared memory

// Loads of the sampler's search arrays.  Arrays written by an earlier kernel
// are read with plain loads; the persistent kernel reads arrays that other
// CTAs wrote earlier in the same launch through L2 only (never a stale L1
// line).
struct LdPlain {
  template <class T>
  __device__ __forceinline__ T operator()(const T* p) const { return *p; }
};
struct LdL2 {
  template <class T>
  __device__ __forceinline__ T operator()(const T* p) const { return __ldcg(p); }
};

// Draw buckets: the top guide_log2(L) bits of a draw's 53-bit random number
// (about two leaves per bucket).
inline int guide_log2(int64_t L) {
  int f = 0;
  while ((int64_t(1) << (f + 1)) <= L) ++f;  // floor(log2 L)
  return f > 0 ? f - 1 : 0;
}

inline int coarse_stride_log2(int64_t L) {
  int s = 0;
  while (ceil_div(L, (int64_t)1 << s) > kCoarse) ++s;
  return s;
}

// Quantised weight of one leaf (0 for an invalid weight, which the max pass
// flags; the scan only needs a defined value).
__device__ __forceinline__ double quantised_weight(double x, double m) {
  if (!(m > 0.0)) return 0.0;
  if (!(x >= 0.0) || isinf(x)) return 0.0;
  return rint(ldexp(__ddiv_rn(x, m), 29));
}

// Order key of a searched value.  The CDF holds exact non-negative integers
// as doubles, and non-negative doubles order like their IEEE-754 bit
// patterns read as unsigned integers, so the searches compare 64-bit
// integers (the same decisions, without the narrow FP64 pipe).
__device__ __forceinline__ uint64_t ord(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ uint32_t ord(uint32_t x) { return x; }

// Two-level search tables: the last element of every stride-sized block
// sits in shared memory, the rest is searched in global memory (L2).
// Every thread of the block calls it (one barrier).
template <class T, class Ld>
__device__ __forceinline__ void load_coarse(Ld ld, const T* __restrict__ arr, int64_t L, int stride_log2, T* coarse,
                                            int& n_coarse) {
  n_coarse = (int)ceil_div(L, (int64_t)1 << stride_log2);
  for (int j = threadIdx.x; j < n_coarse; j += blockDim.x) {
    int64_t e = (((int64_t)j + 1) << stride_log2) - 1;
    coarse[j] = ld(arr + (e < L ? e : L - 1));
  }
  __syncthreads();
}

// Smallest i with arr[i] > key (arr non-decreasing, non-negative); L when none.
template <class T, class Ld>
__device__ __forceinline__ int64_t upper_bound2(Ld ld, const T* __restrict__ arr, int64_t L, const T* coarse,
                                                int n_coarse, int stride_log2, T key_value) {
  const auto key = ord(key_value);
  int lo = 0, hi = n_coarse;  // first coarse block whose last element exceeds key
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (ord(coarse[mid]) > key) hi = mid; else lo = mid + 1;
  }
  if (lo == n_coarse) return L;
  int64_t a = (int64_t)lo << stride_log2;
  int64_t b = a + ((int64_t)1 << stride_log2) - 1;
  if (b > L - 1) b = L - 1;
  while (a < b) {  // arr[b] > key holds
    const int64_t mid = (a + b) >> 1;
    if (ord(ld(arr + mid)) > key) b = mid; else a = mid + 1;
  }
  return a;
}

// Guide table entry j (an indexed search): a draw's value r = floor(b Q /
// 2^53) from the 53-bit random b lies, for b in bucket j = b >> (53 - G_l),
// in [floor(j Q / 2^G_l), floor((j + 1) Q / 2^G_l)], and the leaf of r (the
// smallest i with cdf[i] > r) is monotone in r, so guide[j] = the leaf of
// floor(j Q / 2^G_l) and guide[j + 1] bound it.  The bucket bounds are
// formed exactly from the 128-bit product j Q.
template <class Ld>
__device__ __forceinline__ uint32_t guide_entry(Ld ld, const double* __restrict__ cdf, int64_t L, int Gl,
                                                uint64_t Q, int64_t j) {
  const uint64_t pl = (uint64_t)j * Q, ph = __umul64hi((uint64_t)j, Q);
  const uint64_t lo = Gl == 0 ? pl : ((ph << (64 - Gl)) | (pl >> Gl));
  const uint64_t key = ord((double)lo);  // lo <= Q <= 2^53: exact
  int64_t a = 0, z = L;                  // smallest i with cdf[i] > lo; L when none
  while (a < z) {
    const int64_t mid = (a + z) >> 1;
    if (ord(ld(cdf + mid)) > key) z = mid; else a = mid + 1;
  }
  return (uint32_t)a;
}

// Leaf of a draw: the smallest i with cdf[i] > r (key = the bits of r as a
// double), searched between the guide entries of the draw's bucket j.
// Returns L only when Q == 0 (flagged as a device status).
template <class Ld>
__device__ __forceinline__ int64_t guided_leaf(Ld ld, const double* __restrict__ cdf, int64_t L,
                                               const uint32_t* __restrict__ guide, uint32_t j, uint64_t key) {
  int64_t a = ld(guide + j), z = ld(guide + j + 1);
  if (z > L - 1) z = L - 1;
  while (a < z) {  // cdf[z] > r holds
    const int64_t mid = (a + z) >> 1;
    if (ord(ld(cdf + mid)) > key) z = mid; else a = mid + 1;
  }
  return a;
}

// Leaf drawn for random words (r.x, r.y): b = 53 bits, value floor(b Q /
// 2^53) from the exact 106-bit product, clamped to L - 1 (reachable only
// when Q == 0, which is flagged).
template <class Ld>
__device__ __forceinline__ int64_t leaf_of_words(Ld ld, const double* __restrict__ cdf, int64_t L,
                                                 const uint32_t* __restrict__ guide, int Gl, uint64_t Qi, U32x4 r) {
  const uint64_t b = ((uint64_t)(r.y & 0x1FFFFFu) << 32) | (uint64_t)r.x;
  const uint64_t lo = b * Qi;
  const uint64_t hi = __umul64hi(b, Qi);
  const uint64_t rr = (hi << 11) | (lo >> 53);
  int64_t i = guided_leaf(ld, cdf, L, guide, (uint32_t)(b >> (53 - Gl)), ord((double)rr));
  return i >= L ? L - 1 : i;
}

// Leaf of draw s of view view_id (Philox purpose 0).
template <class Ld>
__device__ __forceinline__ int64_t draw_leaf(Ld ld, const double* __restrict__ cdf, int64_t L,
                                             const uint32_t* __restrict__ guide, int Gl, uint64_t Qi, int64_t s,
                                             uint32_t view_id, uint32_t k0, uint32_t k1) {
  const U32x4 r = philox4x32_10((uint32_t)s, (uint32_t)((uint64_t)s >> 32), view_id, 0u, k0, k1);
  return leaf_of_words(ld, cdf, L, guide, Gl, Qi, r);
}

// Position in leaf `leaf` from the random words r: c + (u - 1/2) edge with
// u_d = (r_d >> 8) 2^-24, one FP32 rounding (the offset and the product by
// the power-of-two edge are exact).
__device__ __forceinline__ void leaf_position(U32x4 r, int64_t leaf, const float* __restrict__ centers,
                                              const int32_t* __restrict__ levels, float root_size, float* out) {
  const float edge = ldexpf(root_size, -levels[leaf]);
  out[0] = __fmaf_rn(__fsub_rn((float)(r.x >> 8) * 0x1p-24f, 0.5f), edge, centers[3 * leaf + 0]);
  out[1] = __fmaf_rn(__fsub_rn((float)(r.y >> 8) * 0x1p-24f, 0.5f), edge, centers[3 * leaf + 1]);
  out[2] = __fmaf_rn(__fsub_rn((float)(r.z >> 8) * 0x1p-24f, 0.5f), edge, centers[3 * leaf + 2]);
}

// Output slot k of view view_id: its leaf and position (Philox purpose 1).
__device__ __forceinline__ void place_slot(int64_t k, int64_t leaf, uint32_t view_id, uint32_t k0, uint32_t k1,
                                           const float* __restrict__ centers, const int32_t* __restrict__ levels,
                                           float root_size, int32_t* __restrict__ leaf_out,
                                           float* __restrict__ pos_out) {
  const U32x4 r = philox4x32_10((uint32_t)k, (uint32_t)((uint64_t)k >> 32), view_id, 1u, k0, k1);
  float p[3];
  leaf_position(r, leaf, centers, levels, root_size, p);
  leaf_out[k] = (int32_t)leaf;
  pos_out[3 * k + 0] = p[0];
  pos_out[3 * k + 1] = p[1];
  pos_out[3 * k + 2] = p[2];
}

}  // namespace
}  // namespace inpc
