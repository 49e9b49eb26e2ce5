// scan.cuh -- device-wide prefix sums used by the sampler (leaf CDF, leaf
// slot offsets) and the rasterizer (per-pixel fragment offsets):
// per-block scan of 2048 items, one-CTA scan of the block totals, add.
#pragma once

#include "common.cuh"

namespace inpc {
namespace scan {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kBlock = kThreads * kItems;  // 2048 items per CTA

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
__global__ void __launch_bounds__(kThreads) k_local(Load ld, int64_t L, T* __restrict__ out, T* __restrict__ tops) {
  __shared__ T warp_sums[32];
  __shared__ T total;
  const int64_t base = (int64_t)blockIdx.x * kBlock + (int64_t)threadIdx.x * kItems;
  T v[kItems];
  T run = T(0);
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    v[k] = (base + k < L) ? ld(base + k) : T(0);
    run += v[k];
  }
  const T pre = block_exclusive_scan<T>(run, warp_sums, &total);
  T acc = pre;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    if (kInclusive) acc += v[k];
    if (base + k < L) out[base + k] = acc;
    if (!kInclusive) acc += v[k];
  }
  if (threadIdx.x == 0) tops[blockIdx.x] = total;
}

// Exclusive scan of the block totals in one CTA; the grand total goes to
// tops[nb].
template <class T>
__global__ void __launch_bounds__(kThreads) k_tops(T* tops, int64_t nb) {
  __shared__ T warp_sums[32];
  __shared__ T total;
  T carry = T(0);
  for (int64_t b0 = 0; b0 < nb; b0 += kThreads) {
    const int64_t i = b0 + threadIdx.x;
    const T v = i < nb ? tops[i] : T(0);
    const T ex = block_exclusive_scan<T>(v, warp_sums, &total);
    if (i < nb) tops[i] = carry + ex;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) tops[nb] = carry;
}

template <class T>
__global__ void k_add(T* __restrict__ out, const T* __restrict__ tops, int64_t L) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < L) out[i] += tops[i / kBlock];
}

inline int64_t n_tops(int64_t L) { return ceil_div(L, kBlock) + 1; }

// out[0..L) = scan of ld(0..L); tops needs n_tops(L) entries and ends with
// the grand total at tops[ceil(L / kBlock)].
template <class T, class Load, bool kInclusive>
inpc_status run(Load ld, int64_t L, T* out, T* tops, cudaStream_t s) {
  const int64_t nb = ceil_div(L, kBlock);
  k_local<T, Load, kInclusive><<<(unsigned)nb, kThreads, 0, s>>>(ld, L, out, tops);
  k_tops<T><<<1, kThreads, 0, s>>>(tops, nb);
  if (nb > 1) k_add<T><<<(unsigned)ceil_div(L, 256), 256, 0, s>>>(out, tops, L);
  return check_launch("prefix sum", nb > 1 ? 3 : 2);
}

}  // namespace scan
}  // namespace inpc
