// raster_impl.cuh -- differentiable bilinear point rasterizer (Sec. 3.4, Eq. 1,
// Eq. 5, Eq. 6, App. A.6, Algorithm 1), forward and backward.
//
// Ordering.  Algorithm 1 sorts all splats globally by (pixel, depth).  Here
// the pixel is the most significant radix digit and is handled by a
// counting sort into per-pixel buckets (k_pix_count, prefix sum,
// k_pix_scatter); each bucket is then ordered by the remaining key
// (depth field << idb | point index) by the threads that blend it: in
// registers by a group of GA lanes per pixel for buckets of at most
// GA * kRegMax fragments (on 32-bit keys relative to the bucket's nearest
// depth whenever those order it exactly); by a CTA for larger ones, which
// first selects the nearest fragments by a depth histogram and has one warp
// sort them in registers, and falls back to a shared-memory bitonic network
// or, beyond the shared-memory capacity, a stable LSD radix sort in global
// memory.  Every path yields the exact (depth, point) order.  Tiles of
// small buckets, and the lists of larger ones, are worked through cursors so
// that uneven bucket sizes leave no warp idle.
//
// Blending.  The scatter pass stores each fragment's alpha (Eq. 6 with the
// clamp) beside its key, so blending gathers nothing but the feature rows of
// the blended fragments.  T_k = prod_{j<k} (1 - alpha_j) is a product scan
// across lanes (chunks of GA fragments on the group path, 256 on the CTA
// path), the stopping fragment (first with T_{k+1} < t_min) comes from a
// ballot, and sum_k T_k alpha_k c_k is an independent gather-reduce over the
// feature rows (V channels per lane, float4 loads).
//
// Backward.  Per pixel, T_k is recomputed by the forward's own scan (same
// rounding, nothing stored between the passes) and the suffix sums
// S_k = sum_{j>k} T_j alpha_j (c_j . g) run back to front.  Each fragment's
// two scalars (T_k alpha_k, dL/dalpha_k) go to the point's entry for the
// footprint corner the fragment came from (point-major, zero where nothing
// blended); a per-point kernel then reads its four pairs together, gathers
// the matching upstream-gradient rows and writes the point's gradient with
// plain stores: no atomics.
#pragma once

#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "scan.cuh"

namespace inpc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// Sort keys: (FP32 depth bits - dbase) << idb | point index.  Up to 2^25
// points the depth field is the raw bits of the positive depth (31 bits) and
// idb = 25; beyond that idb is the bit width of n - 1 and the depth field the
// bits above those of the near plane (every kept depth lies strictly between
// near and far, so the field is positive and monotone in depth).  Either way
// a key fits in 56 bits: the register sorts append an 8-bit bucket position.
constexpr int kIdBits = 25;
constexpr int kKeyBits = 56;
constexpr int64_t kMaxFwdPoints = int64_t(1) << 28;  // 4n fragment slots stay below 2^32
constexpr int kHeavyKeys = 2048;  // shared-memory bucket entries on the CTA path (larger buckets sort in global memory)
constexpr uint32_t kNoSlot = 0xFFFFFFFFu;

struct RP {
  Cam cam;
  int TW, TH, tiles_x, tiles_y, n_tiles;
  int F;
  int head;
  int bf16;  // feature rows and image in BF16 (arithmetic stays FP32)
  float t_min, alpha_max;
  long long n;
  long long n_pix;
  int idb;                  // point-index bits of the sort key
  uint32_t dbase;           // subtracted from the FP32 depth bits in the key
  unsigned long long idm;   // (1 << idb) - 1
};

struct RasterWs {
  uint32_t* status;
  uint32_t* heavy_count;     // header word 1
  uint32_t* large_count;     // header word 2
  uint32_t* large_next;      // header word 3: the list kernel's next list entry (forward, then backward)
  uint32_t* heavy_next;      // header word 4: the forward CTA kernel's next list entry
  uint32_t* wide_count;      // header word 5: forward list entries with 8 registers per lane (at the list's end)
  uint32_t* wide_next;       // header word 6: their cursor
  uint32_t* pix_count;       // [n_pix]
  uint32_t* pix_start;       // [n_pix + 1]
  uint32_t* tops;            // prefix-sum block totals
  uint32_t* heavy;           // [n_pix] pixels on the CTA path
  uint32_t* large;           // [n_pix] pixels with 4 or 8 registers per lane
  unsigned long long* keys;  // [4n] bucketed fragment keys
  float* alpha;              // [4n] fragment alphas
  uint32_t* pslot;           // [4n] bucket slot of each point corner (kNoSlot off-image)
  uint32_t* porg;            // [n] footprint origin of each point: (i0 + 1) | (j0 + 1) << 16
  float* pexp;               // [n] exp(h0) of each point (head mode)
  float2* fscal;             // [4n] backward per-fragment scalars, point-major: entry 4 p + c is point p's
                             // footprint corner c (the per-point blending weights keep their own slot-major
                             // values here)
  unsigned long long* ka;    // [4n] global-sort result (largest buckets only)
  uint32_t* va;
  unsigned long long* kb;    // [4n] global-sort scratch, then per-fragment (T_k, c_k . g)
  uint32_t* vb;
  uint2* order;              // [4n] per pixel, the blended prefix in blending order: (bucket position, point)
  size_t bytes;
};

RasterWs carve(void* base, long long n_pix, long long n) {
  Carver c(base);
  RasterWs w;
  w.status = reinterpret_cast<uint32_t*>(base);
  w.heavy_count = base ? reinterpret_cast<uint32_t*>(base) + 1 : nullptr;
  w.large_count = base ? reinterpret_cast<uint32_t*>(base) + 2 : nullptr;
  w.large_next = base ? reinterpret_cast<uint32_t*>(base) + 3 : nullptr;
  w.heavy_next = base ? reinterpret_cast<uint32_t*>(base) + 4 : nullptr;
  w.wide_count = base ? reinterpret_cast<uint32_t*>(base) + 5 : nullptr;
  w.wide_next = base ? reinterpret_cast<uint32_t*>(base) + 6 : nullptr;
  const long long nf = std::max<long long>(4 * n, 1);
  w.pix_count = c.take<uint32_t>(n_pix);
  w.pix_start = c.take<uint32_t>(n_pix + 1);
  w.tops = c.take<uint32_t>(scan::n_tops(n_pix));
  w.heavy = c.take<uint32_t>(n_pix);
  w.large = c.take<uint32_t>(n_pix);
  w.keys = c.take<unsigned long long>(nf);
  w.alpha = c.take<float>(nf);
  w.pslot = c.take<uint32_t>(nf);
  w.porg = c.take<uint32_t>(std::max<long long>(n, 1));
  w.pexp = c.take<float>(std::max<long long>(n, 1));
  w.fscal = c.take<float2>(nf);
  w.ka = c.take<unsigned long long>(nf);
  w.va = c.take<uint32_t>(nf);
  w.kb = c.take<unsigned long long>(nf);
  w.vb = c.take<uint32_t>(nf);
  w.order = c.take<uint2>(nf);
  w.bytes = c.bytes();
  return w;
}

// ------------------------------------------------------------ splatting ---
struct Splat {
  Footprint f;
  float d;
};

__device__ __forceinline__ bool splat_xyz(const RP& P, float x, float y, float z, Splat& s) {
  float u, v;
  if (!project_point(P.cam, x, y, z, u, v, s.d)) return false;
  return footprint(P.cam, u, v, s.f);
}

__device__ __forceinline__ bool splat_point(const RP& P, const float* __restrict__ pos, long long id, Splat& s) {
  return splat_xyz(P, __ldg(pos + 3 * id), __ldg(pos + 3 * id + 1), __ldg(pos + 3 * id + 2), s);
}

// Pixel of corner k (= a + 2b) of a footprint, or -1 if off-image (images
// are at most 32768 x 32768, so the index fits in an int).
__device__ __forceinline__ int corner_pixel(const RP& P, const Footprint& f, int k) {
  const int px = f.i0 + (k & 1);
  const int py = f.j0 + (k >> 1);
  if (px < 0 || px >= P.cam.W || py < 0 || py >= P.cam.H) return -1;
  return py * P.cam.W + px;
}

// Feature elements are FP32 or BF16; all arithmetic is FP32.
__device__ __forceinline__ float ld1(const float* __restrict__ p) { return __ldg(p); }
__device__ __forceinline__ float ld1(const __nv_bfloat16* __restrict__ p) {
  return __uint_as_float(((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p))) << 16);
}

// Point opacity alpha_h: given, or 1 - exp(-exp(h0)) (Sec. 3.3) in head mode.
template <class FT>
__device__ __forceinline__ float point_alpha_h(const RP& P, const float* __restrict__ opacity,
                                               const FT* __restrict__ feat, long long id, float* e_h0) {
  if (P.head) {
    const float e = expf(ld1(feat + (long long)P.F * id));
    if (e_h0) *e_h0 = e;
    return -expm1f(-e);
  }
  return __ldg(opacity + id);
}

// ---------------------------------------------------------------- binning ---
// The input of a point's alpha_h: h0 in head mode, else the given opacity
// (the scatter forms alpha_h from it with point_alpha_h's operations).
template <class FT>
__device__ __forceinline__ float alpha_input(const RP& P, const float* __restrict__ opacity,
                                             const FT* __restrict__ feat, long long id) {
  return P.head ? ld1(feat + (long long)P.F * id) : __ldg(opacity + id);
}

// Warp aggregation of the per-pixel counters: points come grouped by leaf,
// so consecutive lanes often hit the same pixel.  A run of equal pixels over
// consecutive lanes is found with one shuffle and one ballot (its start is a
// lane whose pixel differs from the previous lane's), and its first lane
// updates the counter for the whole run.
struct LaneRun {
  int start;  // first lane of this lane's run
  int len;    // lanes in the run (valid in the first lane)
};

__device__ __forceinline__ LaneRun lane_run(int q, int lane) {
  const int prev = __shfl_up_sync(0xffffffffu, q, 1);
  const unsigned starts = __ballot_sync(0xffffffffu, lane == 0 || prev != q);
  const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
  const unsigned later = starts & ~upto;
  LaneRun r;
  r.start = 31 - __clz(starts & upto);
  r.len = (later ? __ffs(later) - 1 : 32) - lane;
  return r;
}

__global__ void __launch_bounds__(256) k_pix_count(RP P, const float* __restrict__ pos,
                                                   uint32_t* __restrict__ pix_count) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int n = (int)P.n;  // <= 2^28
  const int stride = gridDim.x * blockDim.x;
  // each iteration loads the next point's position while it bins this one
  float x = 0.f, y = 0.f, z = 0.f;
  if (blockIdx.x * blockDim.x + threadIdx.x < n) {
    const long long id = blockIdx.x * blockDim.x + threadIdx.x;
    x = __ldg(pos + 3 * id); y = __ldg(pos + 3 * id + 1); z = __ldg(pos + 3 * id + 2);
  }
  for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
    const int id = base + threadIdx.x;
    const long long nid = (long long)id + stride;
    float nx = 0.f, ny = 0.f, nz = 0.f;
    if (nid < n) {
      nx = __ldg(pos + 3 * nid); ny = __ldg(pos + 3 * nid + 1); nz = __ldg(pos + 3 * nid + 2);
    }
    int q[4] = {-1, -1, -1, -1};
    Splat s;
    if (id < n && splat_xyz(P, x, y, z, s))
      for (int k = 0; k < 4; ++k) q[k] = corner_pixel(P, s.f, k);
    x = nx; y = ny; z = nz;
    for (int k = 0; k < 4; ++k) {
      const LaneRun run = lane_run(q[k], lane);
      if (q[k] >= 0 && run.start == lane) atomicAdd(pix_count + q[k], (uint32_t)run.len);
    }
  }
}

template <class FT>
__global__ void __launch_bounds__(256) k_pix_scatter(RP P, const float* __restrict__ pos,
                                                     const float* __restrict__ opacity,
                                                     const FT* __restrict__ feat,
                                                     const uint32_t* __restrict__ pix_start,
                                                     uint32_t* __restrict__ pix_count,
                                                     unsigned long long* __restrict__ keys,
                                                     float* __restrict__ alpha, uint32_t* __restrict__ pslot,
                                                     uint32_t* __restrict__ porg, float* __restrict__ pexp) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int n = (int)P.n;  // <= 2^28
  const int stride = gridDim.x * blockDim.x;
  // each iteration loads the next point's position and alpha input while it
  // bins this one, so those round trips overlap this point's atomics
  float x = 0.f, y = 0.f, z = 0.f, av = 0.f;
  if (blockIdx.x * blockDim.x + threadIdx.x < n) {
    const long long id = blockIdx.x * blockDim.x + threadIdx.x;
    x = __ldg(pos + 3 * id); y = __ldg(pos + 3 * id + 1); z = __ldg(pos + 3 * id + 2);
    av = alpha_input(P, opacity, feat, id);
  }
  for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
    const int id = base + threadIdx.x;
    const long long nid = (long long)id + stride;
    float nx = 0.f, ny = 0.f, nz = 0.f, na = 0.f;
    if (nid < n) {
      nx = __ldg(pos + 3 * nid); ny = __ldg(pos + 3 * nid + 1); nz = __ldg(pos + 3 * nid + 2);
      na = alpha_input(P, opacity, feat, nid);
    }
    int q[4] = {-1, -1, -1, -1};
    Splat s;
    float ah = 0.f;
    bool splat_ok = false;
    float e_h0 = 0.f;
    if (id < n && splat_xyz(P, x, y, z, s)) {
      for (int k = 0; k < 4; ++k) q[k] = corner_pixel(P, s.f, k);
      // head mode: alpha_h = 1 - exp(-exp(h0)) as in point_alpha_h, with
      // exp(h0) kept for the backward's opacity path
      e_h0 = P.head ? expf(av) : 0.f;
      ah = P.head ? -expm1f(-e_h0) : av;
      splat_ok = true;
    }
    x = nx; y = ny; z = nz; av = na;
    const unsigned long long key = ((unsigned long long)(__float_as_uint(s.d) - P.dbase) << P.idb) | (unsigned long long)id;
    // the four corners' bucket offsets and atomics are all issued before
    // any result is used, so their round trips overlap
    LaneRun run[4];
    uint32_t start[4], top[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      run[k] = lane_run(q[k], lane);
      start[k] = q[k] >= 0 ? __ldg(pix_start + q[k]) : 0u;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      // counts run down from the bucket size, so the buckets fill back to front
      top[k] = 0;
      if (q[k] >= 0 && run[k].start == lane) top[k] = atomicSub(pix_count + q[k], (uint32_t)run[k].len);
    }
    uint32_t slots[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t t = __shfl_sync(full, top[k], run[k].start);
      slots[k] = kNoSlot;
      if (q[k] >= 0) {
        slots[k] = start[k] + t - 1 - (uint32_t)(lane - run[k].start);
        keys[slots[k]] = key;
        alpha[slots[k]] = fminf(__fmul_rn(ah, corner_weight(s.f, k & 1, k >> 1)), P.alpha_max);
      }
    }
    if (id < n) reinterpret_cast<uint4*>(pslot)[id] = make_uint4(slots[0], slots[1], slots[2], slots[3]);
    if (id < n) porg[id] = splat_ok ? ((uint32_t)(s.f.i0 + 1) & 0xffffu) | ((uint32_t)(s.f.j0 + 1) << 16) : 0u;
    if (id < n && P.head) pexp[id] = e_h0;
  }
}

struct CountLoad {
  const uint32_t* c;
  __device__ uint32_t operator()(int64_t i) const { return c[i]; }
};

// Bucket-size classes: up to cap_small fragments (at most 2 registers per
// lane) stay with the tile-order kernel; up to cap_mid go to the front of
// the list of the register kernel with 4 registers per lane, up to
// cap_large to its back, for the kernel with 8 (two kernels, each with half
// the code: the unrolled sorting networks of both sizes in one kernel
// stalled it on instruction fetch); larger ones go to the CTA path.
__global__ void k_classify(const uint32_t* __restrict__ pix_start, long long n_pix, const uint32_t* __restrict__ tops,
                           long long nb, uint32_t cap_small, uint32_t cap_large, uint32_t* __restrict__ heavy,
                           uint32_t* heavy_count, uint32_t* __restrict__ large, uint32_t* large_count,
                           uint32_t* __restrict__ pix_start_w, uint32_t cap_mid, uint32_t* wide_count) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q == 0) pix_start_w[n_pix] = tops[nb];
  if (q >= n_pix) return;
  const uint32_t end = q + 1 < n_pix ? pix_start[q + 1] : tops[nb];
  const uint32_t m = end - pix_start[q];
  if (m > cap_large) heavy[atomicAdd(heavy_count, 1u)] = (uint32_t)q;
  else if (m > cap_mid) large[n_pix - 1 - atomicAdd(wide_count, 1u)] = (uint32_t)q;
  else if (m > cap_small) large[atomicAdd(large_count, 1u)] = (uint32_t)q;
}

// Backward classes by blended count (the forward's n_contrib, clamped to the
// bucket): the tile kernel takes nb <= cap_small, the list kernels the rest.
__global__ void k_classify_bwd(const int32_t* __restrict__ n_contrib, const uint32_t* __restrict__ pix_start,
                               long long n_pix, uint32_t cap_small, uint32_t cap_large, uint32_t* __restrict__ heavy,
                               uint32_t* heavy_count, uint32_t* __restrict__ large, uint32_t* large_count) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n_pix) return;
  const int c = n_contrib[q];
  const uint32_t m = pix_start[q + 1] - pix_start[q];
  const uint32_t nb = c < 0 ? 0u : min((uint32_t)c, m);
  if (nb > cap_large) heavy[atomicAdd(heavy_count, 1u)] = (uint32_t)q;
  else if (nb > cap_small) large[atomicAdd(large_count, 1u)] = (uint32_t)q;
}

__device__ __forceinline__ int blended_count(const int32_t* __restrict__ n_contrib, long long q, int m) {
  const int c = n_contrib[q];
  return c < 0 ? 0 : min(c, m);
}

// Entry k of a pixel's blended prefix; an entry the forward did not write
// (only reachable with a mismatched n_contrib) is clamped into the bucket.
__device__ __forceinline__ uint2 order_at(const RP& P, const RasterWs& ws, uint32_t s0, int m, int k) {
  uint2 o = ws.order[s0 + k];
  if (o.x >= (uint32_t)m) o.x = 0;
  if ((long long)o.y >= P.n) o.y = 0;
  return o;
}

// Point-major index of the backward scalars of point pid's fragment at
// pixel (qx, qy): 4 pid + c, c = (qx - i0) + 2 (qy - j0) the footprint
// corner of that pixel, from the point's footprint origin (a 4-byte record
// per point that stays in L2).  The per-point pass then reads a point's four
// pairs as one 32-byte sector instead of four scattered ones.  (A
// mismatched pixel stays within the point's four entries.)
__device__ __forceinline__ uint32_t frag_index(const RasterWs& ws, uint32_t pid, int qx, int qy) {
  const uint32_t o = __ldg(ws.porg + pid);
  const int c = (qx + 1 - (int)(o & 0xffffu)) + 2 * (qy + 1 - (int)(o >> 16));
  return 4u * pid + ((uint32_t)c & 3u);
}

// ------------------------------------------------------------- ordering ---
// Ascending sort of idx[0..m) by K[idx[.]] with an all-ascending bitonic
// network (every comparator puts the minimum at the lower index), so the
// virtual +infinity padding beyond m is never touched.  `lg`/`nl`: this
// thread's index and the number of cooperating threads; `sync` orders them.
template <class Sync>
__device__ void bitonic_sort_idx(const unsigned long long* K, uint16_t* idx, int m, int lg, int nl, Sync sync) {
  if (m < 2) return;
  int P2 = 1;
  while (P2 < m) P2 <<= 1;
  for (int k = 2; k <= P2; k <<= 1) {
    const int half = k >> 1;
    for (int q = lg; q < (P2 >> 1); q += nl) {
      const int i = (q / half) * k + (q % half);
      const int j = i ^ (k - 1);
      if (j < m) {
        const uint16_t a = idx[i], b = idx[j];
        if (K[a] > K[b]) {
          idx[i] = b;
          idx[j] = a;
        }
      }
    }
    sync();
    for (int jj = k >> 2; jj >= 1; jj >>= 1) {
      for (int q = lg; q < (P2 >> 1); q += nl) {
        const int i = (q / jj) * (2 * jj) + (q % jj);
        const int j = i + jj;
        if (j < m) {
          const uint16_t a = idx[i], b = idx[j];
          if (K[a] > K[b]) {
            idx[i] = b;
            idx[j] = a;
          }
        }
      }
      sync();
    }
  }
}

struct SortSmem {
  uint32_t hist[256];
  uint32_t dbase[256];
  uint32_t ctot[256];
  uint16_t wcnt[kWarps][256];
  unsigned long long red64[kWarps];
  uint32_t warp_sums[32];
};

__device__ __forceinline__ uint32_t cta_excl_scan256(uint32_t v, uint32_t* warp_sums) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  __syncthreads();
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t t = warp_sums[w];
      warp_sums[w] = run;
      run += t;
    }
  }
  __syncthreads();
  return warp_sums[wid] + incl - v;
}

// Stable 8-bit LSD radix sort of one bucket in global memory by one CTA:
// in[0..n) -> ka (keys), va (positions within the bucket); kb/vb scratch.
// Digits that are equal across the bucket are skipped.
__device__ void cta_sort_global(const unsigned long long* __restrict__ in, int n, unsigned long long* ka,
                                uint32_t* va, unsigned long long* kb, uint32_t* vb, SortSmem& S) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned long long k0 = in[0];
  unsigned long long diff = 0;
  for (int i = threadIdx.x; i < n; i += kThreads) {
    const unsigned long long k = in[i];
    ka[i] = k;
    va[i] = (uint32_t)i;
    diff |= k ^ k0;
  }
  for (int o = 16; o > 0; o >>= 1) diff |= __shfl_xor_sync(0xffffffffu, diff, o);
  if (lane == 0) S.red64[wid] = diff;
  __syncthreads();
  diff = 0;
  for (int w = 0; w < kWarps; ++w) diff |= S.red64[w];
  bool in_a = true;
  for (int dgt = 0; dgt < 8; ++dgt) {
    const int sh = 8 * dgt;
    if (((diff >> sh) & 0xFFull) == 0) continue;
    unsigned long long* sk = in_a ? ka : kb;
    uint32_t* sv = in_a ? va : vb;
    unsigned long long* dk = in_a ? kb : ka;
    uint32_t* dv = in_a ? vb : va;
    S.hist[threadIdx.x] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kThreads) atomicAdd(&S.hist[(int)((sk[i] >> sh) & 0xFF)], 1u);
    __syncthreads();
    S.dbase[threadIdx.x] = cta_excl_scan256(S.hist[threadIdx.x], S.warp_sums);
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += kThreads) {
      const int i = c0 + threadIdx.x;
      const bool valid = i < n;
      unsigned long long key = 0;
      uint32_t val = 0;
      int dg = 256;
      if (valid) {
        key = sk[i];
        val = sv[i];
        dg = (int)((key >> sh) & 0xFF);
      }
      const unsigned peers = __match_any_sync(0xffffffffu, dg);
      const int rank = __popc(peers & ((1u << lane) - 1));
      for (int w = 0; w < kWarps; ++w) S.wcnt[w][threadIdx.x] = 0;
      __syncthreads();
      if (valid && lane == __ffs(peers) - 1) S.wcnt[wid][dg] = (uint16_t)__popc(peers);
      __syncthreads();
      {
        uint32_t run = 0;
        for (int w = 0; w < kWarps; ++w) {
          const uint32_t c = S.wcnt[w][threadIdx.x];
          S.wcnt[w][threadIdx.x] = (uint16_t)run;
          run += c;
        }
        S.ctot[threadIdx.x] = run;
      }
      __syncthreads();
      if (valid) {
        const uint32_t dst = S.dbase[dg] + S.wcnt[wid][dg] + rank;
        dk[dst] = key;
        dv[dst] = val;
      }
      __syncthreads();
      S.dbase[threadIdx.x] += S.ctot[threadIdx.x];
      __syncthreads();
    }
    in_a = !in_a;
  }
  if (!in_a) {
    for (int i = threadIdx.x; i < n; i += kThreads) {
      ka[i] = kb[i];
      va[i] = vb[i];
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------- lane groups ---
template <int GA>
struct Group {
  int lg;          // lane within the group
  int base_lane;   // first lane of the group within its warp
  unsigned mask;   // the group's lanes
  __device__ Group() {
    const int lane = threadIdx.x & 31;
    lg = lane % GA;
    base_lane = lane - lg;
    mask = GA == 32 ? 0xffffffffu : (((1u << GA) - 1u) << base_lane);
  }
  __device__ void sync() const {
    if (GA > 1) __syncwarp(mask);
  }
  template <class T>
  __device__ T bcast(T v, int src) const {
    return GA > 1 ? __shfl_sync(mask, v, src, GA) : v;
  }
  __device__ float sum(float x) const {
#pragma unroll
    for (int o = GA / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o, GA);
    return x;
  }
  // Inclusive product scan over the group's lanes.
  __device__ float prod_scan(float x) const {
#pragma unroll
    for (int o = 1; o < GA; o <<= 1) {
      const float t = __shfl_up_sync(mask, x, o, GA);
      if (lg >= o) x = __fmul_rn(x, t);
    }
    return x;
  }
  // Inclusive suffix-sum scan over the group's lanes (lane j gets sum_{i>=j}).
  __device__ float suffix_scan(float x) const {
#pragma unroll
    for (int o = 1; o < GA; o <<= 1) {
      const float t = __shfl_down_sync(mask, x, o, GA);
      if (lg + o < GA) x += t;
    }
    return x;
  }
  // Value of the next lane of the group (0 for the last lane).
  __device__ float shift_down(float x) const {
    if (GA == 1) return 0.f;
    const float t = __shfl_down_sync(mask, x, 1, GA);
    return lg + 1 < GA ? t : 0.f;
  }
  __device__ unsigned ballot(bool p) const {
    return (__ballot_sync(mask, p) >> base_lane) & (GA == 32 ? 0xffffffffu : ((1u << GA) - 1u));
  }
};

template <int V>
__device__ __forceinline__ void load_vec(const float* __restrict__ p, float* c) {
  if (V == 4) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    c[0] = t.x; c[1] = t.y; c[2] = t.z; c[3] = t.w;
  } else if (V == 2) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    c[0] = t.x; c[1] = t.y;
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) c[v] = __ldg(p + v);
  }
}

// This lane's V channels of a point's blended color: its features, with
// channel 0 replaced by 1 in head mode.
template <int V>
__device__ __forceinline__ void load_vec(const __nv_bfloat16* __restrict__ p, float* c) {
  if (V == 4) {
    const uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
    c[0] = __uint_as_float(raw.x << 16);
    c[1] = __uint_as_float(raw.x & 0xFFFF0000u);
    c[2] = __uint_as_float(raw.y << 16);
    c[3] = __uint_as_float(raw.y & 0xFFFF0000u);
  } else if (V == 2) {
    const uint32_t raw = __ldg(reinterpret_cast<const unsigned int*>(p));
    c[0] = __uint_as_float(raw << 16);
    c[1] = __uint_as_float(raw & 0xFFFF0000u);
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) c[v] = ld1(p + v);
  }
}

template <int V, class FT>
__device__ __forceinline__ void load_color(const RP& P, const FT* __restrict__ feat, long long id, int ch, float* c) {
  load_vec<V>(feat + (long long)P.F * id + ch, c);
  if (P.head && ch == 0) c[0] = 1.0f;
}

template <int V>
__device__ __forceinline__ void write_pixel(const RP& P, long long pix, int ch, const float* C, float* __restrict__ image) {
  if (ch >= P.F) return;
  float* o = image + pix * P.F + ch;
  if (V == 4) __stcs(reinterpret_cast<float4*>(o), make_float4(C[0], C[1], C[2], C[3]));
  else if (V == 2) __stcs(reinterpret_cast<float2*>(o), make_float2(C[0], C[1]));
  else
#pragma unroll
    for (int v = 0; v < V; ++v) __stcs(o + v, C[v]);
}

template <int V>
__device__ __forceinline__ void write_pixel(const RP& P, long long pix, int ch, const float* C,
                                            __nv_bfloat16* __restrict__ image) {
  if (ch >= P.F) return;
  __nv_bfloat16* o = image + pix * P.F + ch;
  if (V == 4) {
    __nv_bfloat162 a = __floats2bfloat162_rn(C[0], C[1]);
    __nv_bfloat162 b = __floats2bfloat162_rn(C[2], C[3]);
    uint2 raw;
    raw.x = *reinterpret_cast<uint32_t*>(&a);
    raw.y = *reinterpret_cast<uint32_t*>(&b);
    __stcs(reinterpret_cast<uint2*>(o), raw);
  } else if (V == 2) {
    __nv_bfloat162 a = __floats2bfloat162_rn(C[0], C[1]);
    *reinterpret_cast<__nv_bfloat162*>(o) = a;
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) o[v] = __float2bfloat16_rn(C[v]);
  }
}

// Transmittance of one chunk of GA fragments: lane j holds the alpha of
// fragment b + j (0 beyond the list).  The inclusive product scan of
// (1 - alpha) gives the transmittance behind each fragment, the shifted scan
// the one in front of it; the first lane whose T drops below t_min stops the
// pixel (that fragment is blended).
template <int GA>
struct ChunkT {
  float Tk;   // transmittance in front of this lane's fragment
  float Tn;   // transmittance behind it
  int take;   // fragments of the chunk that are blended
  bool stop;
};

template <int GA>
__device__ __forceinline__ ChunkT<GA> chunk_transmittance(const Group<GA>& G, const RP& P, float a, bool valid,
                                                          int avail, float T) {
  ChunkT<GA> r;
  const float incl = G.prod_scan(__fsub_rn(1.0f, a));
  float excl = G.bcast(incl, G.lg > 0 ? G.lg - 1 : 0);
  if (G.lg == 0) excl = 1.0f;
  r.Tk = __fmul_rn(T, excl);
  r.Tn = __fmul_rn(T, incl);
  const unsigned st = G.ballot(valid && r.Tn < P.t_min);
  r.stop = st != 0;
  r.take = r.stop ? __ffs(st) : avail;
  return r;
}

// ------------------------------------------------------ group path (fwd) ---
// One pixel per group of GA lanes.  The bucket (at most GA * kRegMax
// fragments) is sorted in registers: lane lg holds elements r * GA + lg,
// r < R, and a bitonic network exchanges across lanes (shuffles) for strides
// below GA and between registers above.  After the sort, register r of the
// group is chunk r of the blending order.  Each element carries its bucket
// position in the low 8 bits (key << 8 | position), which locates its alpha.
constexpr int kRegMax = 8;

// Stages up to block size k leave the lowest k elements sorted ascending;
// elements at or above m are the maximum key, so a bucket of m <= k needs
// no later stage (m is uniform over the group).
template <int GA, int R>
__device__ __forceinline__ void reg_sort(const Group<GA>& G, unsigned long long (&key)[R], int m = GA * R) {
  constexpr int P2 = GA * R;
#pragma unroll
  for (int k = 2; k <= P2; k <<= 1) {
    if ((k >> 1) >= m) break;
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= GA) {
        const int jr = j / GA;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int r2 = r ^ jr;
          if (r2 > r) {
            const bool up = (((r * GA + G.lg) & k) == 0);
            const unsigned long long x = key[r], y = key[r2];
            if ((x > y) == up) {
              key[r] = y;
              key[r2] = x;
            }
          }
        }
      } else {
        const bool lower = (G.lg & j) == 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const bool up = (((r * GA + G.lg) & k) == 0);
          const unsigned long long o = __shfl_xor_sync(G.mask, key[r], j, GA);
          key[r] = (lower == up) ? (key[r] < o ? key[r] : o) : (key[r] > o ? key[r] : o);
        }
      }
    }
  }
}

// The same network on 32-bit keys: one shuffle and a min/max per element
// and stage instead of two shuffles and a 64-bit compare and select.
template <int GA, int R>
__device__ __forceinline__ void reg_sort32(const Group<GA>& G, uint32_t (&key)[R], int m) {
  constexpr int P2 = GA * R;
#pragma unroll
  for (int k = 2; k <= P2; k <<= 1) {
    if ((k >> 1) >= m) break;
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= GA) {
        const int jr = j / GA;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int r2 = r ^ jr;
          if (r2 > r) {
            const bool up = (((r * GA + G.lg) & k) == 0);
            const uint32_t lo = min(key[r], key[r2]), hi = max(key[r], key[r2]);
            key[r] = up ? lo : hi;
            key[r2] = up ? hi : lo;
          }
        }
      } else {
        const bool lower = (G.lg & j) == 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const bool up = (((r * GA + G.lg) & k) == 0);
          const uint32_t o = __shfl_xor_sync(G.mask, key[r], j, GA);
          key[r] = (lower == up) ? min(key[r], o) : max(key[r], o);
        }
      }
    }
  }
}

template <int GA>
__device__ __forceinline__ uint32_t group_umin(const Group<GA>& G, uint32_t v) {
  if constexpr (GA == 32) return __reduce_min_sync(0xffffffffu, v);
#pragma unroll
  for (int o = GA / 2; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(G.mask, v, o, GA));
  return v;
}

template <int GA>
__device__ __forceinline__ uint32_t group_umax(const Group<GA>& G, uint32_t v) {
  if constexpr (GA == 32) return __reduce_max_sync(0xffffffffu, v);
#pragma unroll
  for (int o = GA / 2; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(G.mask, v, o, GA));
  return v;
}

// Sorts m <= GA * R fragment keys, load(e) giving the key at position e,
// by (depth, point), each element returned as key << 8 | position.  Within one pixel
// the depths usually span far fewer than 2^24 FP32 values, so the sort runs
// on 32-bit keys (depth field - the bucket's minimum) << 8 | position,
// which order the bucket exactly as the full keys do unless two fragments
// have the same depth (then the point index decides).  Such ties show up as
// equal neighbours after the sort; a bucket with one, or with a wider depth
// span, is sorted again on the full 64-bit keys.  The full key of each
// sorted element is then fetched by its position: from the lane that loaded
// it (R <= 2) or through load again (an L1 or shared-memory hit).
template <int GA, int R, class Load>
__device__ __forceinline__ void sort_loaded(const Group<GA>& G, const RP& P, Load load, int m,
                                            unsigned long long (&key)[R]) {
  unsigned long long raw[R];
  uint32_t k[R];
  uint32_t lo = 0xFFFFFFFFu, hi = 0u;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int e = r * GA + G.lg;
    raw[r] = e < m ? load(e) : 0ull;
    k[r] = (uint32_t)(raw[r] >> P.idb);
    if (e < m) {
      lo = min(lo, k[r]);
      hi = max(hi, k[r]);
    }
  }
  lo = group_umin<GA>(G, lo);
  hi = group_umax<GA>(G, hi);
  // valid keys stay below the 0xFFFFFFFF of the empty places
  if (hi - lo < 0xFFFFFFu) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = r * GA + G.lg;
      k[r] = e < m ? ((k[r] - lo) << 8) | (uint32_t)e : 0xFFFFFFFFu;
    }
    reg_sort32<GA, R>(G, k, m);
    bool tie = false;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      uint32_t nx = __shfl_down_sync(G.mask, k[r], 1, GA);
      const uint32_t n0 = r + 1 < R ? __shfl_sync(G.mask, k[r + 1 < R ? r + 1 : r], 0, GA) : 0xFFFFFFFFu;
      if (G.lg == GA - 1) nx = n0;
      if (r * GA + G.lg + 1 < m && (nx >> 8) == (k[r] >> 8)) tie = true;
    }
    if (G.ballot(tie) == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t e = k[r] & 0xFFu;
        unsigned long long full;
        if constexpr (R <= 2) {
          const unsigned long long v0 = __shfl_sync(G.mask, raw[0], (int)(e % GA), GA);
          const unsigned long long v1 = __shfl_sync(G.mask, raw[R - 1], (int)(e % GA), GA);
          full = (R == 2 && e >= (uint32_t)GA) ? v1 : v0;
        } else {
          full = k[r] != 0xFFFFFFFFu ? load((int)e) : 0ull;
        }
        key[r] = k[r] != 0xFFFFFFFFu ? (full << 8) | e : ~0ull;
      }
      return;
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int e = r * GA + G.lg;
    key[r] = e < m ? (raw[r] << 8) | (unsigned long long)e : ~0ull;
  }
  reg_sort<GA, R>(G, key, m);
}

// A bucket of m <= GA * R fragments at keys[s0 ..], sorted as above.
template <int GA, int R>
__device__ __forceinline__ void load_sorted(const Group<GA>& G, const RP& P, const unsigned long long* __restrict__ keys,
                                            uint32_t s0, int m, unsigned long long (&key)[R]) {
  sort_loaded<GA, R>(G, P, [&](int e) { return keys[s0 + e]; }, m, key);
}

__device__ __forceinline__ long long reg_id(const RP& P, unsigned long long k) { return (long long)((k >> 8) & P.idm); }
__device__ __forceinline__ uint32_t reg_pos(unsigned long long k) { return (uint32_t)(k & 0xFF); }

// ------------------------------------------- 64 channels: fragment slots ---
// For F = 64 on a 32-lane group the gather-reduce runs on 8 fragment slots
// of 4 lanes: lane (slot f = lane / 4, part q = lane % 4) reads 16 channels
// of the feature row of fragment 8p + f in pass p with 16-byte loads (4
// FP32 chunks of 4 channels, chunk 4i + q; or 2 BF16 chunks of 8 channels),
// so one pass moves 8 rows with 4 (FP32) or 2 (BF16) loads per lane.  The
// forward accumulates per slot and reduce-scatters over the slots at the
// end of the pixel (each lane then holds 2 channels); the backward's dot
// products c_j . g are per slot sums over 16 channels plus two shuffles.
template <class FT>
struct Slot64;

template <>
struct Slot64<float> {
  // channel of element e (0..15) of part q
  __device__ static int channel(int q, int e) { return 16 * (e >> 2) + 4 * q + (e & 3); }
  __device__ static void load(const float* __restrict__ row, int q, float (&c)[16]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(row + 4 * (4 * i + q)));
      c[4 * i + 0] = t.x;
      c[4 * i + 1] = t.y;
      c[4 * i + 2] = t.z;
      c[4 * i + 3] = t.w;
    }
  }
  __device__ static void store2(float* __restrict__ row, int ch, float a, float b) {
    __stcs(reinterpret_cast<float2*>(row + ch), make_float2(a, b));
  }
};

template <>
struct Slot64<__nv_bfloat16> {
  __device__ static int channel(int q, int e) { return 32 * (e >> 3) + 8 * q + (e & 7); }
  __device__ static void load(const __nv_bfloat16* __restrict__ row, int q, float (&c)[16]) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const uint4 raw = __ldg(reinterpret_cast<const uint4*>(row + 8 * (4 * i + q)));
      const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        c[8 * i + 2 * k] = __uint_as_float(w[k] << 16);
        c[8 * i + 2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
      }
    }
  }
  __device__ static void store2(__nv_bfloat16* __restrict__ row, int ch, float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    __stcs(reinterpret_cast<unsigned int*>(row + ch), *reinterpret_cast<unsigned int*>(&v));
  }
};

// The upstream gradient (FP32) of this lane's 16 channels, in the layout of FT.
template <class FT>
__device__ __forceinline__ void load_grad16(const float* __restrict__ g, int q, float (&out)[16]) {
#pragma unroll
  for (int e = 0; e < 16; e += 4) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(g + Slot64<FT>::channel(q, e)));
    out[e] = t.x;
    out[e + 1] = t.y;
    out[e + 2] = t.z;
    out[e + 3] = t.w;
  }
}

// L2 prefetch of point id's 64-channel feature row (each of its 128-byte
// lines), issued as soon as a lane knows which row it will need so that the
// gather finds it in L2.
template <class FT>
__device__ __forceinline__ void prefetch_row64(const FT* __restrict__ feat, uint32_t id) {
  const char* p = reinterpret_cast<const char*>(feat + 64ll * id);
#pragma unroll
  for (int k = 0; k < (int)(64 * sizeof(FT)) / 128; ++k) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + 128 * k));
}

template <class FT, int R>
__device__ void blend_fwd_slots(const Group<32>& G, const RP& P, const RasterWs& ws, uint32_t s0, int m,
                                long long pix, const FT* __restrict__ feat, FT* __restrict__ image,
                                float* __restrict__ T_final, int32_t* __restrict__ n_contrib) {
  if (m == 0) {  // no fragment: the background
    Slot64<FT>::store2(image + pix * 64, 2 * G.lg, 0.f, 0.f);
    if (G.lg == 0) {
      T_final[pix] = 1.0f;
      n_contrib[pix] = 0;
    }
    return;
  }
  unsigned long long key[R];
  // Small buckets (R <= 2): the alphas are loaded in bucket order beside the
  // keys, and after the sort each lane takes its fragment's alpha from the
  // lane that loaded that bucket position, instead of gathering it after
  // the sort (one dependent round trip less per pixel).
  float a_in[R];
  if constexpr (R <= 2) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = r * 32 + G.lg;
      a_in[r] = e < m ? ws.alpha[s0 + e] : 0.f;
    }
  }
  load_sorted<32, R>(G, P, ws.keys, s0, m, key);
  // the nearest 64 fragments' rows (blending usually stops within them)
#pragma unroll
  for (int r = 0; r < (R < 2 ? R : 2); ++r)
    if (r * 32 + G.lg < m) prefetch_row64(feat, (uint32_t)reg_id(P, key[r]));
  float a_sorted[R];
  if constexpr (R <= 2) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t pos = reg_pos(key[r]);
      const float v0 = __shfl_sync(0xffffffffu, a_in[0], pos & 31);
      const float v1 = R == 2 ? __shfl_sync(0xffffffffu, a_in[R - 1], pos & 31) : 0.f;
      a_sorted[r] = (R == 2 && (pos >> 5) == 1) ? v1 : v0;
    }
  }
  const int q = G.lg & 3, f = G.lg >> 2;
  float acc[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) acc[e] = 0.f;
  float T = 1.0f;
  int cnt = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int b = r * 32;
    if (b >= m) break;
    const bool valid = b + G.lg < m;
    float a = 0.f;
    if constexpr (R <= 2) a = valid ? a_sorted[r] : 0.f;
    else a = valid ? ws.alpha[s0 + reg_pos(key[r])] : 0.f;
    const uint32_t id = valid ? (uint32_t)reg_id(P, key[r]) : 0u;
    const ChunkT<32> ct = chunk_transmittance<32>(G, P, a, valid, min(32, m - b), T);
    const float wk = __fmul_rn(ct.Tk, a);
    if (G.lg < ct.take) ws.order[s0 + b + G.lg] = make_uint2(reg_pos(key[r]), id);
#pragma unroll 2
    for (int p = 0; p * 8 < ct.take; ++p) {
      const int j = 8 * p + f;
      const uint32_t idj = __shfl_sync(0xffffffffu, id, j);
      const float wj = __shfl_sync(0xffffffffu, wk, j);
      if (j < ct.take) {
        float c[16];
        Slot64<FT>::load(feat + 64ll * idj, q, c);
        if (P.head && q == 0) c[0] = 1.0f;
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] = __fmaf_rn(wj, c[e], acc[e]);
      }
    }
    cnt += ct.take;
    T = G.bcast(ct.Tn, ct.take - 1);
    if (ct.stop) break;
  }
  // reduce-scatter over the 8 slots (lane bits 4, 3, 2)
  const int h4 = (G.lg >> 4) & 1, h3 = (G.lg >> 3) & 1, h2 = (G.lg >> 2) & 1;
  float r8[8], r4[4], r2[2];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float send = h4 ? acc[k] : acc[8 + k];
    const float keep = h4 ? acc[8 + k] : acc[k];
    r8[k] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, 16));
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float send = h3 ? r8[k] : r8[4 + k];
    const float keep = h3 ? r8[4 + k] : r8[k];
    r4[k] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, 8));
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = h2 ? r4[k] : r4[2 + k];
    const float keep = h2 ? r4[2 + k] : r4[k];
    r2[k] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, 4));
  }
  const int e0 = 8 * h4 + 4 * h3 + 2 * h2;
  Slot64<FT>::store2(image + pix * 64, Slot64<FT>::channel(q, e0), r2[0], r2[1]);
  if (G.lg == 0) {
    T_final[pix] = T;
    n_contrib[pix] = cnt;
  }
}

template <class FT, int R>
__device__ void blend_bwd_slots(const Group<32>& G, const RP& P, const RasterWs& ws, uint32_t s0, int m, int nb,
                                long long pix, const FT* __restrict__ feat, const float* __restrict__ d_image) {
  const int qy = (int)(pix / P.cam.W), qx = (int)(pix - (long long)qy * P.cam.W);  // this pixel
  if (nb == 0) return;
  uint32_t slot[R], idr[R];
  float a[R], Tc[R];
  float T = 1.0f;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    a[r] = 0.f;
    Tc[r] = T;
    slot[r] = 0;
    idr[r] = 0;
    const int b = r * 32;
    if (b < nb) {
      const bool valid = b + G.lg < nb;
      if (valid) {
        const uint2 o = order_at(P, ws, s0, m, b + G.lg);
        slot[r] = o.x;
        idr[r] = o.y;
        a[r] = ws.alpha[s0 + o.x];
        prefetch_row64(feat, o.y);
      }
      const ChunkT<32> ct = chunk_transmittance<32>(G, P, a[r], valid, min(32, nb - b), T);
      T = G.bcast(ct.Tn, ct.take - 1);
    }
  }
  const int q = G.lg & 3, f = G.lg >> 2;
  float g[16];
  load_grad16<FT>(d_image + pix * 64, q, g);
  float S = 0.f;
#pragma unroll
  for (int r = R - 1; r >= 0; --r) {
    const int b = r * 32;
    if (b >= nb) continue;
    const bool valid = b + G.lg < nb;
    const uint32_t id = idr[r];
    // issued here, used at the end of the chunk
    const uint32_t dst = valid ? frag_index(ws, id, qx, qy) : 0u;
    const ChunkT<32> ct = chunk_transmittance<32>(G, P, a[r], valid, min(32, nb - b), Tc[r]);
    float mydot = 0.f;
#pragma unroll 2
    for (int p = 0; p * 8 < ct.take; ++p) {
      const int j = 8 * p + f;
      const uint32_t idj = __shfl_sync(0xffffffffu, id, j);
      float part = 0.f;
      if (j < ct.take) {
        float c[16];
        Slot64<FT>::load(feat + 64ll * idj, q, c);
        if (P.head && q == 0) c[0] = 1.0f;
#pragma unroll
        for (int e = 0; e < 16; ++e) part = __fmaf_rn(c[e], g[e], part);
      }
      part = __fadd_rn(part, __shfl_xor_sync(0xffffffffu, part, 1));
      part = __fadd_rn(part, __shfl_xor_sync(0xffffffffu, part, 2));
      // fragment 8p + s's dot product goes to lane 8p + s (from slot s's lane 4s)
      const float v = __shfl_sync(0xffffffffu, part, (4 * (G.lg - 8 * p)) & 31);
      if (G.lg >= 8 * p && G.lg < 8 * p + 8) mydot = v;
    }
    const bool mine = G.lg < ct.take;
    const float wk = mine ? __fmul_rn(ct.Tk, a[r]) : 0.f;
    const float term = __fmul_rn(wk, mydot);
    const float suf = G.suffix_scan(term);             // this chunk, at or behind k
    const float Sk = __fadd_rn(S, G.shift_down(suf));  // strictly behind k
    const float da = __fsub_rn(__fmul_rn(ct.Tk, mydot), __fdiv_rn(Sk, __fsub_rn(1.0f, a[r])));
    if (mine) ws.fscal[dst] = make_float2(wk, da);
    S = __fadd_rn(S, G.bcast(suf, 0));
  }
}

template <int V, int GA, class FT, int R>
__device__ void blend_fwd_reg(const Group<GA>& G, const RP& P, const RasterWs& ws, uint32_t s0, int m, long long pix,
                              const FT* __restrict__ feat, FT* __restrict__ image, float* __restrict__ T_final,
                              int32_t* __restrict__ n_contrib) {
  if constexpr (V == 2 && GA == 32) {  // F = 64
    blend_fwd_slots<FT, R>(G, P, ws, s0, m, pix, feat, image, T_final, n_contrib);
    return;
  }
  unsigned long long key[R];
  load_sorted<GA, R>(G, P, ws.keys, s0, m, key);
  const int ch = G.lg * V;
  float C[V];
#pragma unroll
  for (int v = 0; v < V; ++v) C[v] = 0.f;
  float T = 1.0f;
  int cnt = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int b = r * GA;
    if (b >= m) break;
    const bool valid = b + G.lg < m;
    const float a = valid ? ws.alpha[s0 + reg_pos(key[r])] : 0.f;
    const long long id = valid ? reg_id(P, key[r]) : 0;
    const ChunkT<GA> ct = chunk_transmittance<GA>(G, P, a, valid, min(GA, m - b), T);
    const float wk = __fmul_rn(ct.Tk, a);
    if (G.lg < ct.take) ws.order[s0 + b + G.lg] = make_uint2(reg_pos(key[r]), (uint32_t)id);
#pragma unroll 8
    for (int j = 0; j < ct.take; ++j) {
      const long long idj = G.bcast(id, j);
      const float wj = G.bcast(wk, j);
      if (ch < P.F) {
        float c[V];
        load_color<V, FT>(P, feat, idj, ch, c);
#pragma unroll
        for (int v = 0; v < V; ++v) C[v] = __fmaf_rn(wj, c[v], C[v]);
      }
    }
    cnt += ct.take;
    T = G.bcast(ct.Tn, ct.take - 1);
    if (ct.stop) break;
  }
  write_pixel<V>(P, pix, ch, C, image);
  if (G.lg == 0) {
    T_final[pix] = T;
    n_contrib[pix] = cnt;
  }
}

// A tile's pixels in shared memory: bucket start, size (-1 outside the
// image) and blended count of tile pixel i, loaded by thread i
// (TW * TH <= kThreads), and the list of the pixels this kernel works on.
// The CTA's groups take pixels from the list through a cursor, so a group
// done with small buckets takes more and no warp waits on another's share.
struct TileSmem {
  uint32_t s0[kThreads];
  int m[kThreads];
  int nb[kThreads];
  uint16_t list[kThreads];
  int count, next;
};

// kBwd: the work pixels are those with 0 < blended count <= cap (else
// 0 < bucket size <= cap).
template <bool kBwd>
__device__ __forceinline__ void load_tile(const RP& P, const RasterWs& ws, int tx, int ty,
                                          const int32_t* __restrict__ n_contrib, int cap, TileSmem& S) {
  const int i = threadIdx.x;
  if (i == 0) {
    S.count = 0;
    S.next = 0;
  }
  __syncthreads();
  if (i < P.TW * P.TH) {
    int m = -1, nb = 0;
    uint32_t s0 = 0;
    const int px = tx * P.TW + i % P.TW, py = ty * P.TH + i / P.TW;
    if (px < P.cam.W && py < P.cam.H) {
      const long long q = (long long)py * P.cam.W + px;
      s0 = ws.pix_start[q];
      m = (int)(ws.pix_start[q + 1] - s0);
      if (kBwd && m > 0) nb = blended_count(n_contrib, q, m);
    }
    S.s0[i] = s0;
    S.m[i] = m;
    S.nb[i] = nb;
    const int w = kBwd ? nb : m;
    if (w > 0 && w <= cap) S.list[atomicAdd(&S.count, 1)] = (uint16_t)i;
  }
  __syncthreads();
}

// The next work pixel of the tile for this group, or -1.
template <int GA>
__device__ __forceinline__ int next_tile_pixel(const Group<GA>& G, TileSmem& S) {
  int k = 0;
  if (G.lg == 0) k = atomicAdd(&S.next, 1);
  k = G.bcast(k, 0);
  return k < S.count ? (int)S.list[k] : -1;
}

__device__ __forceinline__ long long tile_pixel_index(const RP& P, int tx, int ty, int j) {
  return (long long)(ty * P.TH + j / P.TW) * P.cam.W + tx * P.TW + j % P.TW;
}

// The background (zero color, T = 1, no fragment) of the tile's empty
// pixels, one warp per pixel.
template <class FT>
__device__ __forceinline__ void fill_empty(const RP& P, int tx, int ty, const TileSmem& S, FT* __restrict__ image,
                                           float* __restrict__ T_final, int32_t* __restrict__ n_contrib) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int bytes = P.F * (int)sizeof(FT);
  for (int j = warp; j < P.TW * P.TH; j += kWarps) {
    if (S.m[j] != 0) continue;
    const long long q = tile_pixel_index(P, tx, ty, j);
    char* row = reinterpret_cast<char*>(image + q * P.F);
    if (bytes % 8 == 0) {
      for (int u = lane; u < bytes / 8; u += 32) reinterpret_cast<uint2*>(row)[u] = make_uint2(0u, 0u);
    } else {
      for (int u = lane; u < bytes / 4; u += 32) reinterpret_cast<uint32_t*>(row)[u] = 0u;
    }
    if (lane == 0) {
      T_final[q] = 1.0f;
      n_contrib[q] = 0;
    }
  }
}

// Tile-order kernel for small buckets (at most 2 registers per lane): high
// occupancy; the groups take the tile's pixels from a shared cursor.
template <int V, int GA, class FT>
__global__ void __launch_bounds__(kThreads, 5) k_blend_fwd(RP P, const FT* __restrict__ feat, RasterWs ws,
                                                         FT* __restrict__ image, float* __restrict__ T_final,
                                                         int32_t* __restrict__ n_contrib) {
  __shared__ TileSmem S;
  const Group<GA> G;
  const int t = blockIdx.x;
  const int tx = t % P.tiles_x, ty = t / P.tiles_x;
  load_tile<false>(P, ws, tx, ty, nullptr, 2 * GA, S);
  fill_empty<FT>(P, tx, ty, S, image, T_final, n_contrib);
  // the next pixel is taken before the current one is blended
  for (int j = next_tile_pixel(G, S); j >= 0;) {
    const int jn = next_tile_pixel(G, S);
    const int m = S.m[j];
    const uint32_t s0 = S.s0[j];
    const long long q = tile_pixel_index(P, tx, ty, j);
    if (m <= GA) blend_fwd_reg<V, GA, FT, 1>(G, P, ws, s0, m, q, feat, image, T_final, n_contrib);
    else blend_fwd_reg<V, GA, FT, 2>(G, P, ws, s0, m, q, feat, image, T_final, n_contrib);
    j = jn;
  }
}

// List kernel for buckets of 2 GA < m <= 4 GA (R = 4, the list's front) or
// 4 GA < m <= kRegMax GA (R = kRegMax, the list's back): each group takes
// the next pixel of its list when it is done with one (bucket sizes differ
// by up to 4x, so a fixed stride leaves tails).
template <int V, int GA, class FT, int R>
__global__ void __launch_bounds__(kThreads, R == kRegMax ? 3 : 4) k_blend_fwd_large(RP P, const FT* __restrict__ feat,
                                                                                    RasterWs ws,
                                                                                    FT* __restrict__ image,
                                                                                    float* __restrict__ T_final,
                                                                                    int32_t* __restrict__ n_contrib) {
  const Group<GA> G;
  const bool wide = R == kRegMax;
  const uint32_t n_list = wide ? *ws.wide_count : *ws.large_count;
  uint32_t* cursor = wide ? ws.wide_next : ws.large_next;
  for (;;) {
    uint32_t h = 0;
    if (G.lg == 0) h = atomicAdd(cursor, 1u);
    h = G.bcast(h, 0);
    if (h >= n_list) break;
    const long long q = wide ? ws.large[P.n_pix - 1 - h] : ws.large[h];
    const uint32_t s0 = ws.pix_start[q];
    const int m = (int)(ws.pix_start[q + 1] - s0);
    blend_fwd_reg<V, GA, FT, R>(G, P, ws, s0, m, q, feat, image, T_final, n_contrib);
  }
}

// ------------------------------------------------------ group path (bwd) ---
// Pass 1 recomputes the forward's chunk scans (front to back) and keeps the
// transmittance in front of each chunk; pass 2 walks the blended chunks back
// to front accumulating S_k = sum_{j>k} T_j alpha_j (c_j . g) and writes
// fscal[4 p + c] = (T_k alpha_k, dL/dalpha_k = T_k (c_k . g) - S_k / (1 - alpha_k)) for the
// fragment k of point p at its footprint corner c.
template <int V, int GA, class FT, int R>
__device__ void blend_bwd_reg(const Group<GA>& G, const RP& P, const RasterWs& ws, uint32_t s0, int m, int nb,
                              long long pix, const FT* __restrict__ feat, const float* __restrict__ d_image) {
  const int qy = (int)(pix / P.cam.W), qx = (int)(pix - (long long)qy * P.cam.W);  // this pixel
  if constexpr (V == 2 && GA == 32) {  // F = 64
    blend_bwd_slots<FT, R>(G, P, ws, s0, m, nb, pix, feat, d_image);
    return;
  }
  if (nb == 0) return;
  const int ch = G.lg * V;
  uint32_t slot[R], idr[R];
  float a[R], Tc[R];
  float T = 1.0f;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    a[r] = 0.f;
    Tc[r] = T;
    slot[r] = 0;
    idr[r] = 0;
    const int b = r * GA;
    if (b < nb) {
      const bool valid = b + G.lg < nb;
      if (valid) {
        const uint2 o = order_at(P, ws, s0, m, b + G.lg);
        slot[r] = o.x;
        idr[r] = o.y;
        a[r] = ws.alpha[s0 + o.x];
      }
      const ChunkT<GA> ct = chunk_transmittance<GA>(G, P, a[r], valid, min(GA, nb - b), T);
      T = G.bcast(ct.Tn, ct.take - 1);
    }
  }
  float g[V];
  if (ch < P.F) load_vec<V>(d_image + pix * P.F + ch, g);
  else
#pragma unroll
    for (int v = 0; v < V; ++v) g[v] = 0.f;
  float S = 0.f;
#pragma unroll
  for (int r = R - 1; r >= 0; --r) {
    const int b = r * GA;
    if (b >= nb) continue;
    const bool valid = b + G.lg < nb;
    const long long id = idr[r];
    // issued here, used at the end of the chunk
    const uint32_t dst = valid ? frag_index(ws, (uint32_t)id, qx, qy) : 0u;
    const ChunkT<GA> ct = chunk_transmittance<GA>(G, P, a[r], valid, min(GA, nb - b), Tc[r]);
    float mydot = 0.f;
#pragma unroll 2
    for (int j = 0; j < ct.take; ++j) {
      const long long idj = G.bcast(id, j);
      float part = 0.f;
      if (ch < P.F) {
        float cc[V];
        load_color<V, FT>(P, feat, idj, ch, cc);
#pragma unroll
        for (int v = 0; v < V; ++v) part = __fmaf_rn(cc[v], g[v], part);
      }
      const float dj = G.sum(part);
      if (G.lg == j) mydot = dj;
    }
    const bool mine = G.lg < ct.take;
    const float wk = mine ? __fmul_rn(ct.Tk, a[r]) : 0.f;
    const float term = __fmul_rn(wk, mydot);
    const float suf = G.suffix_scan(term);             // this chunk, at or behind k
    const float Sk = __fadd_rn(S, G.shift_down(suf));  // strictly behind k
    const float da = __fsub_rn(__fmul_rn(ct.Tk, mydot), __fdiv_rn(Sk, __fsub_rn(1.0f, a[r])));
    if (mine) ws.fscal[dst] = make_float2(wk, da);
    S = __fadd_rn(S, G.bcast(suf, 0));
  }
}

template <int V, int GA, class FT>
__global__ void __launch_bounds__(kThreads, 4) k_blend_bwd(RP P, const FT* __restrict__ feat,
                                                         const int32_t* __restrict__ n_contrib,
                                                         const float* __restrict__ d_image, RasterWs ws) {
  __shared__ TileSmem S;
  const Group<GA> G;
  const int t = blockIdx.x;
  const int tx = t % P.tiles_x, ty = t / P.tiles_x;
  load_tile<true>(P, ws, tx, ty, n_contrib, 2 * GA, S);
  // the next pixel is taken before the current one is revisited
  for (int j = next_tile_pixel(G, S); j >= 0;) {
    const int jn = next_tile_pixel(G, S);
    const int nb = S.nb[j];
    const int m = S.m[j];
    const uint32_t s0 = S.s0[j];
    const long long q = tile_pixel_index(P, tx, ty, j);
    if (nb <= GA) blend_bwd_reg<V, GA, FT, 1>(G, P, ws, s0, m, nb, q, feat, d_image);
    else blend_bwd_reg<V, GA, FT, 2>(G, P, ws, s0, m, nb, q, feat, d_image);
    j = jn;
  }
}

template <int V, int GA, class FT>
__global__ void __launch_bounds__(kThreads, 3) k_blend_bwd_large(RP P, const FT* __restrict__ feat,
                                                               const int32_t* __restrict__ n_contrib,
                                                               const float* __restrict__ d_image, RasterWs ws) {
  const Group<GA> G;
  const uint32_t n_large = *ws.large_count;
  // as in the forward list kernel, each group takes the next pixel when done
  for (;;) {
    uint32_t h = 0;
    if (G.lg == 0) h = atomicAdd(ws.large_next, 1u);
    h = G.bcast(h, 0);
    if (h >= n_large) break;
    const long long q = ws.large[h];
    const uint32_t s0 = ws.pix_start[q];
    const int m = (int)(ws.pix_start[q + 1] - s0);
    const int nb = blended_count(n_contrib, q, m);
    if (nb <= 4 * GA) blend_bwd_reg<V, GA, FT, 4>(G, P, ws, s0, m, nb, q, feat, d_image);
    else blend_bwd_reg<V, GA, FT, kRegMax>(G, P, ws, s0, m, nb, q, feat, d_image);
  }
}

// --------------------------------------------------------------- CTA path ---
// Large buckets: the whole CTA sorts, scans and gathers for one pixel.
struct HeavySmem {
  float warp_tot[kWarps];
  float prev[kThreads];
  float red[kThreads];
  float red64[kWarps][64];  // per-warp partial colors of the 64-channel slot blend
  float carry;
  int stop;
};

// Inclusive product scan over the CTA's 256 threads (fixed order).
__device__ __forceinline__ float cta_prod_scan(float x, float* warp_tot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x = __fmul_rn(x, t);
  }
  __syncthreads();
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  float pre = 1.0f;
  for (int w = 0; w < wid; ++w) pre = __fmul_rn(pre, warp_tot[w]);
  return __fmul_rn(pre, x);
}

// Inclusive suffix-sum scan over the CTA's 256 threads (thread t gets the
// sum over threads >= t).
__device__ __forceinline__ float cta_suffix_scan(float x, float* warp_tot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float t = __shfl_down_sync(0xffffffffu, x, o);
    if (lane + o < 32) x += t;
  }
  __syncthreads();
  if (lane == 0) warp_tot[wid] = x;
  __syncthreads();
  float post = 0.0f;
  for (int w = kWarps - 1; w > wid; --w) post += warp_tot[w];
  return x + post;
}

// Transmittance in front of every fragment of a sorted bucket (product scan
// in chunks of 256), stored through t_store(k, T_k); returns the number of
// blended fragments and the final transmittance.
template <class AlphaAt, class TStore>
__device__ int cta_transmittance(const RP& P, AlphaAt alpha_at, int m, TStore t_store, HeavySmem& H, float* T_out) {
  float T = 1.0f;
  int n = m;
  for (int b = 0; b < m; b += kThreads) {
    const int k = b + threadIdx.x;
    const bool valid = k < m;
    const float a = valid ? alpha_at(k) : 0.f;
    const float incl = cta_prod_scan(__fsub_rn(1.0f, a), H.warp_tot);
    H.prev[threadIdx.x] = incl;
    if (threadIdx.x == 0) H.stop = INT_MAX;
    __syncthreads();
    const float ex = threadIdx.x > 0 ? H.prev[threadIdx.x - 1] : 1.0f;
    const float Tn = __fmul_rn(T, incl);
    if (valid) t_store(k, __fmul_rn(T, ex));
    if (valid && Tn < P.t_min) atomicMin(&H.stop, k);
    __syncthreads();
    const int st = H.stop;
    const int last = st != INT_MAX ? st : min(b + kThreads, m) - 1;
    if (k == last) H.carry = Tn;
    __syncthreads();
    T = H.carry;
    __syncthreads();
    if (st != INT_MAX) {
      n = st + 1;
      break;
    }
  }
  *T_out = T;
  return n;
}

// 64 channels on the CTA path: the 8 warps x 8 fragment slots take 64
// fragments per pass (lane: slot f = lane / 4, part q = lane % 4, 16
// channels), accumulate per slot, reduce-scatter within the warp and sum
// the 8 warps' partial colors in shared memory.
template <class FT, class KeyAt, class AlphaAt, class TLoad>
__device__ void blend_fwd_cta_slots(const RP& P, KeyAt key_at, AlphaAt alpha_at, TLoad t_load, int n, float T,
                                    long long pix, const FT* __restrict__ feat, FT* __restrict__ image,
                                    float* __restrict__ T_final, int32_t* __restrict__ n_contrib, HeavySmem& H) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int q = lane & 3, f = lane >> 2;
  float acc[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) acc[e] = 0.f;
#pragma unroll 2
  for (int k = 8 * wid + f; k < n; k += 64) {
    const float wk = __fmul_rn(t_load(k), alpha_at(k));
    float c[16];
    Slot64<FT>::load(feat + 64ll * (long long)(key_at(k) & P.idm), q, c);
    if (P.head && q == 0) c[0] = 1.0f;
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[e] = __fmaf_rn(wk, c[e], acc[e]);
  }
  const int h4 = (lane >> 4) & 1, h3 = (lane >> 3) & 1, h2 = (lane >> 2) & 1;
  float r8[8], r4[4], r2[2];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float send = h4 ? acc[k] : acc[8 + k];
    const float keep = h4 ? acc[8 + k] : acc[k];
    r8[k] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, 16));
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float send = h3 ? r8[k] : r8[4 + k];
    const float keep = h3 ? r8[4 + k] : r8[k];
    r4[k] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, 8));
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = h2 ? r4[k] : r4[2 + k];
    const float keep = h2 ? r4[2 + k] : r4[k];
    r2[k] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, 4));
  }
  const int ch0 = Slot64<FT>::channel(q, 8 * h4 + 4 * h3 + 2 * h2);
  __syncthreads();
  H.red64[wid][ch0] = r2[0];
  H.red64[wid][ch0 + 1] = r2[1];
  __syncthreads();
  if (threadIdx.x < 64) {  // warps 0 and 1, whole
    float sum = 0.f;
    for (int w = 0; w < kWarps; ++w) sum = __fadd_rn(sum, H.red64[w][threadIdx.x]);
    const float other = __shfl_down_sync(0xffffffffu, sum, 1);
    if (threadIdx.x % 2 == 0) Slot64<FT>::store2(image + pix * 64, threadIdx.x, sum, other);
  }
  if (threadIdx.x == 0) {
    T_final[pix] = T;
    n_contrib[pix] = n;
  }
  __syncthreads();
}

template <int V, int GA, class FT, class KeyAt, class AlphaAt, class TLoad>
__device__ void blend_fwd_cta(const RP& P, KeyAt key_at, AlphaAt alpha_at, TLoad t_load, int n, float T, long long pix,
                              const FT* __restrict__ feat, FT* __restrict__ image, float* __restrict__ T_final,
                              int32_t* __restrict__ n_contrib, HeavySmem& H) {
  if constexpr (V == 2 && GA == 32) {  // F = 64
    blend_fwd_cta_slots<FT>(P, key_at, alpha_at, t_load, n, T, pix, feat, image, T_final, n_contrib, H);
    return;
  }
  constexpr int kGroups = kThreads / GA;
  const Group<GA> G;
  const int group = threadIdx.x / GA;
  const int ch = G.lg * V;
  float C[V];
#pragma unroll
  for (int v = 0; v < V; ++v) C[v] = 0.f;
  if (ch < P.F) {
    for (int k = group; k < n; k += kGroups) {
      const float w = __fmul_rn(t_load(k), alpha_at(k));
      float c[V];
      load_color<V, FT>(P, feat, (long long)(key_at(k) & P.idm), ch, c);
#pragma unroll
      for (int v = 0; v < V; ++v) C[v] = __fmaf_rn(w, c[v], C[v]);
    }
  }
  // sum the groups' partial colors, one channel of each lane at a time
  for (int v = 0; v < V; ++v) {
    __syncthreads();
    H.red[threadIdx.x] = C[v];
    __syncthreads();
    if (threadIdx.x < GA) {
      float s = 0.f;
      for (int g2 = 0; g2 < kGroups; ++g2) s += H.red[g2 * GA + threadIdx.x];
      C[v] = s;
    }
  }
  if (threadIdx.x < GA) write_pixel<V>(P, pix, threadIdx.x * V, C, image);
  if (threadIdx.x == 0) {
    T_final[pix] = T;
    n_contrib[pix] = n;
  }
  __syncthreads();
}

// Backward on the CTA path: T_k via the forward's scan, c_k . g split over
// the groups, suffix sums by a CTA-wide reverse scan.
template <int V, int GA, class FT, class KeyAt, class AlphaAt, class DstAt, class TLoad, class DStore, class DLoad>
__device__ void blend_bwd_cta(const RP& P, KeyAt key_at, AlphaAt alpha_at, DstAt dst_at, TLoad t_load,
                              DStore d_store, DLoad d_load, int nb, long long pix, const FT* __restrict__ feat,
                              const float* __restrict__ d_image, float2* __restrict__ fscal, HeavySmem& H) {
  constexpr int kGroups = kThreads / GA;
  const Group<GA> G;
  const int group = threadIdx.x / GA;
  const int ch = G.lg * V;
  float g[V];
  if (ch < P.F) load_vec<V>(d_image + pix * P.F + ch, g);
  else
#pragma unroll
    for (int v = 0; v < V; ++v) g[v] = 0.f;
  for (int k = group; k < nb; k += kGroups) {
    float part = 0.f;
    if (ch < P.F) {
      float c[V];
      load_color<V, FT>(P, feat, (long long)(key_at(k) & P.idm), ch, c);
#pragma unroll
      for (int v = 0; v < V; ++v) part = __fmaf_rn(c[v], g[v], part);
    }
    const float d = G.sum(part);
    if (G.lg == 0) d_store(k, d);
  }
  __syncthreads();
  float S = 0.f;  // sum over the fragments behind the current 256-block
  const int n_blocks = (nb + kThreads - 1) / kThreads;
  for (int blk = n_blocks - 1; blk >= 0; --blk) {
    const int k = blk * kThreads + threadIdx.x;
    const bool valid = k < nb;
    const float a = valid ? alpha_at(k) : 0.f;
    const float Tk = valid ? t_load(k) : 0.f;
    const float dk = valid ? d_load(k) : 0.f;
    const float wk = __fmul_rn(Tk, a);
    const float term = __fmul_rn(wk, dk);
    const float suf = cta_suffix_scan(term, H.warp_tot);
    H.prev[threadIdx.x] = suf;
    __syncthreads();
    const float behind = threadIdx.x + 1 < kThreads ? H.prev[threadIdx.x + 1] : 0.f;
    const float Sk = __fadd_rn(S, behind);
    if (valid) fscal[dst_at(k)] = make_float2(wk, __fsub_rn(__fmul_rn(Tk, dk), __fdiv_rn(Sk, __fsub_rn(1.0f, a))));
    S = __fadd_rn(S, H.prev[0]);
    __syncthreads();
  }
}

struct HeavyBuf {
  unsigned long long* K;
  float* A;
  uint16_t* idx;
  float* Tk;
  uint32_t* pos;  // bucket position of a selected candidate
  __device__ explicit HeavyBuf(unsigned char* dyn) {
    K = reinterpret_cast<unsigned long long*>(dyn);
    A = reinterpret_cast<float*>(K + kHeavyKeys);
    Tk = A + kHeavyKeys;
    pos = reinterpret_cast<uint32_t*>(Tk + kHeavyKeys);
    idx = reinterpret_cast<uint16_t*>(pos + kHeavyKeys);
  }
  static constexpr size_t bytes() { return (size_t)kHeavyKeys * (8 + 4 + 4 + 4 + 2); }
};

// Front selection for the forward CTA path.  Blending stops once T drops
// below t_min, which on these buckets usually takes well under a hundred
// fragments, so only the front of a large bucket needs ordering: a 256-bin
// histogram of the FP32 depth bits (range [min, max] of the bucket, bins
// of 2^shift, monotone in depth) gives the smallest bin b* whose cumulative
// count reaches `want`; every key in bins < b* is nearer than every key in
// b* and above.  When b* holds many keys (a tight cluster of depths), a
// second 256-bin histogram over b*'s finer bits picks the sub-bin where the
// count reaches `want`.  Either way the selected keys (depth bits up to a
// threshold) are an exact prefix of the order.  Up to 256 candidates are
// sorted by one warp in registers (no barrier between the network's
// stages), more by the CTA in shared memory (bitonic_sort_idx).  Returns
// the candidate count C, or 0 when the prefix does not fit (C > kHeavyKeys).
// The caller blends the candidates when they reach t_min and otherwise asks
// again with a larger `want` (the depth range is measured once per pixel,
// on the first call).  (On the benchmark scene 99 % of the pixels blend at
// most 66 fragments; targets of 64 and 96 ran equally fast, 256 took 15 %
// longer.)
constexpr int kSelectWant = 96;

struct SelSmem {
  uint32_t dmin, dmax;
  int bstar, count, fill;
  uint32_t before;  // keys in the bins below b*
  int b2star;       // sub-bin of b* (-1: the whole bin)
};

// One warp sorts the C <= 32 R candidates B.K[0 .. C) and writes the
// blending order to B.idx.
template <int R>
__device__ __forceinline__ void warp_sort_candidates(const RP& P, const HeavyBuf& B, int C) {
  const Group<32> G;
  unsigned long long key[R];
  sort_loaded<32, R>(G, P, [&](int e) { return B.K[e]; }, C, key);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int k = r * 32 + G.lg;
    if (k < C) B.idx[k] = (uint16_t)reg_pos(key[r]);
  }
}

__device__ int cta_select_front(const RP& P, const RasterWs& ws, uint32_t s0, int m, const HeavyBuf& B, SortSmem& S,
                                SelSmem& X, int want, bool range_known) {
  const int lane = threadIdx.x & 31;
  // the sweeps load kUnroll keys per thread before using them, so that the
  // loads of a sweep are in flight together
  constexpr int kUnroll = 8;
  if (!range_known) {
    if (threadIdx.x == 0) {
      X.dmin = 0xFFFFFFFFu;
      X.dmax = 0u;
    }
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    for (int i0 = threadIdx.x; i0 < m; i0 += kUnroll * kThreads) {
      uint32_t d[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int i = i0 + u * kThreads;
        d[u] = i < m ? (uint32_t)(__ldg(ws.keys + s0 + i) >> P.idb) : 0u;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        if (i0 + u * kThreads < m) {
          lo = min(lo, d[u]);
          hi = max(hi, d[u]);
        }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    __syncthreads();
    if (lane == 0) {
      atomicMin(&X.dmin, lo);
      atomicMax(&X.dmax, hi);
    }
  }
  if (threadIdx.x == 0) {
    X.fill = 0;
    X.bstar = 255;  // reached below whenever want <= m
    X.count = m;
    X.before = 0;
    X.b2star = -1;
  }
  S.hist[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t dmin = X.dmin, span = X.dmax - X.dmin;
  int shift = 0;
  while ((span >> shift) > 255u) ++shift;
  for (int i0 = threadIdx.x; i0 < m; i0 += kUnroll * kThreads) {
    uint32_t d[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = i0 + u * kThreads;
      d[u] = i < m ? (uint32_t)(__ldg(ws.keys + s0 + i) >> P.idb) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
      if (i0 + u * kThreads < m) atomicAdd(&S.hist[(d[u] - dmin) >> shift], 1u);
  }
  __syncthreads();
  {
    const uint32_t h = S.hist[threadIdx.x];
    const uint32_t ex = cta_excl_scan256(h, S.warp_sums);  // bins below this thread's bin
    if (ex < (uint32_t)want && ex + h >= (uint32_t)want) {
      X.bstar = threadIdx.x;
      X.count = (int)(ex + h);
      X.before = ex;
    }
  }
  __syncthreads();
  const uint32_t bstar = (uint32_t)X.bstar;
  // sub-bins of b*: the next (at most 8) depth bits below the bin's
  const int subshift = shift > 8 ? shift - 8 : 0;
  const uint32_t submask = (1u << (shift - subshift)) - 1u;
  if (X.count > 256 && shift > 0) {
    S.hist[threadIdx.x] = 0;
    __syncthreads();
    for (int i0 = threadIdx.x; i0 < m; i0 += kUnroll * kThreads) {
      uint32_t d[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int i = i0 + u * kThreads;
        d[u] = i < m ? (uint32_t)(__ldg(ws.keys + s0 + i) >> P.idb) : 0u;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        if (i0 + u * kThreads < m && ((d[u] - dmin) >> shift) == bstar)
          atomicAdd(&S.hist[((d[u] - dmin) >> subshift) & submask], 1u);
    }
    __syncthreads();
    const uint32_t before = X.before;
    const uint32_t h = S.hist[threadIdx.x];
    const uint32_t ex = cta_excl_scan256(h, S.warp_sums);
    if (before + ex < (uint32_t)want && before + ex + h >= (uint32_t)want) {
      X.b2star = threadIdx.x;
      X.count = (int)(before + ex + h);
    }
    __syncthreads();
  }
  const int C = X.count;
  const int b2star = X.b2star;
  if (C > kHeavyKeys) return 0;
  for (int i0 = threadIdx.x; i0 < m; i0 += kUnroll * kThreads) {
    unsigned long long key[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = i0 + u * kThreads;
      key[u] = i < m ? __ldg(ws.keys + s0 + i) : ~0ull;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = i0 + u * kThreads;
      const uint32_t dd = (uint32_t)(key[u] >> P.idb) - dmin;
      const uint32_t bin = dd >> shift;
      const bool take = bin < bstar || (bin == bstar && (b2star < 0 || ((dd >> subshift) & submask) <= (uint32_t)b2star));
      if (i < m && take) {
        const int slot = atomicAdd(&X.fill, 1);
        B.K[slot] = key[u];
        B.A[slot] = ws.alpha[s0 + i];
        B.pos[slot] = (uint32_t)i;
        B.idx[slot] = (uint16_t)slot;
      }
    }
  }
  __syncthreads();
  if (C <= 256) {
    if (threadIdx.x < 32) {
      if (C <= 128) warp_sort_candidates<4>(P, B, C);
      else warp_sort_candidates<8>(P, B, C);
    }
    __syncthreads();
  } else {
    bitonic_sort_idx(B.K, B.idx, C, threadIdx.x, kThreads, [] { __syncthreads(); });
  }
  return C;
}

// Sort one large bucket: in shared memory (m <= kHeavyKeys) through the
// index array, or in global memory (ka/va) beyond that.
__device__ void cta_order_bucket(const RasterWs& ws, uint32_t s0, int m, const HeavyBuf& B, SortSmem& S) {
  if (m <= kHeavyKeys) {
    for (int j = threadIdx.x; j < m; j += kThreads) {
      B.K[j] = ws.keys[s0 + j];
      B.A[j] = ws.alpha[s0 + j];
      B.pos[j] = (uint32_t)j;
      B.idx[j] = (uint16_t)j;
    }
    __syncthreads();
    bitonic_sort_idx(B.K, B.idx, m, threadIdx.x, kThreads, [] { __syncthreads(); });
  } else {
    cta_sort_global(ws.keys + s0, m, ws.ka + s0, ws.va + s0, ws.kb + s0, ws.vb + s0, S);
  }
}

template <int V, int GA, class FT>
__global__ void __launch_bounds__(kThreads, 4) k_blend_fwd_heavy(RP P, const FT* __restrict__ feat, RasterWs ws,
                                                               FT* __restrict__ image, float* __restrict__ T_final,
                                                               int32_t* __restrict__ n_contrib) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ SortSmem S;
  __shared__ HeavySmem H;
  __shared__ SelSmem X;
  const HeavyBuf B(dyn);
  __shared__ uint32_t next;
  const uint32_t n_heavy = *ws.heavy_count;
  // the CTA takes the next pixel of the list when it is done with one; every
  // iteration ends with a barrier, so `next` is read before it is rewritten
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(ws.heavy_next, 1u);
    __syncthreads();
    const uint32_t h = next;
    if (h >= n_heavy) break;
    const long long q = ws.heavy[h];
    const uint32_t s0 = ws.pix_start[q];
    const int m = (int)(ws.pix_start[q + 1] - s0);
    float T;
    bool done = false;
    // the nearest 96 fragments, then 384, then 1,536, until the candidates
    // reach t_min; only then (or when they do not fit) the whole bucket
    for (int want = kSelectWant; !done && 2 * want < m && want <= kHeavyKeys; want *= 4) {
      const int C = cta_select_front(P, ws, s0, m, B, S, X, want, want != kSelectWant);
      if (C == 0) break;
      auto key_at = [&](int k) { return B.K[B.idx[k]]; };
      auto alpha_at = [&](int k) { return B.A[B.idx[k]]; };
      const int n = cta_transmittance(P, alpha_at, C, [&](int k, float v) { B.Tk[k] = v; }, H, &T);
      if (T < P.t_min || C == m) {  // the candidates reach the stop: the prefix is all that blends
        for (int k = threadIdx.x; k < n; k += kThreads)
          ws.order[s0 + k] = make_uint2(B.pos[B.idx[k]], (uint32_t)(B.K[B.idx[k]] & P.idm));
        __syncthreads();
        blend_fwd_cta<V, GA, FT>(P, key_at, alpha_at, [&](int k) { return B.Tk[k]; }, n, T, q, feat, image,
                             T_final, n_contrib, H);
        done = true;
      }
      __syncthreads();
    }
    if (done) continue;
    cta_order_bucket(ws, s0, m, B, S);
    if (m <= kHeavyKeys) {
      auto key_at = [&](int k) { return B.K[B.idx[k]]; };
      auto alpha_at = [&](int k) { return B.A[B.idx[k]]; };
      const int n = cta_transmittance(P, alpha_at, m, [&](int k, float v) { B.Tk[k] = v; }, H, &T);
      for (int k = threadIdx.x; k < n; k += kThreads)
        ws.order[s0 + k] = make_uint2(B.pos[B.idx[k]], (uint32_t)(B.K[B.idx[k]] & P.idm));
      __syncthreads();
      blend_fwd_cta<V, GA, FT>(P, key_at, alpha_at, [&](int k) { return B.Tk[k]; }, n, T, q, feat, image, T_final,
                           n_contrib, H);
    } else {
      const unsigned long long* ka = ws.ka + s0;
      const uint32_t* va = ws.va + s0;
      float2* tmp = reinterpret_cast<float2*>(ws.kb + s0);
      auto key_at = [&](int k) { return ka[k]; };
      auto alpha_at = [&](int k) { return ws.alpha[s0 + va[k]]; };
      const int n = cta_transmittance(P, alpha_at, m, [&](int k, float v) { tmp[k].x = v; }, H, &T);
      for (int k = threadIdx.x; k < n; k += kThreads) ws.order[s0 + k] = make_uint2(va[k], (uint32_t)(ka[k] & P.idm));
      __syncthreads();
      blend_fwd_cta<V, GA, FT>(P, key_at, alpha_at, [&](int k) { return tmp[k].x; }, n, T, q, feat, image, T_final,
                           n_contrib, H);
    }
    __syncthreads();
  }
}

// Backward of the pixels with more than kRegMax * GA blended fragments: the
// whole CTA on one pixel, over the blended prefix the forward recorded (no
// sort); T_k and c_k . g in shared memory (or, beyond kHeavyKeys, in the
// global scratch kb).
struct HeavyBwdBuf {
  float* Tk;
  float* D;
  __device__ explicit HeavyBwdBuf(unsigned char* dyn) {
    Tk = reinterpret_cast<float*>(dyn);
    D = Tk + kHeavyKeys;
  }
  static constexpr size_t bytes() { return (size_t)kHeavyKeys * 8; }
};

template <int V, int GA, class FT>
__global__ void __launch_bounds__(kThreads) k_blend_bwd_heavy(RP P, const FT* __restrict__ feat,
                                                               const int32_t* __restrict__ n_contrib,
                                                               const float* __restrict__ d_image, RasterWs ws) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ HeavySmem H;
  const HeavyBwdBuf B(dyn);
  const uint32_t n_heavy = *ws.heavy_count;
  for (uint32_t h = blockIdx.x; h < n_heavy; h += gridDim.x) {
    const long long q = ws.heavy[h];
    const uint32_t s0 = ws.pix_start[q];
    const int m = (int)(ws.pix_start[q + 1] - s0);
    const int nb = blended_count(n_contrib, q, m);
    auto key_at = [&](int k) { return (unsigned long long)order_at(P, ws, s0, m, k).y; };
    auto alpha_at = [&](int k) { return ws.alpha[s0 + order_at(P, ws, s0, m, k).x]; };
    const int qy = (int)(q / P.cam.W), qx = (int)(q - (long long)qy * P.cam.W);
    auto dst_at = [&](int k) { return frag_index(ws, order_at(P, ws, s0, m, k).y, qx, qy); };
    float T;
    if (nb <= kHeavyKeys) {
      cta_transmittance(P, alpha_at, nb, [&](int k, float v) { B.Tk[k] = v; }, H, &T);
      __syncthreads();
      blend_bwd_cta<V, GA, FT>(P, key_at, alpha_at, dst_at, [&](int k) { return B.Tk[k]; },
                           [&](int k, float v) { B.D[k] = v; }, [&](int k) { return B.D[k]; }, nb, q, feat, d_image,
                           ws.fscal, H);
    } else {
      float2* tmp = reinterpret_cast<float2*>(ws.kb + s0);
      cta_transmittance(P, alpha_at, nb, [&](int k, float v) { tmp[k].x = v; }, H, &T);
      __syncthreads();
      blend_bwd_cta<V, GA, FT>(P, key_at, alpha_at, dst_at, [&](int k) { return tmp[k].x; },
                           [&](int k, float v) { tmp[k].y = v; }, [&](int k) { return tmp[k].y; }, nb, q, feat,
                           d_image, ws.fscal, H);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------ per-point gradient ---
// Per point: gather the scalars of its (at most four) splats and the
// upstream-gradient rows of their pixels.  d_feat row = sum_k (T_k alpha_k) g_k;
// d alpha_h = sum_k w_k [unclamped] dL/dalpha_k.
template <int V, int GA, class FT>
__global__ void __launch_bounds__(kThreads) k_point_grad(RP P, const float* __restrict__ pos,
                                                          const float* __restrict__ opacity,
                                                          const FT* __restrict__ feat,
                                                          const float* __restrict__ d_image, RasterWs ws,
                                                          float* __restrict__ d_opacity, float* __restrict__ d_feat) {
  constexpr int kGroups = kThreads / GA;
  const Group<GA> G;
  const int ch = G.lg * V;
  const bool active = ch < P.F;
  const long long g0 = (long long)blockIdx.x * kGroups + threadIdx.x / GA;
  for (long long id = g0; id < P.n; id += (long long)gridDim.x * kGroups) {
    const uint4 sl = __ldg(reinterpret_cast<const uint4*>(ws.pslot) + id);
    const uint32_t slots[4] = {sl.x, sl.y, sl.z, sl.w};
    float dc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) dc[v] = 0.f;
    float dah = 0.f, e_h0 = 0.f;
    Splat s;
    if ((sl.x & sl.y & sl.z & sl.w) != kNoSlot) {
      splat_point(P, pos, id, s);
      const float ah = point_alpha_h(P, opacity, feat, id, &e_h0);
      float2 sc[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) sc[k] = slots[k] == kNoSlot ? make_float2(0.f, 0.f) : __ldg(ws.fscal + 4 * id + k);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (slots[k] == kNoSlot) continue;
        const float w = corner_weight(s.f, k & 1, k >> 1);
        if (__fmul_rn(ah, w) <= P.alpha_max) dah = __fmaf_rn(w, sc[k].y, dah);
        if (active) {
          const long long pix = (long long)(s.f.j0 + (k >> 1)) * P.cam.W + (s.f.i0 + (k & 1));
          float g[V];
          load_vec<V>(d_image + pix * P.F + ch, g);
#pragma unroll
          for (int v = 0; v < V; ++v) dc[v] = __fmaf_rn(sc[k].x, g[v], dc[v]);
        }
      }
    }
    // head mode: channel 0 of the blended color is the constant 1; the
    // opacity gradient reaches h0 through alpha_h = 1 - exp(-exp(h0))
    if (P.head && G.lg == 0) dc[0] = dah * (e_h0 * expf(-e_h0));
    if (active) {
      float* o = d_feat + id * P.F + ch;
      if (V == 4) *reinterpret_cast<float4*>(o) = make_float4(dc[0], dc[1], dc[2], dc[3]);
      else if (V == 2) *reinterpret_cast<float2*>(o) = make_float2(dc[0], dc[1]);
      else
#pragma unroll
        for (int v = 0; v < V; ++v) o[v] = dc[v];
    }
    if (!P.head && G.lg == 0) d_opacity[id] = dah;
  }
}

// ---------------------------------------------------------------- host ---
// max_n: 2^28 for the forward alone (and its workspace), 2^25 for the calls
// that continue from it (backward, per-point blending weights).
inpc_status make_rp(const inpc_camera* cam, const inpc_raster_opts* o, int64_t n, RP& P,
                    int64_t max_n = int64_t(1) << kIdBits) {
  if (!cam || !o) return fail(INPC_ERR_INVALID_ARG, "camera or options is null");
  if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
    return fail(INPC_ERR_INVALID_ARG, "image size %dx%d out of range", cam->width, cam->height);
  if (!(cam->near_plane > 0.0f) || !(cam->far_plane > cam->near_plane))
    return fail(INPC_ERR_INVALID_ARG, "need 0 < near < far");
  if (n < 0 || n > max_n) return fail(INPC_ERR_CAPACITY, "n must be in [0, 2^%d]", max_n > (int64_t(1) << kIdBits) ? 28 : 25);
  if (n <= (int64_t(1) << kIdBits)) {
    P.idb = kIdBits;
    P.dbase = 0u;
  } else {
    P.idb = 64 - __builtin_clzll((unsigned long long)(n - 1));
    uint32_t nb, fb;
    std::memcpy(&nb, &cam->near_plane, 4);
    std::memcpy(&fb, &cam->far_plane, 4);
    P.dbase = nb;
    // kept depths lie strictly inside (near, far): their field is below fb - nb
    if ((unsigned long long)(fb - nb) >= (1ull << (kKeyBits - P.idb)))
      return fail(INPC_ERR_CAPACITY, "far/near = %g/%g leaves too few depth bits beside %d-bit point indices",
                  (double)cam->far_plane, (double)cam->near_plane, P.idb);
  }
  P.idm = (1ull << P.idb) - 1;
  if (o->opacity_mode != INPC_OPACITY_GIVEN && o->opacity_mode != INPC_OPACITY_FROM_CH0)
    return fail(INPC_ERR_INVALID_ARG, "bad opacity_mode");
  if ((o->feat_dtype != INPC_F32 && o->feat_dtype != INPC_BF16) || o->image_dtype != o->feat_dtype)
    return fail(INPC_ERR_UNSUPPORTED, "feat_dtype must be INPC_F32 or INPC_BF16 and image_dtype must equal it");
  if (o->n_channels < 1 || o->n_channels > 128) return fail(INPC_ERR_UNSUPPORTED, "n_channels must be in [1, 128]");
  if (o->n_channels % 4 != 0 && o->n_channels > 32)
    return fail(INPC_ERR_UNSUPPORTED, "n_channels > 32 must be a multiple of 4");
  if (!(o->t_min >= 0.0f && o->t_min < 1.0f)) return fail(INPC_ERR_INVALID_ARG, "t_min must be in [0, 1)");
  if (!(o->alpha_max > 0.0f && o->alpha_max < 1.0f)) return fail(INPC_ERR_INVALID_ARG, "alpha_max must be in (0, 1)");
  P.cam = to_cam(*cam);
  P.TW = o->tile_w > 0 ? o->tile_w : 16;
  P.TH = o->tile_h > 0 ? o->tile_h : 8;
  if (P.TW * P.TH > 256) return fail(INPC_ERR_INVALID_ARG, "tile_w * tile_h must be <= 256");
  P.tiles_x = (int)ceil_div(cam->width, P.TW);
  P.tiles_y = (int)ceil_div(cam->height, P.TH);
  P.n_tiles = P.tiles_x * P.tiles_y;
  P.F = o->n_channels;
  P.head = o->opacity_mode == INPC_OPACITY_FROM_CH0;
  P.bf16 = o->feat_dtype == INPC_BF16;
  P.t_min = o->t_min;
  P.alpha_max = o->alpha_max;
  P.n = n;
  P.n_pix = (long long)cam->width * cam->height;
  return INPC_OK;
}

int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// (V, GA): V channels per lane, GA lanes per pixel.  Channel counts that are
// multiples of 32 use full warps; other multiples of 4 use V = 4 and the next
// power of two of F / 4 lanes; anything else (F <= 32) uses one channel per
// lane of a full warp.
template <class Fn>
inpc_status dispatch(int F, Fn&& fn) {
  using I = std::integral_constant<int, 1>;
  using II = std::integral_constant<int, 2>;
  using IV = std::integral_constant<int, 4>;
  using W = std::integral_constant<int, 32>;
  if (F == 32) return fn(I(), W());
  if (F == 64) return fn(II(), W());
  if (F == 128) return fn(IV(), W());
  if (F % 4 == 0) {
    switch (next_pow2(F / 4)) {
      case 1: return fn(IV(), std::integral_constant<int, 1>());
      case 2: return fn(IV(), std::integral_constant<int, 2>());
      case 4: return fn(IV(), std::integral_constant<int, 4>());
      case 8: return fn(IV(), std::integral_constant<int, 8>());
      case 16: return fn(IV(), std::integral_constant<int, 16>());
      case 32: return fn(IV(), W());
    }
  }
  if (F <= 32) return fn(I(), W());
  return fail(INPC_ERR_UNSUPPORTED, "no kernel for n_channels = %d", F);
}

unsigned point_grid(long long n) {
  const long long cap = (long long)device_sm_count() * 16;
  return (unsigned)std::max<long long>(1, std::min<long long>(ceil_div(n, 256), cap));
}

// Raises a kernel's dynamic shared-memory limit once per device (the
// attribute belongs to the kernel on the current device).
struct SmemOnce {
  std::mutex mu;
  uint64_t done = 0;  // bit d: set on device d
};

template <class K>
inpc_status set_smem(K kernel, size_t bytes, SmemOnce& once) {
  int dev = 0;
  INPC_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  std::lock_guard<std::mutex> lk(once.mu);
  const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
  if (bit && (once.done & bit)) return INPC_OK;
  INPC_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes),
            "cudaFuncSetAttribute");
  once.done |= bit;
  return INPC_OK;
}

// Forward binning: per-pixel counts, offsets, buckets (keys and alphas),
// per-point slots and the list of pixels for the CTA path (all kept in the
// workspace for the backward).
template <class FT>
inpc_status bin_fragments(const RP& P, const float* pos, const float* opacity, const FT* feat, const RasterWs& ws,
                          uint32_t cap_small, uint32_t cap_group, cudaStream_t s) {
  INPC_CUDA(cudaMemsetAsync(ws.pix_count, 0, sizeof(uint32_t) * P.n_pix, s), "clear pixel counts");
  if (P.n > 0) {
    INPC_TIMED("k_pix_count", s, k_pix_count<<<point_grid(P.n), 256, 0, s>>>(P, pos, ws.pix_count));
    INPC_TRY(check_launch("k_pix_count"));
  }
  INPC_TRY((scan::run<uint32_t, CountLoad, false>(CountLoad{ws.pix_count}, P.n_pix, ws.pix_start, ws.tops, s)));
  const long long nb = ceil_div(P.n_pix, scan::kBlock);
  k_classify<<<(unsigned)ceil_div(P.n_pix, 256), 256, 0, s>>>(ws.pix_start, P.n_pix, ws.tops, nb, cap_small, cap_group,
                                                               ws.heavy, ws.heavy_count, ws.large, ws.large_count,
                                                               ws.pix_start, 4 * (cap_small / 2), ws.wide_count);
  INPC_TRY(check_launch("k_classify"));
  if (P.n > 0) {
    INPC_TIMED("k_pix_scatter", s,
               k_pix_scatter<FT><<<point_grid(P.n), 256, 0, s>>>(P, pos, opacity, feat, ws.pix_start, ws.pix_count,
                                                                 ws.keys, ws.alpha, ws.pslot, ws.porg, ws.pexp));
    INPC_TRY(check_launch("k_pix_scatter"));
  }
  return INPC_OK;
}

template <int V, int GA, class FT>
inpc_status launch_fwd(const RP& P, const float* pos, const float* opacity, const FT* feat, const RasterWs& ws,
                       FT* image, float* T_final, int32_t* n_contrib, cudaStream_t s) {
  INPC_TRY(bin_fragments(P, pos, opacity, feat, ws, 2 * GA, GA * kRegMax, s));
  static SmemOnce f2;
  INPC_TRY(set_smem(k_blend_fwd_heavy<V, GA, FT>, HeavyBuf::bytes(), f2));
  INPC_TIMED("k_blend_fwd", s,
             k_blend_fwd<V, GA, FT><<<P.n_tiles, kThreads, 0, s>>>(P, feat, ws, image, T_final, n_contrib));
  INPC_TRY(check_launch("k_blend_fwd"));
  INPC_TIMED("k_blend_fwd_large", s,
             k_blend_fwd_large<V, GA, FT, 4><<<device_sm_count() * 4, kThreads, 0, s>>>(P, feat, ws, image, T_final,
                                                                                      n_contrib));
  INPC_TRY(check_launch("k_blend_fwd_large"));
  INPC_TIMED("k_blend_fwd_large", s,
             k_blend_fwd_large<V, GA, FT, kRegMax><<<device_sm_count() * 3, kThreads, 0, s>>>(P, feat, ws, image,
                                                                                            T_final, n_contrib));
  INPC_TRY(check_launch("k_blend_fwd_large"));
  INPC_TIMED("k_blend_fwd_heavy", s,
             k_blend_fwd_heavy<V, GA, FT><<<device_sm_count() * 4, kThreads, HeavyBuf::bytes(), s>>>(
                 P, feat, ws, image, T_final, n_contrib));
  return check_launch("k_blend_fwd_heavy");
}

template <int V, int GA, class FT>
inpc_status launch_blend_bwd(const RP& P, const FT* feat, const int32_t* n_contrib, const float* d_image,
                             const RasterWs& ws, cudaStream_t s) {
  // fragments that were not blended keep zero scalars
  INPC_CUDA(cudaMemsetAsync(ws.fscal, 0, sizeof(float2) * std::max<long long>(4 * P.n, 1), s), "clear fscal");
  // the class counts and the list cursors (header words 1-4; the forward's
  // kernels are done with them)
  INPC_CUDA(cudaMemsetAsync(ws.heavy_count, 0, 4 * sizeof(uint32_t), s), "clear class counts");
  INPC_TIMED("k_classify_bwd", s,
             k_classify_bwd<<<(unsigned)ceil_div(P.n_pix, 256), 256, 0, s>>>(
                 n_contrib, ws.pix_start, P.n_pix, 2 * GA, GA * kRegMax, ws.heavy, ws.heavy_count, ws.large,
                 ws.large_count));
  INPC_TRY(check_launch("k_classify_bwd"));
  INPC_TIMED("k_blend_bwd", s, k_blend_bwd<V, GA, FT><<<P.n_tiles, kThreads, 0, s>>>(P, feat, n_contrib, d_image, ws));
  INPC_TRY(check_launch("k_blend_bwd"));
  INPC_TIMED("k_blend_bwd_large", s,
             k_blend_bwd_large<V, GA, FT><<<device_sm_count() * 3, kThreads, 0, s>>>(P, feat, n_contrib, d_image, ws));
  INPC_TRY(check_launch("k_blend_bwd_large"));
  INPC_TIMED("k_blend_bwd_heavy", s,
             k_blend_bwd_heavy<V, GA, FT><<<device_sm_count() * 4, kThreads, HeavyBwdBuf::bytes(), s>>>(
                 P, feat, n_contrib, d_image, ws));
  return check_launch("k_blend_bwd_heavy");
}

template <int V, int GA, class FT>
inpc_status launch_bwd(const RP& P, const float* pos, const float* opacity, const FT* feat,
                       const int32_t* n_contrib, const float* d_image, const RasterWs& ws, float* d_opacity,
                       float* d_feat, cudaStream_t s) {
  INPC_TRY((launch_blend_bwd<V, GA, FT>(P, feat, n_contrib, d_image, ws, s)));
  constexpr int kGroups = kThreads / GA;
  const long long grid = std::min<long long>(ceil_div(P.n, kGroups), (long long)device_sm_count() * 32);
  INPC_TIMED("k_point_grad", s,
             k_point_grad<V, GA, FT><<<(unsigned)std::max<long long>(grid, 1), kThreads, 0, s>>>(
                 P, pos, opacity, feat, d_image, ws, d_opacity, d_feat));
  return check_launch("k_point_grad");
}

}  // namespace
}  // namespace inpc

