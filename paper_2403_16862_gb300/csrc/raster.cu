// raster.cu -- differentiable bilinear point rasterizer (Sec. 3.4, Eq. 1,
// Eq. 5, Eq. 6, App. A.6, Algorithm 1), forward and backward.
//
// Algorithm 1's global "RadixSortPairs" over (pixel, depth) keys is replaced
// by a two-level radix ordering:
//   1. k_bin_count / k_scan_tiles / k_bin_scatter: a counting sort of the
//      fragments by screen tile (the most significant digit).  Each point's
//      fragments in one tile land in consecutive slots (point-grouped).
//      Fragment record: 64-bit key = pixel-in-tile (8 bits) | FP32 depth
//      bits (31, depth > 0) | point index (25).
//   2. per tile, one CTA orders its bucket by the remaining key bits:
//      fast path -- the bucket fits in shared memory: counting sort by
//      pixel, then an all-ascending bitonic network per pixel segment;
//      fallback -- a stable 8-bit LSD radix sort of the bucket in global
//      memory by the same CTA (digits that are constant in the bucket are
//      skipped).  Both give the (pixel, depth, point) order exactly.
// Blending runs in the same CTA: a group of GA lanes owns one pixel, each
// lane V contiguous channels (float4 loads of the point's feature row).
// The backward revisits each pixel's blended fragments back to front,
// recovering T_k = T_{k+1} / (1 - alpha_k) from T_final, and stores two
// scalars per fragment (T_k alpha_k and dL/dalpha_k) in shared memory; the
// per-point gradient is then assembled from the point-grouped bucket order
// with plain stores (atomics only for points whose footprint spans tiles).
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace inpc {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kIdBits = 25;
constexpr unsigned long long kIdMask = (1ull << kIdBits) - 1;
constexpr int kCapFwd = 8192;  // fragments per tile on the shared-memory path (forward)
constexpr int kCapBwd = 4096;  // ... (backward: key + index + two scalars per fragment)

struct RP {
  Cam cam;
  int TW, TH, tiles_x, tiles_y, n_tiles;
  int F;
  int head;
  float t_min, alpha_max;
  long long n;
};

struct RasterWs {
  uint32_t* status;
  uint32_t* tile_count;   // [n_tiles]
  uint32_t* tile_offset;  // [n_tiles + 1]
  uint32_t* tile_cursor;  // [n_tiles]
  unsigned long long* keys;  // [4n] binned fragments
  unsigned long long* ka;    // [4n] per-tile sorted keys (fallback path)
  uint32_t* va;              // [4n] their bucket positions
  unsigned long long* kb;    // [4n] scratch
  uint32_t* vb;              // [4n] scratch
  float2* fscal;             // [4n] backward per-fragment scalars (fallback path)
  size_t bytes;
};

RasterWs carve(void* base, int n_tiles, long long n) {
  Carver c(base);
  RasterWs w;
  w.status = reinterpret_cast<uint32_t*>(base);
  const long long nf = std::max<long long>(4 * n, 1);
  w.tile_count = c.take<uint32_t>(n_tiles);
  w.tile_offset = c.take<uint32_t>(n_tiles + 1);
  w.tile_cursor = c.take<uint32_t>(n_tiles);
  w.keys = c.take<unsigned long long>(nf);
  w.ka = c.take<unsigned long long>(nf);
  w.va = c.take<uint32_t>(nf);
  w.kb = c.take<unsigned long long>(nf);
  w.vb = c.take<uint32_t>(nf);
  w.fscal = c.take<float2>(nf);
  w.bytes = c.bytes();
  return w;
}

// ------------------------------------------------------------ splatting ---
struct Splat {
  Footprint f;
  float d;
};

__device__ __forceinline__ bool splat_point(const RP& P, const float* __restrict__ pos, long long id, Splat& s) {
  float u, v;
  const float x = __ldg(pos + 3 * id), y = __ldg(pos + 3 * id + 1), z = __ldg(pos + 3 * id + 2);
  if (!project_point(P.cam, x, y, z, u, v, s.d)) return false;
  return footprint(P.cam, u, v, s.f);
}

// Tile of corner k (= a + 2b) of a footprint, or -1 if the pixel is off-image.
__device__ __forceinline__ int corner_tile(const RP& P, const Footprint& f, int k, int& px, int& py) {
  px = f.i0 + (k & 1);
  py = f.j0 + (k >> 1);
  if (px < 0 || px >= P.cam.W || py < 0 || py >= P.cam.H) return -1;
  return (py / P.TH) * P.tiles_x + (px / P.TW);
}

__device__ __forceinline__ float point_alpha_h(const RP& P, const float* __restrict__ opacity,
                                               const float* __restrict__ feat, long long id, float* e_h0) {
  if (P.head) {
    const float e = expf(__ldg(feat + (long long)P.F * id));
    if (e_h0) *e_h0 = e;
    return -expm1f(-e);
  }
  return __ldg(opacity + id);
}

__device__ __forceinline__ float splat_alpha(const RP& P, float ah, float w) {
  return fminf(__fmul_rn(ah, w), P.alpha_max);
}

// ---------------------------------------------------------------- binning ---
__global__ void __launch_bounds__(256) k_bin_count(RP P, const float* __restrict__ pos, uint32_t* tile_count) {
  const unsigned full = 0xffffffffu;
  for (long long base = blockIdx.x * (long long)blockDim.x; base < P.n; base += (long long)gridDim.x * blockDim.x) {
    const long long id = base + threadIdx.x;
    int tile[4] = {-1, -1, -1, -1};
    Splat s;
    if (id < P.n && splat_point(P, pos, id, s)) {
      for (int k = 0; k < 4; ++k) {
        int px, py;
        tile[k] = corner_tile(P, s.f, k, px, py);
      }
    }
    // distinct tiles of this point with their corner counts; warp-aggregate
    for (int k = 0; k < 4; ++k) {
      int t = tile[k];
      uint32_t cnt = 0;
      if (t >= 0) {
        bool first = true;
        for (int q = 0; q < k; ++q) first &= (tile[q] != t);
        if (first)
          for (int q = k; q < 4; ++q) cnt += (tile[q] == t);
        else
          t = -1;
      }
      const unsigned peers = __match_any_sync(full, t);
      const uint32_t sum = __reduce_add_sync(peers, cnt);
      if (t >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(tile_count + t, sum);
    }
  }
}

__global__ void __launch_bounds__(1024) k_scan_tiles(const uint32_t* __restrict__ cnt, int n_tiles,
                                                     uint32_t* __restrict__ offset, uint32_t* __restrict__ cursor) {
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t chunk_total;
  uint32_t carry = 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int b0 = 0; b0 < n_tiles; b0 += 1024) {
    const int i = b0 + threadIdx.x;
    const uint32_t v = i < n_tiles ? cnt[i] : 0u;
    uint32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const uint32_t s = warp_sums[lane];
      uint32_t si = s;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, si, o);
        if (lane >= o) si += t;
      }
      warp_sums[lane] = si - s;
      if (lane == 31) chunk_total = si;
    }
    __syncthreads();
    if (i < n_tiles) {
      offset[i] = carry + warp_sums[wid] + incl - v;
      cursor[i] = 0;
    }
    carry += chunk_total;
    __syncthreads();
  }
  if (threadIdx.x == 0) offset[n_tiles] = carry;
}

__global__ void __launch_bounds__(256) k_bin_scatter(RP P, const float* __restrict__ pos,
                                                     const uint32_t* __restrict__ tile_offset,
                                                     uint32_t* __restrict__ tile_cursor,
                                                     unsigned long long* __restrict__ keys) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  for (long long base = blockIdx.x * (long long)blockDim.x; base < P.n; base += (long long)gridDim.x * blockDim.x) {
    const long long id = base + threadIdx.x;
    int tile[4] = {-1, -1, -1, -1};
    int pix[4] = {0, 0, 0, 0};
    Splat s;
    s.d = 0.f;
    if (id < P.n && splat_point(P, pos, id, s)) {
      for (int k = 0; k < 4; ++k) {
        int px, py;
        tile[k] = corner_tile(P, s.f, k, px, py);
        pix[k] = (py % P.TH) * P.TW + (px % P.TW);
      }
    }
    const unsigned long long hi = ((unsigned long long)__float_as_uint(s.d) << kIdBits) | (unsigned long long)id;
    for (int k = 0; k < 4; ++k) {
      int t = tile[k];
      uint32_t cnt = 0;
      if (t >= 0) {
        bool first = true;
        for (int q = 0; q < k; ++q) first &= (tile[q] != t);
        if (first)
          for (int q = k; q < 4; ++q) cnt += (tile[q] == t);
        else
          t = -1;
      }
      const unsigned peers = __match_any_sync(full, t);
      // exclusive prefix of cnt among the peers (lane order), one atomic per group
      uint32_t pre = 0, sum = 0;
      for (unsigned m = peers; m; m &= m - 1) {
        const int src = __ffs(m) - 1;
        const uint32_t c = __shfl_sync(peers, cnt, src);
        if (src < lane) pre += c;
        sum += c;
      }
      const int leader = __ffs(peers) - 1;
      uint32_t slot = 0;
      if (t >= 0 && lane == leader) slot = atomicAdd(tile_cursor + t, sum);
      slot = __shfl_sync(peers, slot, leader);
      if (t >= 0) {
        unsigned long long* dst = keys + tile_offset[t] + slot + pre;
        int w = 0;
        for (int q = k; q < 4; ++q)
          if (tile[q] == t) dst[w++] = ((unsigned long long)pix[q] << 56) | hi;
      }
    }
  }
}

// ------------------------------------------------------- tile ordering ---
struct TileSmem {
  uint32_t pixcnt[256];
  uint32_t pixbeg[257];
  uint32_t pixcur[256];
  uint16_t wcnt[kWarps][256];
  uint32_t dbase[256];
  uint32_t ctot[256];
  unsigned long long red64[kWarps];
};

// Exclusive scan of 256 values (one per thread of a 256-thread CTA).
__device__ __forceinline__ uint32_t cta_excl_scan256(uint32_t v, uint32_t* warp_sums, uint32_t* total) {
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
    if (total) *total = run;
  }
  __syncthreads();
  return warp_sums[wid] + incl - v;
}

// Per-pixel segments of a key sequence sorted or bucketed by the pixel byte.
template <class KeyAt>
__device__ void pixel_segments(KeyAt key_at, int n, TileSmem& S) {
  S.pixcnt[threadIdx.x] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += kThreads) atomicAdd(&S.pixcnt[(int)(key_at(i) >> 56)], 1u);
  __syncthreads();
  const uint32_t ex = cta_excl_scan256(S.pixcnt[threadIdx.x], S.ctot, nullptr);
  S.pixbeg[threadIdx.x] = ex;
  S.pixcur[threadIdx.x] = ex;
  if (threadIdx.x == kThreads - 1) S.pixbeg[256] = ex + S.pixcnt[kThreads - 1];
  __syncthreads();
}

// Stable 8-bit LSD radix sort of one tile's bucket in global memory by one
// CTA: in[0..n) -> ka (keys), va (bucket positions); kb/vb are scratch.
__device__ void cta_sort_global(const unsigned long long* __restrict__ in, int n, unsigned long long* ka,
                                uint32_t* va, unsigned long long* kb, uint32_t* vb, TileSmem& S) {
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
    S.pixcnt[threadIdx.x] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kThreads) atomicAdd(&S.pixcnt[(int)((sk[i] >> sh) & 0xFF)], 1u);
    __syncthreads();
    S.dbase[threadIdx.x] = cta_excl_scan256(S.pixcnt[threadIdx.x], S.ctot, nullptr);
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

template <int GA>
__device__ __forceinline__ void gsync(unsigned mask) {
  if (GA > 1) __syncwarp(mask);
}

// Ascending sort of the index segment idx[0..m) by key K[idx[.]] with an
// all-ascending bitonic network (every comparator puts the minimum at the
// lower index), so indices >= m act as +infinity and are never touched.
template <int GA>
__device__ void group_sort(const unsigned long long* K, uint16_t* idx, int m, int lg, unsigned gmask) {
  if (m < 2) return;
  int P = 1;
  while (P < m) P <<= 1;
  for (int k = 2; k <= P; k <<= 1) {
    for (int q = lg; q < (P >> 1); q += GA) {
      const int half = k >> 1;
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
    gsync<GA>(gmask);
    for (int jj = k >> 2; jj >= 1; jj >>= 1) {
      for (int q = lg; q < (P >> 1); q += GA) {
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
      gsync<GA>(gmask);
    }
  }
}

template <int V>
__device__ __forceinline__ void load_vec(const float* __restrict__ p, float* c) {
  if (V == 4) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    c[0] = t.x; c[1] = t.y; c[2] = t.z; c[3] = t.w;
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) c[v] = __ldg(p + v);
  }
}

template <int GA>
__device__ __forceinline__ float group_sum(float x, unsigned gmask) {
#pragma unroll
  for (int o = GA / 2; o > 0; o >>= 1) x += __shfl_xor_sync(gmask, x, o);
  return x;
}

// ------------------------------------------------------------- forward ---
template <int V, int GA, class KeyAt>
__device__ void blend_fwd(const RP& P, KeyAt key_at, int m, int px, int py, const float* __restrict__ pos,
                          const float* __restrict__ opacity, const float* __restrict__ feat,
                          float* __restrict__ image, float* __restrict__ T_final, int32_t* __restrict__ n_contrib,
                          int lg) {
  const int ch = lg * V;
  const bool active = ch < P.F;
  float T = 1.0f;
  float C[V];
#pragma unroll
  for (int v = 0; v < V; ++v) C[v] = 0.f;
  int cnt = 0;
  for (int k = 0; k < m; ++k) {
    const unsigned long long key = key_at(k);
    const long long id = (long long)(key & kIdMask);
    Splat s;
    splat_point(P, pos, id, s);
    const float w = corner_weight(s.f, px - s.f.i0, py - s.f.j0);
    const float a = splat_alpha(P, point_alpha_h(P, opacity, feat, id, nullptr), w);
    float c[V];
    if (active) load_vec<V>(feat + (long long)P.F * id + ch, c);
    else
#pragma unroll
      for (int v = 0; v < V; ++v) c[v] = 0.f;
    if (P.head && lg == 0) c[0] = 1.0f;
    const float ta = __fmul_rn(T, a);
#pragma unroll
    for (int v = 0; v < V; ++v) C[v] = __fmaf_rn(ta, c[v], C[v]);
    T = __fmul_rn(T, __fsub_rn(1.0f, a));
    ++cnt;
    if (T < P.t_min) break;
  }
  const long long pix = (long long)py * P.cam.W + px;
  if (active) {
    float* o = image + pix * P.F + ch;
    if (V == 4) __stcs(reinterpret_cast<float4*>(o), make_float4(C[0], C[1], C[2], C[3]));
    else
#pragma unroll
      for (int v = 0; v < V; ++v) __stcs(o + v, C[v]);
  }
  if (lg == 0) {
    T_final[pix] = T;
    n_contrib[pix] = cnt;
  }
}

template <int V, int GA>
__global__ void __launch_bounds__(kThreads) k_raster_fwd(RP P, const float* __restrict__ pos,
                                                          const float* __restrict__ opacity,
                                                          const float* __restrict__ feat, RasterWs ws,
                                                          float* __restrict__ image, float* __restrict__ T_final,
                                                          int32_t* __restrict__ n_contrib) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ TileSmem S;
  const int t = blockIdx.x;
  const int tx = t % P.tiles_x, ty = t / P.tiles_x;
  const int n_t = (int)ws.tile_count[t];
  const uint32_t base = ws.tile_offset[t];
  const int lane = threadIdx.x & 31;
  const int lg = lane % GA;
  const int group = threadIdx.x / GA;
  constexpr int kGroups = kThreads / GA;
  const unsigned gmask = GA == 32 ? 0xffffffffu : (((1u << GA) - 1u) << (lane - lg));
  const int npix = P.TW * P.TH;
  if (n_t <= kCapFwd) {
    unsigned long long* K = reinterpret_cast<unsigned long long*>(dyn);
    uint16_t* idx = reinterpret_cast<uint16_t*>(K + kCapFwd);
    for (int i = threadIdx.x; i < n_t; i += kThreads) K[i] = ws.keys[base + i];
    __syncthreads();
    pixel_segments([&](int i) { return K[i]; }, n_t, S);
    for (int i = threadIdx.x; i < n_t; i += kThreads) {
      const uint32_t dst = atomicAdd(&S.pixcur[(int)(K[i] >> 56)], 1u);
      idx[dst] = (uint16_t)i;
    }
    __syncthreads();
    for (int p = group; p < npix; p += kGroups) {
      const int px = tx * P.TW + p % P.TW, py = ty * P.TH + p / P.TW;
      if (px >= P.cam.W || py >= P.cam.H) continue;
      const int b = (int)S.pixbeg[p], m = (int)(S.pixbeg[p + 1] - S.pixbeg[p]);
      group_sort<GA>(K, idx + b, m, lg, gmask);
      blend_fwd<V, GA>(P, [&](int k) { return K[idx[b + k]]; }, m, px, py, pos, opacity, feat, image, T_final,
                       n_contrib, lg);
    }
  } else {
    unsigned long long* ka = ws.ka + base;
    cta_sort_global(ws.keys + base, n_t, ka, ws.va + base, ws.kb + base, ws.vb + base, S);
    pixel_segments([&](int i) { return ka[i]; }, n_t, S);
    for (int p = group; p < npix; p += kGroups) {
      const int px = tx * P.TW + p % P.TW, py = ty * P.TH + p / P.TW;
      if (px >= P.cam.W || py >= P.cam.H) continue;
      const int b = (int)S.pixbeg[p], m = (int)(S.pixbeg[p + 1] - S.pixbeg[p]);
      blend_fwd<V, GA>(P, [&](int k) { return ka[b + k]; }, m, px, py, pos, opacity, feat, image, T_final,
                       n_contrib, lg);
    }
  }
}

// ------------------------------------------------------------ backward ---
// Phase 1: one pixel, back to front.  Writes (T_k alpha_k, dL/dalpha_k) for
// each of its blended fragments at the fragment's bucket position.
template <int V, int GA, class KeyAt, class PosAt, class ScalAt>
__device__ void blend_bwd_pixel(const RP& P, KeyAt key_at, PosAt bucket_pos, ScalAt scal, int n_blend, int px,
                                int py, const float* __restrict__ pos, const float* __restrict__ opacity,
                                const float* __restrict__ feat, const float* __restrict__ T_final,
                                const float* __restrict__ d_image, int lg, unsigned gmask) {
  const int ch = lg * V;
  const bool active = ch < P.F;
  const long long pix = (long long)py * P.cam.W + px;
  float g[V];
  if (active) load_vec<V>(d_image + pix * P.F + ch, g);
  else
#pragma unroll
    for (int v = 0; v < V; ++v) g[v] = 0.f;
  float T = T_final[pix];
  float S = 0.f;
  for (int k = n_blend - 1; k >= 0; --k) {
    const unsigned long long key = key_at(k);
    const long long id = (long long)(key & kIdMask);
    Splat s;
    splat_point(P, pos, id, s);
    const float w = corner_weight(s.f, px - s.f.i0, py - s.f.j0);
    const float a = splat_alpha(P, point_alpha_h(P, opacity, feat, id, nullptr), w);
    const float om = __fsub_rn(1.0f, a);
    const float Tk = __fdiv_rn(T, om);
    float c[V];
    if (active) load_vec<V>(feat + (long long)P.F * id + ch, c);
    else
#pragma unroll
      for (int v = 0; v < V; ++v) c[v] = 0.f;
    if (P.head && lg == 0) c[0] = 1.0f;
    float dot = 0.f;
#pragma unroll
    for (int v = 0; v < V; ++v) dot = __fmaf_rn(c[v], g[v], dot);
    dot = group_sum<GA>(dot, gmask);
    const float aw = __fmul_rn(Tk, a);
    const float da = __fsub_rn(__fmul_rn(Tk, dot), __fdiv_rn(S, om));
    S = __fmaf_rn(aw, dot, S);
    T = Tk;
    if (lg == 0) scal(bucket_pos(k)) = make_float2(aw, da);
  }
}

// Phase 2: one point's fragments in this tile (consecutive bucket entries
// [i, i + c)).  d_feat row = sum_k (T_k alpha_k) g_pixel(k); d alpha_h =
// sum_k w_k [unclamped] dL/dalpha_k.
template <int V, int GA, class KeyAt, class ScalAt>
__device__ void point_grad(const RP& P, KeyAt key_at, ScalAt scal, int i, int c, int tx, int ty,
                           const float* __restrict__ pos, const float* __restrict__ opacity,
                           const float* __restrict__ feat, const float* __restrict__ d_image,
                           float* __restrict__ d_opacity, float* __restrict__ d_feat, int lg) {
  const int ch = lg * V;
  const bool active = ch < P.F;
  const long long id = (long long)(key_at(i) & kIdMask);
  Splat s;
  splat_point(P, pos, id, s);
  int on_image = 0;
  for (int k = 0; k < 4; ++k) {
    int px, py;
    on_image += corner_tile(P, s.f, k, px, py) >= 0;
  }
  const bool straddle = c < on_image;
  float e_h0 = 0.f;
  const float ah = point_alpha_h(P, opacity, feat, id, &e_h0);
  float dc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) dc[v] = 0.f;
  float dah = 0.f;
  for (int j = 0; j < c; ++j) {
    const unsigned long long key = key_at(i + j);
    const int p = (int)(key >> 56);
    const int px = tx * P.TW + p % P.TW, py = ty * P.TH + p / P.TW;
    const float2 sc = scal(i + j);
    const float w = corner_weight(s.f, px - s.f.i0, py - s.f.j0);
    if (__fmul_rn(ah, w) <= P.alpha_max) dah = __fmaf_rn(w, sc.y, dah);
    if (active) {
      float g[V];
      load_vec<V>(d_image + ((long long)py * P.cam.W + px) * P.F + ch, g);
#pragma unroll
      for (int v = 0; v < V; ++v) dc[v] = __fmaf_rn(sc.x, g[v], dc[v]);
    }
  }
  if (P.head && lg == 0) dc[0] = dah * e_h0 * (1.0f - ah);
  if (active) {
    float* o = d_feat + id * P.F + ch;
    if (straddle) {
#pragma unroll
      for (int v = 0; v < V; ++v) atomicAdd(o + v, dc[v]);
    } else if (V == 4) {
      *reinterpret_cast<float4*>(o) = make_float4(dc[0], dc[1], dc[2], dc[3]);
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) o[v] = dc[v];
    }
  }
  if (!P.head && lg == 0) {
    if (straddle) atomicAdd(d_opacity + id, dah);
    else d_opacity[id] = dah;
  }
}

template <int V, int GA>
__global__ void __launch_bounds__(kThreads) k_raster_bwd(RP P, const float* __restrict__ pos,
                                                          const float* __restrict__ opacity,
                                                          const float* __restrict__ feat,
                                                          const float* __restrict__ T_final,
                                                          const int32_t* __restrict__ n_contrib,
                                                          const float* __restrict__ d_image, RasterWs ws,
                                                          float* __restrict__ d_opacity, float* __restrict__ d_feat) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ TileSmem S;
  const int t = blockIdx.x;
  const int tx = t % P.tiles_x, ty = t / P.tiles_x;
  const int n_t = (int)ws.tile_count[t];
  if (n_t == 0) return;
  const uint32_t base = ws.tile_offset[t];
  const int lane = threadIdx.x & 31;
  const int lg = lane % GA;
  const int group = threadIdx.x / GA;
  constexpr int kGroups = kThreads / GA;
  const unsigned gmask = GA == 32 ? 0xffffffffu : (((1u << GA) - 1u) << (lane - lg));
  const int npix = P.TW * P.TH;
  if (n_t <= kCapBwd) {
    unsigned long long* K = reinterpret_cast<unsigned long long*>(dyn);
    float2* sc = reinterpret_cast<float2*>(K + kCapBwd);
    uint16_t* idx = reinterpret_cast<uint16_t*>(sc + kCapBwd);
    for (int i = threadIdx.x; i < n_t; i += kThreads) {
      K[i] = ws.keys[base + i];
      sc[i] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    pixel_segments([&](int i) { return K[i]; }, n_t, S);
    for (int i = threadIdx.x; i < n_t; i += kThreads) {
      const uint32_t dst = atomicAdd(&S.pixcur[(int)(K[i] >> 56)], 1u);
      idx[dst] = (uint16_t)i;
    }
    __syncthreads();
    for (int p = group; p < npix; p += kGroups) {
      const int px = tx * P.TW + p % P.TW, py = ty * P.TH + p / P.TW;
      if (px >= P.cam.W || py >= P.cam.H) continue;
      const int b = (int)S.pixbeg[p], m = (int)(S.pixbeg[p + 1] - S.pixbeg[p]);
      group_sort<GA>(K, idx + b, m, lg, gmask);
      const int nb = min(m, (int)n_contrib[(long long)py * P.cam.W + px]);
      blend_bwd_pixel<V, GA>(
          P, [&](int k) { return K[idx[b + k]]; }, [&](int k) { return (int)idx[b + k]; },
          [&](int q) -> float2& { return sc[q]; }, nb, px, py, pos, opacity, feat, T_final, d_image, lg, gmask);
    }
    __syncthreads();
    for (int i = group; i < n_t; i += kGroups) {
      const long long id = (long long)(K[i] & kIdMask);
      if (i > 0 && (long long)(K[i - 1] & kIdMask) == id) continue;
      int c = 1;
      while (i + c < n_t && c < 4 && (long long)(K[i + c] & kIdMask) == id) ++c;
      point_grad<V, GA>(P, [&](int q) { return K[q]; }, [&](int q) { return sc[q]; }, i, c, tx, ty, pos, opacity,
                        feat, d_image, d_opacity, d_feat, lg);
    }
  } else {
    unsigned long long* ka = ws.ka + base;
    uint32_t* va = ws.va + base;
    float2* fs = ws.fscal + base;
    const unsigned long long* kin = ws.keys + base;
    for (int i = threadIdx.x; i < n_t; i += kThreads) fs[i] = make_float2(0.f, 0.f);
    cta_sort_global(kin, n_t, ka, va, ws.kb + base, ws.vb + base, S);
    pixel_segments([&](int i) { return ka[i]; }, n_t, S);
    for (int p = group; p < npix; p += kGroups) {
      const int px = tx * P.TW + p % P.TW, py = ty * P.TH + p / P.TW;
      if (px >= P.cam.W || py >= P.cam.H) continue;
      const int b = (int)S.pixbeg[p], m = (int)(S.pixbeg[p + 1] - S.pixbeg[p]);
      const int nb = min(m, (int)n_contrib[(long long)py * P.cam.W + px]);
      blend_bwd_pixel<V, GA>(
          P, [&](int k) { return ka[b + k]; }, [&](int k) { return (int)va[b + k]; },
          [&](int q) -> float2& { return fs[q]; }, nb, px, py, pos, opacity, feat, T_final, d_image, lg, gmask);
    }
    __syncthreads();
    for (int i = group; i < n_t; i += kGroups) {
      const long long id = (long long)(kin[i] & kIdMask);
      if (i > 0 && (long long)(kin[i - 1] & kIdMask) == id) continue;
      int c = 1;
      while (i + c < n_t && c < 4 && (long long)(kin[i + c] & kIdMask) == id) ++c;
      point_grad<V, GA>(P, [&](int q) { return kin[q]; }, [&](int q) { return fs[q]; }, i, c, tx, ty, pos,
                        opacity, feat, d_image, d_opacity, d_feat, lg);
    }
  }
}

// Zero the gradient rows that the tile kernels will not overwrite: culled
// points (no fragment) and points whose fragments span several tiles (those
// receive per-tile partial sums through atomics).
__global__ void __launch_bounds__(256) k_bwd_prep(RP P, const float* __restrict__ pos, float* __restrict__ d_opacity,
                                                  float* __restrict__ d_feat) {
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < P.n;
       id += (long long)gridDim.x * blockDim.x) {
    Splat s;
    int first = -1;
    bool zero = true;
    if (splat_point(P, pos, id, s)) {
      bool multi = false;
      for (int k = 0; k < 4; ++k) {
        int px, py;
        const int t = corner_tile(P, s.f, k, px, py);
        if (t < 0) continue;
        if (first < 0) first = t;
        else if (t != first) multi = true;
      }
      zero = first < 0 || multi;
    }
    if (!zero) continue;
    float* row = d_feat + id * P.F;
    for (int c = 0; c < P.F; ++c) row[c] = 0.f;
    if (d_opacity) d_opacity[id] = 0.f;
  }
}

// ---------------------------------------------------------------- host ---
inpc_status make_rp(const inpc_camera* cam, const inpc_raster_opts* o, int64_t n, RP& P) {
  if (!cam || !o) return fail(INPC_ERR_INVALID_ARG, "camera or options is null");
  if (cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768)
    return fail(INPC_ERR_INVALID_ARG, "image size %dx%d out of range", cam->width, cam->height);
  if (!(cam->near_plane > 0.0f) || !(cam->far_plane > cam->near_plane))
    return fail(INPC_ERR_INVALID_ARG, "need 0 < near < far");
  if (n < 0 || n > (int64_t(1) << kIdBits)) return fail(INPC_ERR_CAPACITY, "n must be in [0, 2^25]");
  if (o->opacity_mode != INPC_OPACITY_GIVEN && o->opacity_mode != INPC_OPACITY_FROM_CH0)
    return fail(INPC_ERR_INVALID_ARG, "bad opacity_mode");
  if (o->feat_dtype != INPC_F32 || o->image_dtype != INPC_F32)
    return fail(INPC_ERR_UNSUPPORTED, "only INPC_F32 features and images are implemented");
  if (o->n_channels < 1 || o->n_channels > 128) return fail(INPC_ERR_UNSUPPORTED, "n_channels must be in [1, 128]");
  if (o->n_channels % 4 != 0 && o->n_channels > 32)
    return fail(INPC_ERR_UNSUPPORTED, "n_channels > 32 must be a multiple of 4");
  if (!(o->t_min >= 0.0f && o->t_min < 1.0f)) return fail(INPC_ERR_INVALID_ARG, "t_min must be in [0, 1)");
  if (!(o->alpha_max > 0.0f && o->alpha_max < 1.0f)) return fail(INPC_ERR_INVALID_ARG, "alpha_max must be in (0, 1)");
  P.cam = to_cam(*cam);
  P.TW = o->tile_w > 0 ? o->tile_w : 16;
  P.TH = o->tile_h > 0 ? o->tile_h : 16;
  if (P.TW * P.TH > 256) return fail(INPC_ERR_INVALID_ARG, "tile_w * tile_h must be <= 256");
  P.tiles_x = (int)ceil_div(cam->width, P.TW);
  P.tiles_y = (int)ceil_div(cam->height, P.TH);
  P.n_tiles = P.tiles_x * P.tiles_y;
  P.F = o->n_channels;
  P.head = o->opacity_mode == INPC_OPACITY_FROM_CH0;
  P.t_min = o->t_min;
  P.alpha_max = o->alpha_max;
  P.n = n;
  return INPC_OK;
}

int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

template <int V, int GA>
inpc_status launch_fwd(const RP& P, const float* pos, const float* opacity, const float* feat, const RasterWs& ws,
                       float* image, float* T_final, int32_t* n_contrib, cudaStream_t s) {
  const size_t dyn = (size_t)kCapFwd * (8 + 2);
  static std::once_flag once;
  std::call_once(once, [&] {
    cudaFuncSetAttribute(k_raster_fwd<V, GA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  });
  k_raster_fwd<V, GA><<<P.n_tiles, kThreads, dyn, s>>>(P, pos, opacity, feat, ws, image, T_final, n_contrib);
  return check_launch("k_raster_fwd");
}

template <int V, int GA>
inpc_status launch_bwd(const RP& P, const float* pos, const float* opacity, const float* feat, const float* T_final,
                       const int32_t* n_contrib, const float* d_image, const RasterWs& ws, float* d_opacity,
                       float* d_feat, cudaStream_t s) {
  const size_t dyn = (size_t)kCapBwd * (8 + 8 + 2);
  static std::once_flag once;
  std::call_once(once, [&] {
    cudaFuncSetAttribute(k_raster_bwd<V, GA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  });
  k_raster_bwd<V, GA><<<P.n_tiles, kThreads, dyn, s>>>(P, pos, opacity, feat, T_final, n_contrib, d_image, ws,
                                                        d_opacity, d_feat);
  return check_launch("k_raster_bwd");
}

// (V, GA): V channels per lane, GA lanes per pixel.
template <class Fn>
inpc_status dispatch(int F, Fn&& fn) {
  if (F % 4 == 0) {
    switch (next_pow2(F / 4)) {
      case 1: return fn(std::integral_constant<int, 4>(), std::integral_constant<int, 1>());
      case 2: return fn(std::integral_constant<int, 4>(), std::integral_constant<int, 2>());
      case 4: return fn(std::integral_constant<int, 4>(), std::integral_constant<int, 4>());
      case 8: return fn(std::integral_constant<int, 4>(), std::integral_constant<int, 8>());
      case 16: return fn(std::integral_constant<int, 4>(), std::integral_constant<int, 16>());
      case 32: return fn(std::integral_constant<int, 4>(), std::integral_constant<int, 32>());
    }
  } else {
    switch (next_pow2(F)) {
      case 1: return fn(std::integral_constant<int, 1>(), std::integral_constant<int, 1>());
      case 2: return fn(std::integral_constant<int, 1>(), std::integral_constant<int, 2>());
      case 4: return fn(std::integral_constant<int, 1>(), std::integral_constant<int, 4>());
      case 8: return fn(std::integral_constant<int, 1>(), std::integral_constant<int, 8>());
      case 16: return fn(std::integral_constant<int, 1>(), std::integral_constant<int, 16>());
      case 32: return fn(std::integral_constant<int, 1>(), std::integral_constant<int, 32>());
    }
  }
  return fail(INPC_ERR_UNSUPPORTED, "no kernel for n_channels = %d", F);
}

unsigned point_grid(long long n) {
  const long long cap = (long long)device_sm_count() * 16;
  return (unsigned)std::max<long long>(1, std::min<long long>(ceil_div(n, 256), cap));
}

}  // namespace
}  // namespace inpc

using namespace inpc;

extern "C" inpc_status inpc_rasterize_workspace_size(const inpc_camera* cam, const inpc_raster_opts* opts, int64_t n,
                                                     size_t* bytes) {
  if (!bytes) return fail(INPC_ERR_INVALID_ARG, "bytes is null");
  RP P;
  INPC_TRY(make_rp(cam, opts, n, P));
  *bytes = carve(nullptr, P.n_tiles, n).bytes;
  return INPC_OK;
}

extern "C" inpc_status inpc_rasterize_fwd(const inpc_camera* cam, const inpc_raster_opts* opts, const float* pos,
                                          const float* opacity, const void* feat, int64_t n, void* image,
                                          float* T_final, int32_t* n_contrib, void* workspace,
                                          size_t workspace_bytes, inpc_stream_t stream) {
  RP P;
  INPC_TRY(make_rp(cam, opts, n, P));
  const RasterWs need = carve(nullptr, P.n_tiles, n);
  if (!workspace || workspace_bytes < need.bytes || !aligned(workspace, 256))
    return fail(INPC_ERR_INVALID_ARG, "workspace null, unaligned or smaller than %zu bytes", need.bytes);
  if (!image || !T_final || !n_contrib) return fail(INPC_ERR_INVALID_ARG, "null output");
  if (n > 0 && (!pos || !feat)) return fail(INPC_ERR_INVALID_ARG, "null pos or feat");
  if (n > 0 && !P.head && !opacity) return fail(INPC_ERR_INVALID_ARG, "opacity required in INPC_OPACITY_GIVEN mode");
  const size_t va = P.F % 4 == 0 ? 16 : 4;
  if (!aligned(feat, va) || !aligned(image, va) || !aligned(pos, 4))
    return fail(INPC_ERR_INVALID_ARG, "feat/image must be %zu-byte aligned", va);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RasterWs ws = carve(workspace, P.n_tiles, n);
  INPC_CUDA(cudaMemsetAsync(workspace, 0, kHeaderBytes, s), "clear header");
  INPC_CUDA(cudaMemsetAsync(ws.tile_count, 0, sizeof(uint32_t) * P.n_tiles, s), "clear tile counts");
  const float* f32 = static_cast<const float*>(feat);
  if (n > 0) {
    k_bin_count<<<point_grid(n), 256, 0, s>>>(P, pos, ws.tile_count);
    INPC_TRY(check_launch("k_bin_count"));
  }
  k_scan_tiles<<<1, 1024, 0, s>>>(ws.tile_count, P.n_tiles, ws.tile_offset, ws.tile_cursor);
  INPC_TRY(check_launch("k_scan_tiles"));
  if (n > 0) {
    k_bin_scatter<<<point_grid(n), 256, 0, s>>>(P, pos, ws.tile_offset, ws.tile_cursor, ws.keys);
    INPC_TRY(check_launch("k_bin_scatter"));
  }
  return dispatch(P.F, [&](auto Vc, auto Gc) {
    return launch_fwd<decltype(Vc)::value, decltype(Gc)::value>(P, pos, opacity, f32, ws, static_cast<float*>(image),
                                                                 T_final, n_contrib, s);
  });
}

extern "C" inpc_status inpc_rasterize_bwd(const inpc_camera* cam, const inpc_raster_opts* opts, const float* pos,
                                          const float* opacity, const void* feat, int64_t n, const float* T_final,
                                          const int32_t* n_contrib, const float* d_image, float* d_opacity,
                                          float* d_feat, void* workspace, size_t workspace_bytes,
                                          inpc_stream_t stream) {
  RP P;
  INPC_TRY(make_rp(cam, opts, n, P));
  const RasterWs need = carve(nullptr, P.n_tiles, n);
  if (!workspace || workspace_bytes < need.bytes || !aligned(workspace, 256))
    return fail(INPC_ERR_INVALID_ARG, "workspace null, unaligned or smaller than %zu bytes", need.bytes);
  if (n == 0) return INPC_OK;
  if (!pos || !feat || !T_final || !n_contrib || !d_image || !d_feat)
    return fail(INPC_ERR_INVALID_ARG, "null pointer");
  if (!P.head && (!opacity || !d_opacity)) return fail(INPC_ERR_INVALID_ARG, "opacity and d_opacity required");
  const size_t va = P.F % 4 == 0 ? 16 : 4;
  if (!aligned(feat, va) || !aligned(d_image, va) || !aligned(d_feat, va))
    return fail(INPC_ERR_INVALID_ARG, "feat/d_image/d_feat must be %zu-byte aligned", va);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  RasterWs ws = carve(workspace, P.n_tiles, n);
  float* dop = P.head ? nullptr : d_opacity;
  k_bwd_prep<<<point_grid(n), 256, 0, s>>>(P, pos, dop, d_feat);
  INPC_TRY(check_launch("k_bwd_prep"));
  const float* f32 = static_cast<const float*>(feat);
  return dispatch(P.F, [&](auto Vc, auto Gc) {
    return launch_bwd<decltype(Vc)::value, decltype(Gc)::value>(P, pos, opacity, f32, T_final, n_contrib, d_image, ws,
                                                                 dop, d_feat, s);
  });
}
