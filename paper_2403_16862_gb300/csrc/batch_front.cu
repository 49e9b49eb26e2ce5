// batch_front.cu -- the front end of a batch of views in two launches: the
// octree sampling (Sec. 3.2) of every view in ONE persistent kernel driven
// by a work queue with bounded waits, then the grid query (Sec. 3.3) of
// every view in one more launch.
//
// The batch shares one octree and one table (the views differ in view id,
// sample count and outputs), so the quantised CDF and the guide table are
// built once for the batch, not once per view.  Work items of the
// persistent kernel, in the order of their tickets:
//   W  tiles of leaves: max weight (+ weight validation)
//   C  tiles of 2048 leaves: quantised weights, exact prefix sum (single
//      pass: each tile publishes its total, then looks back for the sum of
//      its predecessors)
//   G  tiles of the guide table
//   D  per view, tiles of 4096 draws: leaf of every draw -> per-leaf counts
//   S  per view, tiles of 2048 leaves: exclusive prefix sum of the counts
//      (single pass, as C) -> first output slot of every leaf
//   P  per view, tiles of slots: leaf of the slot, position in the leaf
// CTAs take tickets from one atomic counter and run the item to completion;
// an item waits only for items with smaller tickets (a stage's counter, or a
// predecessor tile's published prefix), which CTAs that run have already
// taken, so the queue always progresses.  Every wait gives up after
// max_wait_ns of the GPU's global timer: it then sets INPC_DEV_TIMEOUT in the
// status word and the abort flag, and every CTA returns at its next wait or
// ticket.  The query launch then covers the views' points concatenated,
// each warp taking 16 points of one view through a group of levels whose
// rows stay in L2; it has no waits (its inputs are complete when it starts)
// and keeps the query's full occupancy, which the sampling stages'
// registers would not allow in one kernel.  The per-item arithmetic
// is that of the per-view kernels (sample_impl.cuh, query_half), so the
// outputs are bit-identical to inpc_sample_octree + inpc_query_hashgrid of
// each view.
#include <algorithm>
#include <atomic>

#include "hashgrid_impl.cuh"
#include "sample_impl.cuh"
#include "scan.cuh"

namespace inpc {

// host-side fault injection (faults.cu): extra count added to one
// dependency target of the next persistent launch
uint32_t fault_take_queue_short();

namespace {

constexpr int kFrontMaxViews = 64;
constexpr int kFrontThreads = 256;
constexpr int kWTile = 8192;          // leaves per max item
constexpr int kPlaceTile = 16384;     // slots per place item
constexpr int kQueryPad = 16;        // query launch: each view's points padded to a multiple of this

enum : int { kStW = 0, kStC, kStG, kStD, kStS, kStP, kStEnd };

struct FrontView {
  uint32_t view_id;
  int64_t n;
  int32_t* leaf;
  float* pos;
  void* h;
};

// The launch's plan (kernel parameter): views, tile counts and the first
// ticket of every stage (and view).
struct FrontPlan {
  int n_views;
  int64_t L;
  int Gl;            // guide table: 2^Gl + 1 entries
  int stride_log2;   // coarse search table of the slot starts
  uint32_t Tw, Tc, Tg;
  uint32_t first[kStEnd + 1];          // first ticket of each stage; first[kStEnd] = total
  uint32_t preD[kFrontMaxViews + 1];   // D tiles of views < v
  uint32_t preP[kFrontMaxViews + 1];
  uint32_t preQ[kFrontMaxViews + 1];   // points of views < v, each view's count padded to a multiple of 16
  uint32_t short_by;                   // fault injection: view 0's count scan waits for this many extra draw tiles
  long long max_wait_ns;
  uint32_t k0, k1;                     // Philox key (seed lo, seed hi)
  FrontView v[kFrontMaxViews];
};

// Workspace: 256-byte header (status word, ticket, abort flag, max weight),
// then the stage counters, the look-back words and the per-view arrays.
struct FrontWs {
  uint32_t* status;
  uint32_t* ticket;
  uint32_t* abort;
  unsigned long long* wmax;
  uint32_t* done;                  // [3 + 3 V]: W, C, G, then D, S, P of each view
  unsigned long long* cdf_state;   // [Tc] look-back words of the CDF tiles
  unsigned long long* cnt_state;   // [V, Tc] look-back words of the count tiles
  double* cdf;                     // [L]
  uint32_t* guide;                 // [2^Gl + 1]
  uint32_t* counts;                // [V, L]
  uint32_t* starts;                // [V, L]
  size_t clear_bytes;              // bytes from the start that every call zeroes
  size_t bytes;
};

FrontWs carve_front(void* base, int64_t L, int n_views) {
  Carver c(base);
  FrontWs w;
  char* b = static_cast<char*>(base);
  w.status = reinterpret_cast<uint32_t*>(b);
  w.ticket = reinterpret_cast<uint32_t*>(b ? b + 4 : nullptr);
  w.abort = reinterpret_cast<uint32_t*>(b ? b + 8 : nullptr);
  w.wmax = reinterpret_cast<unsigned long long*>(b ? b + 16 : nullptr);
  const int64_t Tc = ceil_div(L, kScanBlock);
  w.done = c.take<uint32_t>(3 + 3 * (size_t)n_views);
  w.cdf_state = c.take<unsigned long long>(Tc);
  w.cnt_state = c.take<unsigned long long>((size_t)Tc * n_views);
  w.counts = c.take<uint32_t>((size_t)L * n_views);
  w.clear_bytes = c.bytes();
  w.cdf = c.take<double>(L);
  w.guide = c.take<uint32_t>((int64_t(1) << guide_log2(L)) + 1);
  w.starts = c.take<uint32_t>((size_t)L * n_views);
  w.bytes = c.bytes();
  return w;
}

// Look-back words: flag in the top two bits (1: the tile's own total, 2: the
// inclusive prefix up to and including the tile), the value below (< 2^62).
constexpr unsigned long long kAggregate = 1ull << 62, kInclusive = 2ull << 62, kValMask = (1ull << 62) - 1;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// One thread's bounded wait.  Returns false (after raising the timeout and
// the abort flag, or on seeing the abort flag) when the wait gave up.
struct Waiter {
  uint64_t t0;
  unsigned ns = 32;
  long long limit;
  uint32_t* status;
  uint32_t* abort;
  __device__ Waiter(const FrontPlan& pl, const FrontWs& ws)
      : t0(global_ns()), limit(pl.max_wait_ns), status(ws.status), abort(ws.abort) {}
  // call while the condition is false; false = give up
  __device__ bool again() {
    if (ld_acquire(abort)) return false;
    if ((long long)(global_ns() - t0) > limit) {
      atomicOr(status, INPC_DEV_TIMEOUT);
      atomicExch(abort, 1u);
      return false;
    }
    __nanosleep(ns);
    if (ns < 1024) ns *= 2;
    return true;
  }
};

// Thread 0 waits for *ctr >= target; the block learns the outcome.
__device__ bool block_wait(const uint32_t* ctr, uint32_t target, const FrontPlan& pl, const FrontWs& ws, int* s_ok) {
  if (threadIdx.x == 0) {
    Waiter w(pl, ws);
    bool ok = true;
    while (ld_acquire(ctr) < target)
      if (!w.again()) {
        ok = false;
        break;
      }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Every thread's writes of the item are made visible, then thread 0 counts
// the item as done.
__device__ void block_signal(uint32_t* ctr) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(ctr, 1u);
}

// Single-pass exclusive prefix of tile t (thread 0): publish the tile's own
// total, add the predecessors' values walking back until an inclusive
// prefix, publish this tile's inclusive prefix.  Returns false if a wait
// gave up.
__device__ bool look_back(unsigned long long* state, uint32_t t, unsigned long long total, const FrontPlan& pl,
                          const FrontWs& ws, unsigned long long* exclusive) {
  if (t == 0) {
    atomicExch(state, kInclusive | total);
    *exclusive = 0;
    return true;
  }
  atomicExch(state + t, kAggregate | total);
  unsigned long long ex = 0;
  for (int64_t j = (int64_t)t - 1; j >= 0; --j) {
    Waiter w(pl, ws);
    unsigned long long s;
    while (((s = ld_acquire64(state + j)) >> 62) == 0)
      if (!w.again()) return false;
    ex += s & kValMask;
    if ((s >> 62) == 2) break;
  }
  atomicExch(state + t, kInclusive | (ex + total));
  *exclusive = ex;
  return true;
}

struct __align__(16) FrontSmem {
  union {
    uint32_t coarse[kCoarse];
    uint32_t vals[kSmemLeaves];
    unsigned long long warp_sums[32];
  };
  unsigned long long total;
  unsigned long long exclusive;
  uint32_t ticket;
  int ok;
};

// Which stage, view, level pair and tile a ticket names.
__device__ __forceinline__ int upper_idx(const uint32_t* pre, int n, uint32_t x) {
  int lo = 0, hi = n;  // largest v with pre[v] <= x
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kFrontThreads) k_front(const __grid_constant__ FrontPlan pl, inpc_octree tree,
                                                          FrontWs ws) {
  __shared__ FrontSmem sm;
  const int tid = threadIdx.x;
  const int64_t L = pl.L;
  for (;;) {
    if (tid == 0) sm.ticket = ld_acquire(ws.abort) ? pl.first[kStEnd] : atomicAdd(ws.ticket, 1u);
    __syncthreads();
    const uint32_t t = sm.ticket;
    __syncthreads();
    if (t >= pl.first[kStEnd]) return;
    int st = kStW;
    while (t >= pl.first[st + 1]) ++st;
    const uint32_t r = t - pl.first[st];

    if (st == kStW) {
      // ---- max weight of a tile of leaves (and validation)
      double m = 0.0;
      bool bad = false;
      const int64_t i0 = (int64_t)r * kWTile;
      for (int64_t i = i0 + tid; i < min(L, i0 + kWTile); i += kFrontThreads) {
        const double x = tree.weights[i];
        if (!(x >= 0.0) || isinf(x)) bad = true;
        else m = fmax(m, x);
      }
      if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) raise_status(ws.status, INPC_DEV_BAD_WEIGHT);
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if ((tid & 31) == 0 && m > 0.0) atomicMax(ws.wmax, (unsigned long long)__double_as_longlong(m));
      block_signal(ws.done + 0);
    } else if (st == kStC) {
      // ---- quantised weights, exact prefix sum (integers)
      if (!block_wait(ws.done + 0, pl.Tw, pl, ws, &sm.ok)) return;
      const double wm = __longlong_as_double((long long)__ldcg(ws.wmax));
      const int64_t base = (int64_t)r * kScanBlock + (int64_t)tid * kScanItems;
      unsigned long long q[kScanItems], run = 0;
#pragma unroll
      for (int k = 0; k < kScanItems; ++k) {
        q[k] = base + k < L ? (unsigned long long)quantised_weight(tree.weights[base + k], wm) : 0ull;
        run += q[k];
      }
      const unsigned long long pre = scan::block_exclusive_scan<unsigned long long>(run, sm.warp_sums, &sm.total);
      if (tid == 0) sm.ok = look_back(ws.cdf_state, r, sm.total, pl, ws, &sm.exclusive);
      __syncthreads();
      if (!sm.ok) return;
      unsigned long long acc = sm.exclusive + pre;
#pragma unroll
      for (int k = 0; k < kScanItems; ++k) {
        acc += q[k];
        if (base + k < L) ws.cdf[base + k] = (double)acc;
      }
      block_signal(ws.done + 1);
    } else if (st == kStG) {
      // ---- guide table
      if (!block_wait(ws.done + 1, pl.Tc, pl, ws, &sm.ok)) return;
      const double Qd = __ldcg(ws.cdf + L - 1);
      if (r == 0 && tid == 0 && !(Qd > 0.0)) raise_status(ws.status, INPC_DEV_NO_WEIGHT);
      const int64_t G1 = (int64_t(1) << pl.Gl) + 1;
      for (int64_t j = (int64_t)r * kScanBlock + tid; j < min(G1, (int64_t)(r + 1) * kScanBlock); j += kFrontThreads)
        ws.guide[j] = guide_entry(LdL2(), ws.cdf, L, pl.Gl, (uint64_t)Qd, j);
      block_signal(ws.done + 2);
    } else if (st == kStD) {
      // ---- draws of view v -> per-leaf counts
      const int v = upper_idx(pl.preD, pl.n_views + 1, r);
      const uint32_t tile = r - pl.preD[v];
      if (!block_wait(ws.done + 2, pl.Tg, pl, ws, &sm.ok)) return;
      const FrontView& V = pl.v[v];
      uint32_t* counts = ws.counts + (size_t)v * L;
      const bool smem = L <= kSmemLeaves;
      if (smem) {
        for (int j = tid; j < L; j += kFrontThreads) sm.vals[j] = 0;
        __syncthreads();
      }
      const uint64_t Qi = (uint64_t)__ldcg(ws.cdf + L - 1);
      const int64_t base = (int64_t)tile * kDrawPerCta;
      const int lane = tid & 31;
      for (int k = 0; k < kDrawPerThread; ++k) {
        const int64_t s = base + (int64_t)k * kFrontThreads + tid;
        int leaf = -1;
        if (s < V.n) leaf = (int)draw_leaf(LdL2(), ws.cdf, L, ws.guide, pl.Gl, Qi, s, V.view_id, pl.k0, pl.k1);
        const unsigned peers = __match_any_sync(0xffffffffu, leaf);
        if (leaf >= 0 && lane == __ffs(peers) - 1) {
          if (smem) atomicAdd(&sm.vals[leaf], (uint32_t)__popc(peers));
          else atomicAdd(&counts[leaf], (uint32_t)__popc(peers));
        }
      }
      if (smem) {
        __syncthreads();
        for (int j = tid; j < L; j += kFrontThreads)
          if (sm.vals[j]) atomicAdd(&counts[j], sm.vals[j]);
      }
      block_signal(ws.done + 3 + 3 * v);
    } else if (st == kStS) {
      // ---- exclusive prefix of view v's counts -> first slot of each leaf
      const int v = (int)(r / pl.Tc);
      const uint32_t tile = r - (uint32_t)v * pl.Tc;
      const uint32_t need = pl.preD[v + 1] - pl.preD[v] + (v == 0 ? pl.short_by : 0u);
      if (!block_wait(ws.done + 3 + 3 * v, need, pl, ws, &sm.ok)) return;
      const uint32_t* counts = ws.counts + (size_t)v * L;
      uint32_t* starts = ws.starts + (size_t)v * L;
      const int64_t base = (int64_t)tile * kScanBlock + (int64_t)tid * kScanItems;
      unsigned long long c[kScanItems], run = 0;
#pragma unroll
      for (int k = 0; k < kScanItems; ++k) {
        c[k] = base + k < L ? __ldcg(counts + base + k) : 0u;
        run += c[k];
      }
      const unsigned long long pre = scan::block_exclusive_scan<unsigned long long>(run, sm.warp_sums, &sm.total);
      if (tid == 0) sm.ok = look_back(ws.cnt_state + (size_t)v * pl.Tc, tile, sm.total, pl, ws, &sm.exclusive);
      __syncthreads();
      if (!sm.ok) return;
      unsigned long long acc = sm.exclusive + pre;
#pragma unroll
      for (int k = 0; k < kScanItems; ++k) {
        if (base + k < L) starts[base + k] = (uint32_t)acc;
        acc += c[k];
      }
      block_signal(ws.done + 4 + 3 * v);
    } else {
      // ---- slots of view v: leaf and position
      const int v = upper_idx(pl.preP, pl.n_views + 1, r);
      const uint32_t tile = r - pl.preP[v];
      if (!block_wait(ws.done + 4 + 3 * v, pl.Tc, pl, ws, &sm.ok)) return;
      const FrontView& V = pl.v[v];
      const uint32_t* starts = ws.starts + (size_t)v * L;
      int n_coarse;
      load_coarse(LdL2(), starts, L, pl.stride_log2, sm.coarse, n_coarse);
      const int64_t k1 = min(V.n, (int64_t)(tile + 1) * kPlaceTile);
      for (int64_t k = (int64_t)tile * kPlaceTile + tid; k < k1; k += kFrontThreads) {
        int64_t leaf = upper_bound2<uint32_t>(LdL2(), starts, L, sm.coarse, n_coarse, pl.stride_log2, (uint32_t)k) - 1;
        if (leaf < 0) leaf = 0;
        place_slot(k, leaf, V.view_id, pl.k0, pl.k1, tree.centers, tree.levels, tree.root_size, V.leaf, V.pos);
      }
      block_signal(ws.done + 5 + 3 * v);
    }
  }
}

// The query of every view in one launch, laid out as k_hash_fwd: a warp
// takes 16 consecutive points, two lanes per point, through the levels of
// one level group (grid y); within a group the views go one after another.
// The views' points are concatenated, each view's count padded to a
// multiple of 16, so a warp's points belong to one view; padding lanes join
// the pair exchanges but store nothing.  The grid strides over the groups
// of 16 of all views, view after view, so every CTA keeps its share of
// groups while the view's constants stay in registers for the whole view.
template <class TT, class OT>
__global__ void __launch_bounds__(kFrontThreads) k_front_query(const __grid_constant__ FrontPlan pl, GridParams G,
                                                               LevelGroups LG, const TT* __restrict__ table) {
  const int lb = LG.begin[blockIdx.y], le = LG.begin[blockIdx.y + 1];
  const uint64_t keep = l2_evict_last();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t bx = lane & 1u;
  const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
  uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int v = 0; v < pl.n_views; ++v) {
    const uint32_t g_end = pl.preQ[v + 1] / kQueryPad;
    // the view's arrays indexed by the padded point index pp: shifted by
    // the view's first padded point (pp - preQ[v] is the point's index)
    const uint32_t vlo = pl.preQ[v], vend = vlo + (uint32_t)pl.v[v].n;
    const float* vpos = pl.v[v].pos - 3ll * vlo;
    OT* vh = static_cast<OT*>(pl.v[v].h) - (long long)vlo * 4 * G.n_levels;
    for (; g < g_end; g += n_warps) {
      const uint32_t pp = g * kQueryPad + (lane >> 1);
      const bool valid = pp < vend;  // views end on warp boundaries: only padding lanes fail
      const uint32_t pc = valid ? pp : vend - 1u;  // a padding lane redoes the view's last point
      const float x = __ldg(vpos + 3 * pc + 0), y = __ldg(vpos + 3 * pc + 1), z = __ldg(vpos + 3 * pc + 2);
      OT* hp = vh + (long long)pc * G.n_levels * 4;
      for (int l = lb; l < le; l += 2) {
        const float2 a = query_half<TT>(G, table, x, y, z, l, bx, keep);
        if (l + 1 < le) {
          const float2 b = query_half<TT>(G, table, x, y, z, l + 1, bx, keep);
          // lane 0 keeps level l's row, lane 1 level l + 1's
          const float2 give = bx ? a : b;
          const float r0 = __shfl_xor_sync(0xffffffffu, give.x, 1), r1 = __shfl_xor_sync(0xffffffffu, give.y, 1);
          const float4 row = bx ? make_float4(r0, r1, b.x, b.y) : make_float4(a.x, a.y, r0, r1);
          if (valid) store_out<OT>(hp, l + (int)bx, row);
        } else if (valid) {
          store_half<OT>(hp, l, bx, a);
        }
      }
    }
  }
}

inpc_status make_plan(const inpc_octree* tree, uint64_t seed, const inpc_front_view* views, int32_t n_views,
                      const GridParams& G, int64_t max_wait_us, FrontPlan& pl) {
  const int64_t L = tree->n_leaves;
  pl.n_views = n_views;
  pl.L = L;
  pl.Gl = guide_log2(L);
  pl.stride_log2 = coarse_stride_log2(L);
  pl.Tw = (uint32_t)ceil_div(L, kWTile);
  pl.Tc = (uint32_t)ceil_div(L, kScanBlock);
  pl.Tg = (uint32_t)ceil_div((int64_t(1) << pl.Gl) + 1, kScanBlock);
  pl.k0 = (uint32_t)seed;
  pl.k1 = (uint32_t)(seed >> 32);
  pl.max_wait_ns = max_wait_us * 1000ll;
  pl.preD[0] = pl.preP[0] = pl.preQ[0] = 0;
  int64_t d = 0, p = 0, q = 0;
  for (int v = 0; v < n_views; ++v) {
    const inpc_front_view& fv = views[v];
    pl.v[v] = FrontView{fv.view_id, fv.n_samples, fv.leaf_idx, fv.pos, fv.h};
    d += ceil_div(fv.n_samples, kDrawPerCta);
    p += ceil_div(fv.n_samples, kPlaceTile);
    q += ceil_div(fv.n_samples, kQueryPad) * kQueryPad;
    pl.preD[v + 1] = (uint32_t)d;
    pl.preP[v + 1] = (uint32_t)p;
    pl.preQ[v + 1] = (uint32_t)q;
  }
  const int64_t counts[kStEnd] = {pl.Tw, pl.Tc, pl.Tg, d, (int64_t)pl.Tc * n_views, p};
  int64_t f = 0;
  for (int s = 0; s < kStEnd; ++s) {
    pl.first[s] = (uint32_t)f;
    f += counts[s];
  }
  if (f >= (int64_t(1) << 31) || q >= (int64_t(1) << 31))
    return fail(INPC_ERR_CAPACITY, "inpc_sample_query_batch: too many work items");
  pl.first[kStEnd] = (uint32_t)f;
  pl.short_by = fault_take_queue_short();
  return INPC_OK;
}

// The sampling of all views: a persistent grid, as many CTAs as fit on the
// GPU at once (more would only queue behind them; fewer also completes,
// since a CTA waits only for tickets taken before its own).  Then the query
// of all views in one launch; it has no waits, so it runs at the query's
// own occupancy.
template <class TT, class OT>
inpc_status launch_front(const FrontPlan& pl, const inpc_octree& tree, const GridParams& G, const TT* table,
                         const FrontWs& ws, cudaStream_t s) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_front, kFrontThreads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int sms = device_sm_count();
  INPC_TIMED("k_front", s, k_front<<<per_sm * sms, kFrontThreads, 0, s>>>(pl, tree, ws));
  INPC_TRY(check_launch("k_front"));
  const long long work = 2ll * pl.preQ[pl.n_views];  // two lanes per padded point
  if (work == 0) return INPC_OK;
  const LevelGroups LG = plan_level_groups(G, sizeof(TT) * 4);
  const dim3 grid((unsigned)std::max<long long>(1, std::min<long long>(ceil_div(work, kFrontThreads), (long long)sms * 16)),
                  (unsigned)LG.n);
  INPC_TIMED("k_front_query", s, k_front_query<TT, OT><<<grid, kFrontThreads, 0, s>>>(pl, G, LG, table));
  return check_launch("k_front_query");
}

}  // namespace
}  // namespace inpc

using namespace inpc;

extern "C" inpc_status inpc_sample_query_batch_workspace_size(int64_t n_leaves, int32_t n_views, size_t* bytes) {
  if (inpc::fault_workspace_overflow())
    return inpc::fail(INPC_ERR_CAPACITY, "inpc_sample_query_batch_workspace_size: size overflow (injected fault)");
  if (!bytes) return fail(INPC_ERR_INVALID_ARG, "inpc_sample_query_batch_workspace_size: bytes is null");
  if (n_leaves < 1 || n_leaves > (int64_t(1) << 24))
    return fail(INPC_ERR_CAPACITY, "n_leaves must be in [1, 2^24], got %lld", (long long)n_leaves);
  if (n_views < 1 || n_views > kFrontMaxViews)
    return fail(INPC_ERR_CAPACITY, "n_views must be in [1, %d], got %d", kFrontMaxViews, n_views);
  *bytes = carve_front(nullptr, n_leaves, n_views).bytes;
  return INPC_OK;
}

extern "C" inpc_status inpc_sample_query_batch(const inpc_octree* tree, uint64_t seed, const inpc_hashgrid_desc* grid,
                                               const void* table, const inpc_front_view* views, int32_t n_views,
                                               int64_t max_wait_us, void* workspace, size_t workspace_bytes,
                                               inpc_stream_t stream) {
  inpc::fault_arg(table);
  if (!tree || !grid || !table || !views)
    return fail(INPC_ERR_INVALID_ARG, "inpc_sample_query_batch: null pointer");
  size_t need = 0;
  INPC_TRY(inpc_sample_query_batch_workspace_size(tree->n_leaves, n_views, &need));
  if (!tree->centers || !tree->levels || !tree->weights)
    return fail(INPC_ERR_INVALID_ARG, "inpc_sample_query_batch: null octree array");
  if (!(tree->root_size > 0.0f)) return fail(INPC_ERR_INVALID_ARG, "root_size must be positive");
  if (!workspace || workspace_bytes < need || !aligned(workspace, 256))
    return fail(INPC_ERR_INVALID_ARG, "inpc_sample_query_batch: workspace null, unaligned or smaller than %zu bytes",
                need);
  if (max_wait_us < 1 || max_wait_us > 60ll * 1000 * 1000)
    return fail(INPC_ERR_INVALID_ARG, "max_wait_us must be in [1, 6e7]");
  GridParams G;
  int64_t n_entries = 0;
  INPC_TRY(make_params(grid, G, &n_entries));
  const size_t ta = grid->table_dtype == INPC_F32 ? 16 : 8, oa = grid->out_dtype == INPC_F32 ? 16 : 8;
  if (!aligned(table, ta)) return fail(INPC_ERR_INVALID_ARG, "inpc_sample_query_batch: misaligned table");
  for (int32_t v = 0; v < n_views; ++v) {
    const inpc_front_view& fv = views[v];
    if (fv.n_samples < 0 || fv.n_samples > (int64_t(1) << 29))
      return fail(INPC_ERR_CAPACITY, "inpc_sample_query_batch: view %d: n_samples must be in [0, 2^29]", v);
    if (fv.n_samples > 0 && (!fv.leaf_idx || !fv.pos || !fv.h))
      return fail(INPC_ERR_INVALID_ARG, "inpc_sample_query_batch: view %d: null output", v);
    if (!aligned(fv.h, oa) || !aligned(fv.pos, 4) || !aligned(fv.leaf_idx, 4))
      return fail(INPC_ERR_INVALID_ARG, "inpc_sample_query_batch: view %d: misaligned output", v);
  }
  FrontPlan pl;
  INPC_TRY(make_plan(tree, seed, views, n_views, G, max_wait_us, pl));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  FrontWs ws = carve_front(workspace, tree->n_leaves, n_views);
  INPC_CUDA(cudaMemsetAsync(workspace, 0, ws.clear_bytes, s), "clear batch workspace");
  const bool t32 = grid->table_dtype == INPC_F32, o32 = grid->out_dtype == INPC_F32;
  if (t32 && o32)
    return launch_front<float, float>(pl, *tree, G, static_cast<const float*>(table), ws, s);
  if (t32) return launch_front<float, __nv_bfloat16>(pl, *tree, G, static_cast<const float*>(table), ws, s);
  if (o32) return launch_front<__nv_bfloat16, float>(pl, *tree, G, static_cast<const __nv_bfloat16*>(table), ws, s);
  return launch_front<__nv_bfloat16, __nv_bfloat16>(pl, *tree, G, static_cast<const __nv_bfloat16*>(table), ws, s);
}
