/*
 * inpc.h -- C ABI of the GB300 (sm_103a) hot path of INPC's implicit point
 * cloud: octree point sampling, multi-resolution hash-grid query, and the
 * differentiable bilinear point rasterizer (forward and backward).
 *
 * Conventions for every entry point
 *   - All array pointers are DEVICE pointers owned by the caller, unless a
 *     parameter says otherwise.  Nothing here allocates device memory: work
 *     buffers are caller-provided ("workspace"), sized by the matching
 *     *_workspace_size query, aligned to 256 bytes.
 *   - Every compute call is asynchronous on the caller's stream (a
 *     cudaStream_t passed as inpc_stream_t; NULL = legacy default stream)
 *     and returns once its kernels are enqueued.  Host-detectable errors
 *     (null pointers, bad sizes, misalignment, unsupported options) return a
 *     non-zero inpc_status before anything is enqueued; a failed launch
 *     returns INPC_ERR_CUDA.  Neither aborts nor traps; inpc_last_error()
 *     gives a thread-local message for the last failure.
 *   - Problems that only the device can see (for example a negative or NaN
 *     leaf weight) set bits in a status word at the start of the workspace
 *     instead of faulting; read it with inpc_read_device_status().
 *   - Arrays are dense, row-major, with no padding between rows.
 */
#ifndef INPC_H
#define INPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* inpc_stream_t; /* same type as cudaStream_t */

typedef enum {
  INPC_OK = 0,
  INPC_ERR_INVALID_ARG = 1,  /* null pointer, bad size, misaligned buffer, workspace too small */
  INPC_ERR_CUDA = 2,         /* a CUDA runtime call or kernel launch failed */
  INPC_ERR_CAPACITY = 3,     /* a problem size exceeds a documented limit */
  INPC_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
  INPC_ERR_UNSUPPORTED = 5   /* an option combination without a kernel */
} inpc_status;

/* Device status bits (inpc_read_device_status). */
#define INPC_DEV_BAD_WEIGHT 0x1u   /* a leaf weight was negative, NaN or infinite */
#define INPC_DEV_NO_WEIGHT 0x2u    /* no leaf weight was positive */
#define INPC_DEV_BAD_LEAF 0x4u      /* inpc_octree_update: a leaf index outside [0, n_leaves) (ignored) */
#define INPC_DEV_BAD_BLEND_WEIGHT 0x8u /* inpc_octree_update: a negative or NaN weight (counted as 0) */
#define INPC_DEV_TIMEOUT 0x10u     /* inpc_sample_query_batch: a bounded work-queue wait gave up (outputs undefined) */

typedef enum { INPC_F32 = 0, INPC_BF16 = 1 } inpc_dtype;

/* Thread-local description of the last error returned on this thread. */
const char* inpc_last_error(void);
/* Library version string. */
const char* inpc_version(void);
/* Number of kernels this library has launched in this process (all devices,
 * all threads); a diagnostic for benchmarks.  Memset/memcpy are not counted. */
uint64_t inpc_kernel_launches(void);
/* Per-kernel device timing, a diagnostic for benchmarks and autotuning (the
 * paper has no counterpart).  While enabled (on != 0), each kernel launch of
 * this library that is not being captured into a CUDA graph is bracketed by
 * two CUDA events recorded on the launch's stream; returns the previous
 * state.  Off by default. */
int inpc_kernel_timer_enable(int on);
/* Waits for the recorded launches of kernel `kernel` (its function name, e.g.
 * "k_point_grad_hash"; NULL = every kernel), stores their summed device time
 * in *total_ms and their number in *launches, and forgets them.  Call it with
 * no launch of this library in progress on another host thread.  Errors:
 * INPC_ERR_INVALID_ARG (null output pointer), INPC_ERR_CUDA. */
inpc_status inpc_kernel_timer_read(const char* kernel, double* total_ms, int64_t* launches);
/* Copies the device status word at the start of `workspace` (any workspace
 * of this library) to *status_out after synchronising `stream`.  A null
 * `workspace` reads the status word of inpc_sample_octree_noalloc instead:
 * the first word of its static scratch array on the current device, which
 * every such call clears before it runs.  Errors: INPC_ERR_INVALID_ARG (null
 * status_out), INPC_ERR_CUDA. */
inpc_status inpc_read_device_status(const void* workspace, inpc_stream_t stream, uint32_t* status_out);

/* ======================================================================== */
/* (a) Octree point sampling                                                */
/* ======================================================================== */
/* Sparse point-probability octree (Sec. 3.1; leaf arrays of App. A.4):
 *   centers  float32 [n_leaves, 3]  world-space leaf centers
 *   levels   int32   [n_leaves]     subdivision level l_i; edge root_size * 2^-l
 *   weights  float64 [n_leaves]     non-negative sampling weights p_i
 * n_leaves must be in [1, 2^24] (the paper's 256^3 leaf cap, Sec. 3.1). */
typedef struct {
  const float* centers;
  const int32_t* levels;
  const double* weights;
  float root_size;
  int64_t n_leaves;
} inpc_octree;

inpc_status inpc_sample_workspace_size(int64_t n_leaves, int64_t n_samples, size_t* bytes);

/* Multinomial sampling with replacement over the leaves, then a uniform
 * position inside each chosen leaf (Sec. 3.2, "Viewpoint-Specific Sampling",
 * the sampling and positioning steps).
 *
 * Definition (integer-exact; bit-identical on any conforming implementation):
 *   q_i   = rint(w_i / max_j w_j * 2^29)      (FP64, round half to even)
 *   cdf_i = q_0 + ... + q_i,  Q = cdf_{L-1}   (exact integers held in FP64)
 *   draw s in [0, n_samples): (r0..r3) = Philox4x32-10(key = (seed lo, seed hi),
 *         counter = (s lo, s hi, view_id, 0)); b = (r1 & 0x1FFFFF) << 32 | r0;
 *         leaf(s) = min{ i : cdf_i > floor(b * Q / 2^53) }
 *   count_i = #{ s : leaf(s) = i }
 *   output slot k in [0, n_samples) holds leaf i for
 *         count_0 + .. + count_{i-1} <= k < count_0 + .. + count_i
 *         (samples grouped by leaf, ascending), and position
 *         pos_k = fl32(c_i + (u - 1/2) * root_size * 2^-l_i),
 *         u_d = (r_d >> 8) * 2^-24 from Philox(counter = (k lo, k hi, view_id, 1)),
 *         rounded once to FP32.
 * Outputs:
 *   leaf_idx_out     int32   [n_samples]
 *   pos_out          float32 [n_samples, 3]
 *   leaf_counts_out  int32   [n_leaves], optional (NULL to skip)
 * n_samples in [0, 2^31 - 1].  Bad weights set INPC_DEV_BAD_WEIGHT /
 * INPC_DEV_NO_WEIGHT in the workspace status; the outputs are then undefined
 * but every write stays in bounds. */
inpc_status inpc_sample_octree(const inpc_octree* tree, uint64_t seed, uint32_t view_id, int64_t n_samples,
                               int32_t* leaf_idx_out, float* pos_out, int32_t* leaf_counts_out,
                               void* workspace, size_t workspace_bytes, inpc_stream_t stream);

/* The counter-based generator behind every random number of the sampler
 * (Sec. 3.2 draws leaves and positions at random; this library takes them
 * from Philox4x32-10, Salmon, Moraes, Dror and Shaw, SC'11, ten rounds with
 * the published multipliers and Weyl key increments).  Evaluates it on n
 * caller-given (key, counter) pairs, so that callers can reproduce the
 * sampler's stream and tests can check the generator against its published
 * known-answer values:
 *   keys  uint32 [n, 2]   (k0, k1): the sampler uses (seed lo, seed hi)
 *   ctrs  uint32 [n, 4]   (c0, c1, c2, c3): the sampler uses
 *                         (index lo, index hi, view_id, purpose)
 *   out   uint32 [n, 4]   the four output words
 * All three are device pointers, 4-byte aligned; n >= 0.
 * Errors: INPC_ERR_INVALID_ARG (null pointer with n > 0, negative n). */
inpc_status inpc_philox4x32_10(const uint32_t* keys, const uint32_t* ctrs, int64_t n, uint32_t* out,
                               inpc_stream_t stream);

/* Allocation-free variant of inpc_sample_octree (the paper has no
 * counterpart; this is a deployment aid).  Some callers cannot allocate
 * device memory at all: a host application or engine that owns every byte of
 * the device behind its own allocator, a frame loop that must not stall on a
 * cudaMalloc, or a plugin that is handed buffers but no allocation rights.
 * They still pass the octree and the output arrays; the sampler's scratch
 * lives in a file-scope device array of INPC_SAMPLE_STATIC_SCRATCH_BYTES
 * (4 MiB + 576 KiB: about 266,000 leaves), which every GPU that loads this
 * library holds until the process exits.
 *   - Same definition, outputs and device status bits as inpc_sample_octree;
 *     the status word is the first word of the static array, read with
 *     inpc_read_device_status(NULL, stream, &status) on the same device.
 *   - Returns INPC_ERR_CAPACITY, before touching the device, when the tree
 *     needs more scratch than the array holds.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and caches it with the id of the current CUDA
 *     context; a call in another context of that device (for instance after
 *     cudaDeviceReset, which also discards the array's contents) looks it up
 *     again.  Make the first call on a device before any stream capture.
 *   - Allocates nothing (no cudaMalloc, no library allocation); every call on
 *     a device shares the one array, each call clears what must start at
 *     zero, and calls whose GPU work overlaps (other streams, other host
 *     threads) race on it. */
#define INPC_SAMPLE_STATIC_SCRATCH_BYTES ((4u << 20) + (576u << 10))
inpc_status inpc_sample_octree_noalloc(const inpc_octree* tree, uint64_t seed, uint32_t view_id, int64_t n_samples,
                                       int32_t* leaf_idx_out, float* pos_out, int32_t* leaf_counts_out,
                                       inpc_stream_t stream);

/* ======================================================================== */
/* (b) Multi-resolution hash-grid query                                     */
/* ======================================================================== */
/* Grid description (Sec. 3.3; configuration space of Listing 1, App. A.5).
 *   n_levels    1..32
 *   n_feats     features per level; 4 is the supported value
 *   log2_T      per-level entry budget T = 2^log2_T, 4 <= log2_T <= 24
 *   res[l]      grid resolution N_l >= 1 of level l (host integers)
 *   table_dtype INPC_F32 or INPC_BF16 (dtype of the parameter table)
 *   out_dtype   INPC_F32 or INPC_BF16 (dtype of the query output h)
 * Table layout: level-major; level l has E_l = min(T, (N_l+1)^3) rows of
 * n_feats values and starts on a multiple of 16 rows (the total is rounded
 * up to 16; padding rows are never read and receive no gradient); level l
 * is stored densely iff (N_l+1)^3 <= T (row =
 * x + y (N_l+1) + z (N_l+1)^2), otherwise through the spatial hash
 * row = (x * 1 ^ y * 2654435761 ^ z * 805459861) mod T (uint32 arithmetic). */
typedef struct {
  int32_t n_levels;
  int32_t n_feats;
  int32_t log2_T;
  int32_t res[32];
  int32_t table_dtype;
  int32_t out_dtype;
} inpc_hashgrid_desc;

/* Total table rows (sum of E_l with the 16-row alignment of every level). */
inpc_status inpc_hashgrid_n_entries(const inpc_hashgrid_desc* g, int64_t* n_entries);

/* h[p, l * n_feats + f] = sum over the 8 corners of the level-l cell holding
 * x = clamp(pos[p], 0, 1) of the trilinear weight times table[row, f]
 * (cell = min(floor(x N_l), N_l - 1) per axis; the fraction x N_l - cell is
 * formed exactly).  pos: float32 [n, 3]; table: [n_entries, n_feats] of
 * table_dtype; h_out: [n, n_levels * n_feats] of out_dtype.  Arithmetic is
 * FP32.  n in [0, 2^29] (INPC_ERR_CAPACITY beyond). */
inpc_status inpc_query_hashgrid(const inpc_hashgrid_desc* g, const void* table, const float* pos, int64_t n,
                                void* h_out, inpc_stream_t stream);

/* Adjoint of inpc_query_hashgrid: grad_table[row, f] += weight * dh[p, l * n_feats + f]
 * for every point, level and corner.  dh: float32 [n, n_levels * n_feats];
 * grad_table: float32 [n_entries, n_feats], accumulated (not cleared), FP32
 * even for BF16 tables.  Summation order is unspecified (atomic adds). */
inpc_status inpc_query_hashgrid_bwd(const inpc_hashgrid_desc* g, const float* pos, const float* dh, int64_t n,
                                    float* grad_table, inpc_stream_t stream);

/* ======================================================================== */
/* (c) Differentiable bilinear point rasterizer                             */
/* ======================================================================== */
/* Pinhole camera (Eq. 5): x_c = R x_w + t (R row-major), then
 *   u = fx * (x_c / z_c) + cx,  v = fy * (y_c / z_c) + cy,  depth d = z_c,
 * evaluated in FP32 in exactly this order: each camera coordinate is
 * fma(R[3r+2], z, fma(R[3r+1], y, fma(R[3r], x, t[r]))), the quotient is
 * IEEE-rounded, and u, v are fma(fx, x_c / z_c, cx).  Points with
 * d <= near_plane or d >= far_plane (or NaN) are culled.  Pixel (i, j)
 * covers [i, i+1) x [j, j+1), center (i + 0.5, j + 0.5). */
typedef struct {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  float near_plane, far_plane;
} inpc_camera;

typedef enum {
  INPC_OPACITY_GIVEN = 0,    /* alpha_h = opacity[p] */
  INPC_OPACITY_FROM_CH0 = 1  /* alpha_h = 1 - exp(-exp(feat[p, 0])) (Sec. 3.3 activation);
                                the blended color is (1, feat[p, 1:]) */
} inpc_opacity_mode;

/*   opacity_mode  inpc_opacity_mode
 *   n_channels    F, 1..128 (F/4 <= 32 when F % 4 == 0, else F <= 32)
 *   feat_dtype    INPC_F32 or INPC_BF16 (dtype of the feature rows)
 *   image_dtype   must equal feat_dtype (dtype of the image); blending,
 *                 transmittance and every gradient stay FP32
 *   t_min         blending stops after the fragment that takes T below it (1e-4)
 *   alpha_max     splat opacity clamp, alpha = min(alpha_h w, alpha_max), < 1 (0.99)
 *   tile_w/tile_h screen tile in pixels, tile_w * tile_h <= 256; 0 = default 16 x 8
 *                 (groups pixels into CTAs; never changes a result)
 * Alignment: feat and image 16 bytes when n_channels % 4 == 0 (FP32) or
 * n_channels = 64 (BF16), 8 bytes for other BF16 multiples of 4, else their
 * element size; d_image / d_feat 16 bytes when n_channels % 4 == 0. */
typedef struct {
  int32_t opacity_mode;
  int32_t n_channels;
  int32_t feat_dtype;
  int32_t image_dtype;
  float t_min;
  float alpha_max;
  int32_t tile_w;
  int32_t tile_h;
} inpc_raster_opts;

inpc_status inpc_rasterize_workspace_size(const inpc_camera* cam, const inpc_raster_opts* opts, int64_t n,
                                          size_t* bytes);

/* Forward (Algorithm 1: ProjectAndCull, BilinearSplatting, order, blend).
 * Each visible point p splats to the 2x2 pixels whose centers are nearest to
 * (u, v) (i0 = floor(u - 1/2), j0 = floor(v - 1/2)) with alpha =
 * min(alpha_h (1 - |u - u_i|)(1 - |v - v_j|), alpha_max) (Eq. 6); off-image
 * pixels are dropped.  Per pixel, fragments are ordered by (FP32 depth,
 * point index) ascending and blended front to back (Eq. 1): C += T alpha c,
 * T *= 1 - alpha, stopping after the fragment that takes T below t_min.
 *   pos      float32 [n, 3]
 *   opacity  float32 [n] (INPC_OPACITY_GIVEN only; NULL otherwise)
 *   feat     [n, F] of feat_dtype
 *   image    [H, W, F] of image_dtype;  T_final float32 [H, W];
 *   n_contrib int32 [H, W] (fragments blended per pixel)
 * The workspace must stay untouched until the matching inpc_rasterize_bwd.
 * n in [0, 2^28] (4n fragment slots are 32-bit).  The sort key holds the
 * point index beside the depth: up to 2^25 points the depth's raw FP32 bits,
 * beyond that its bits above those of near_plane, which must then span at
 * fewer than 2^(56 - b) values up to far_plane for b-bit point indices
 * (INPC_ERR_CAPACITY otherwise; near = 0.01, far = 100 allow 2^28 points).
 * The calls that continue from this one (inpc_rasterize_bwd,
 * inpc_rasterize_bwd_hashgrid, inpc_rasterize_point_weights) take n <= 2^25. */
inpc_status inpc_rasterize_fwd(const inpc_camera* cam, const inpc_raster_opts* opts, const float* pos,
                               const float* opacity, const void* feat, int64_t n, void* image, float* T_final,
                               int32_t* n_contrib, void* workspace, size_t workspace_bytes, inpc_stream_t stream);

/* Backward of inpc_rasterize_fwd (App. A.6) for upstream d_image [H, W, F]
 * (float32).  Per pixel, T_k is recomputed from the fragments' alphas by the
 * forward's own front-to-back product (the same rounding, no division by
 * 1 - alpha; nothing stored between the calls), then the blended fragments
 * are revisited back to front with the suffix sums
 * S_k = sum_{j>k} T_j alpha_j (c_j . g):
 * dL/dalpha_k = T_k (c_k . g) - S_k / (1 - alpha_k).  Writes (does not accumulate):
 *   d_feat     float32 [n, F]: sum of the point's splat gradients T_k alpha_k g;
 *              in FROM_CH0 mode column 0 is d alpha_h * exp(h0) exp(-exp(h0))
 *   d_opacity  float32 [n] (GIVEN mode; may be NULL in FROM_CH0 mode):
 *              sum over splats of w_k dL/dalpha_k (0 where alpha was clamped)
 * Culled points get zero rows.  Inputs must be those of the forward call,
 * with its T_final, n_contrib and unmodified workspace. */
inpc_status inpc_rasterize_bwd(const inpc_camera* cam, const inpc_raster_opts* opts, const float* pos,
                               const float* opacity, const void* feat, int64_t n, const float* T_final,
                               const int32_t* n_contrib, const float* d_image, float* d_opacity, float* d_feat,
                               void* workspace, size_t workspace_bytes, inpc_stream_t stream);

/* Rasterizer backward fused with the grid query's adjoint, for head mode
 * (INPC_OPACITY_FROM_CH0) when the features are the grid query's output
 * (n_channels = n_levels * n_feats): the same result as inpc_rasterize_bwd
 * followed by inpc_query_hashgrid_bwd on its d_feat, but each point's
 * gradient row goes from registers straight into the table gradient, so it
 * is never written to and read back from memory (App. A.6 backward, then the
 * adjoint of the Sec. 3.3 query).
 *   grid        descriptor of the query that produced `feat`
 *   grad_table  float32 [n_entries, n_feats], accumulated (+=)
 *   d_feat      optional float32 [n, F]: also written when non-NULL
 * The workspace is the forward's, sized by
 * inpc_rasterize_bwd_hashgrid_workspace_size: the rasterizer's size, plus,
 * when the gradient rows of the fine half of the levels (levels n_levels/2
 * and up for 16 levels) exceed 64 MB, n * (those levels) * 16 bytes in which
 * the fine levels' gradient rows wait for a second pass that adds them
 * level group by level group, so that the rows receiving additions stay in
 * L2.  Additions into grad_table are atomic, so several calls may
 * accumulate into one table concurrently.  Other arguments as for
 * inpc_rasterize_bwd. */
inpc_status inpc_rasterize_bwd_hashgrid_workspace_size(const inpc_camera* cam, const inpc_raster_opts* opts,
                                                       const inpc_hashgrid_desc* grid, int64_t n, size_t* bytes);
inpc_status inpc_rasterize_bwd_hashgrid(const inpc_camera* cam, const inpc_raster_opts* opts,
                                        const inpc_hashgrid_desc* grid, const float* pos, const void* feat, int64_t n,
                                        const float* T_final, const int32_t* n_contrib, const float* d_image,
                                        float* grad_table, float* d_feat, void* workspace, size_t workspace_bytes,
                                        inpc_stream_t stream);

/* View-specific leaf weights (Sec. 3.2 Eq. 4 with App. A.4 "Depth
 * Calculation"): w_i = 1_visible p_i / (d_i 2^(l_i lambda_l)), where
 *   - a leaf is visible unless all 8 corners of its cube lie outside one
 *     plane of the view frustum (near < z < far, 0 <= u < W, 0 <= v < H);
 *   - d_i = max(|z_i - near| / far, tau_d), z_i the view-space depth of the
 *     leaf center;
 *   - 2^(l lambda_l) is evaluated on the host (exp2, levels 0..63; leaves
 *     with other levels get weight 0).
 * FP64 throughout with a fixed operation order (camera coordinates
 * ((R_k0 x + R_k1 y) + R_k2 z) + t_k).  The paper uses lambda_l = 0.5 and
 * tau_d = 1e-8.  tree->weights holds p; w_out float64 [n_leaves].
 * Errors: INPC_ERR_INVALID_ARG (null pointer, bad camera, tau_d <= 0). */
inpc_status inpc_view_weights(const inpc_octree* tree, const inpc_camera* cam, double lambda_l, double tau_d,
                              double* w_out, inpc_stream_t stream);

/* Viewpoint-specific sampling with the re-sampling of App. A.4 ("Ensuring
 * Sample Count"): inpc_sample_octree with tree->weights = the view weights
 * (inpc_view_weights), then up to max_rounds rounds in which every sample
 * whose position is not in view (the rasterizer's FP32 projection keeps it
 * and it lands in [0, W) x [0, H)) draws, in place, a new leaf from the same
 * distribution (Philox counter (j, view, 2 + 2r)) and a new position in it
 * (counter (j, view, 3 + 2r)); samples already in view never change.
 *   n_left  optional device uint32: the number of samples still not in view
 *           after the last round
 * max_rounds in [0, 64]; other arguments, workspace and errors as for
 * inpc_sample_octree.  Asynchronous. */
inpc_status inpc_sample_octree_view(const inpc_octree* tree, const inpc_camera* cam, uint64_t seed,
                                    uint32_t view_id, int64_t n_samples, int32_t max_rounds, int32_t* leaf_idx_out,
                                    float* pos_out, uint32_t* n_left, void* workspace, size_t workspace_bytes,
                                    inpc_stream_t stream);

/* Viewpoint-independent pre-extraction (Sec. 3.2): leaf weights of Eq. 4
 * without the visibility indicator and the depth, w_i = p_i / 2^(l_i lambda_l)
 * (2^(l lambda_l) by exp2 on the host for levels 0..63; other levels get 0),
 * FP64.  tree->weights holds p; w_out float64 [n_leaves]. */
inpc_status inpc_level_weights(const inpc_octree* tree, double lambda_l, double* w_out, inpc_stream_t stream);

/* Pre-extraction sampling: the per-leaf counts of n_samples draws with
 * replacement from tree->weights (exactly inpc_sample_octree's draws with
 * view_id 0), leaf-grouped output, and the k-th sample of a leaf (k = 0, 1,
 * ...) placed at c + (h - 1/2) root_size 2^-l with h the 3D Halton point of
 * index k + 1 (radical inverses in bases 2, 3, 5, each the exact fraction
 * n / b^m divided once in FP64), rounded once to FP32.  Arguments,
 * workspace and errors as for inpc_sample_octree. */
inpc_status inpc_sample_octree_halton(const inpc_octree* tree, uint64_t seed, int64_t n_samples,
                                      int32_t* leaf_idx_out, float* pos_out, int32_t* leaf_counts_out,
                                      void* workspace, size_t workspace_bytes, inpc_stream_t stream);

/* Inference multisampling (Sec. 3.2): several point clouds are rasterized and
 * their feature images averaged per pixel.  acc[i] += scale * image[i] for
 * i < n_elems (FP32 accumulator; image of dtype INPC_F32 or INPC_BF16), one
 * rounding per element (FMA). */
inpc_status inpc_accumulate_image(const void* image, int32_t dtype, int64_t n_elems, float scale, float* acc,
                                  inpc_stream_t stream);

/* ======================================================================== */
/* (e) View-dependent head (Sec. 3.3)                                        */
/* ======================================================================== */

/* Spherical contraction of the query positions (Sec. 3.3, mip-NeRF 360):
 * y = (x - center) / radius; contract(y) = y for |y| <= 1, else
 * (2 - 1/|y|) y / |y|; out = contract(y) / 4 + 1/2, in [0, 1]^3.  FP32 with a
 * fixed operation order: y_d = (x_d - c_d) / radius;
 * r = sqrt(fma(y2, y2, fma(y1, y1, y0 * y0))); s = (2 - 1/r) / r for r > 1;
 * out_d = fma(y_d * s, 1/4, 1/2).  pos, out float32 [n, 3] (may alias);
 * center float32 [3] (host). */
inpc_status inpc_contract_positions(const float* pos, int64_t n, const float* center, float radius, float* out,
                                   inpc_stream_t stream);

/* Appearance head: alpha_h = 1 - exp(-exp(h0)) and a 4D view-dependent
 * color from degree-2 real orthonormal spherical harmonics of the viewing
 * direction d = (x - o) / |x - o| (o the camera center):
 *   color_c = sum_{k<9} Y_k(d) h[1 + 9 c + k],  c < 4
 * with Y_0 = sqrt(1/4pi), Y_1..3 = sqrt(3/4pi) (y, z, x), Y_4..8 =
 * sqrt(15/4pi) xy, sqrt(15/4pi) yz, sqrt(5/16pi)(3z^2 - 1), sqrt(15/4pi) xz,
 * sqrt(15/16pi)(x^2 - y^2).  h [n, n_channels] of h_dtype (n_channels >= 37:
 * 1 opacity + 36 SH coefficients; further channels unused); alpha_out
 * float32 [n]; color_out float32 [n, 4] (16-byte aligned).  The outputs feed
 * inpc_rasterize_fwd in INPC_OPACITY_GIVEN mode with 4 channels. */
inpc_status inpc_sh_head_fwd(const inpc_camera* cam, const float* pos, const void* h, int32_t h_dtype, int64_t n,
                             int32_t n_channels, float* alpha_out, float* color_out, inpc_stream_t stream);

/* Derivative of inpc_sh_head_fwd: dh[0] = d_alpha exp(h0) exp(-exp(h0)),
 * dh[1 + 9c + k] = Y_k(d) d_color_c, every other channel 0; dh_out float32
 * [n, n_channels], written. */
inpc_status inpc_sh_head_bwd(const inpc_camera* cam, const float* pos, const void* h, int32_t h_dtype, int64_t n,
                             int32_t n_channels, const float* d_alpha, const float* d_color, float* dh_out,
                             inpc_stream_t stream);

/* ======================================================================== */
/* (d) Octree maintenance (Sec. 3.1 "Probability Updates", "Subdivision",   */
/*     "Pruning"; App. A.4)                                                  */
/* ======================================================================== */

/* Per-point blending weights for the probability updates: Eq. 2 takes the
 * transmitted blending weight T alpha of every point, and App. A.6 combines
 * a point's four splat weights by their bilinear weights:
 *   b[p] = sum over the point's blended splats k of w_k T_k alpha_k
 * (0 for splats that were not blended and for culled points).  T_k is
 * recomputed from the forward's recorded blending order with the forward's
 * own product scan, so it is bitwise the forward's.
 *   cam, opts, pos, n, n_contrib, workspace: those of the inpc_rasterize_fwd
 *              call (the workspace unmodified since; its per-fragment
 *              scratch of the backward is reused, so call this before or
 *              after inpc_rasterize_bwd, not while it runs)
 *   b_out      float32 [n], written
 * Errors: INPC_ERR_INVALID_ARG (null pointer, workspace too small). */
inpc_status inpc_rasterize_point_weights(const inpc_camera* cam, const inpc_raster_opts* opts, const float* pos,
                                         int64_t n, const int32_t* n_contrib, float* b_out, void* workspace,
                                         size_t workspace_bytes, inpc_stream_t stream);

/* Probability updates after one step (Eq. 2 and Eq. 3): for every leaf i,
 * with B_i the weights b of the points drawn from leaf i in this step,
 *   p_i = max(lambda_u p_i, max B_i),   q_i = max(lambda_u q_i, max B_i - min B_i),
 * max / min over FP32 values, the update in FP64; a leaf no point was drawn
 * from only decays (p_i = lambda_u p_i, q_i = lambda_u q_i).  The paper uses
 * lambda_u = 0.9968 (and skips updates in the first 100 iterations, a
 * schedule left to the caller).
 *   leaf_idx   int32 [n]: leaf of each point (inpc_sample_octree's output)
 *   b          float32 [n]: inpc_rasterize_point_weights' output (>= 0;
 *              negative or NaN values count as 0 and set
 *              INPC_DEV_BAD_BLEND_WEIGHT; out-of-range leaves are ignored
 *              and set INPC_DEV_BAD_LEAF in the workspace status)
 *   p, q       float64 [n_leaves], updated in place (p is the octree's
 *              sampling weight array)
 *   workspace  inpc_octree_update_workspace_size(n_leaves) bytes, 256-aligned
 * n_leaves in [1, 2^24]; lambda_u in [0, 1].  Asynchronous. */
inpc_status inpc_octree_update_workspace_size(int64_t n_leaves, size_t* bytes);
inpc_status inpc_octree_update(const int32_t* leaf_idx, const float* b, int64_t n, double* p, double* q,
                               int64_t n_leaves, double lambda_u, void* workspace, size_t workspace_bytes,
                               inpc_stream_t stream);

/* Subdivision (Sec. 3.1): every leaf with q_i > tau_s (0.5 in the paper) is
 * replaced, in its place in the list, by its 8 children: level l_i + 1,
 * centers c_i + (d - 1/2) root_size 2^-(l_i+1) per axis for d in {0, 1},
 * child k = d_x + 2 d_y + 4 d_z (Morton order within the parent, so a
 * Morton-ordered list stays Morton-ordered); children inherit p_i and start
 * with q = 0.  If the resulting leaf count would not stay below max_leaves
 * (256^3 in the paper, for the sampler's precision), no leaf is subdivided
 * and the tree is copied unchanged.
 *   tree       input leaves (weights = p); q float64 [n_leaves]
 *   *_out      output leaves (centers float32 [cap, 3], levels int32 [cap],
 *              p_out, q_out float64 [cap]); cap = out_capacity, at most
 *              8 n_leaves are ever needed
 *   n_out      receives the new leaf count
 *   workspace  inpc_octree_refine_workspace_size(n_leaves) bytes
 * Synchronises `stream` (the output count decides the capacity check).
 * Errors: INPC_ERR_INVALID_ARG, INPC_ERR_CAPACITY (out_capacity too small;
 * nothing written). */
inpc_status inpc_octree_refine_workspace_size(int64_t n_leaves, size_t* bytes);
inpc_status inpc_octree_subdivide(const inpc_octree* tree, const double* q, double tau_s, int64_t max_leaves,
                                  float* centers_out, int32_t* levels_out, double* p_out, double* q_out,
                                  int64_t out_capacity, int64_t* n_out, void* workspace, size_t workspace_bytes,
                                  inpc_stream_t stream);

/* Pruning (Sec. 3.1): leaves with p_i < tau_p (0.01 in the paper) are
 * removed; the others keep their order.  Arguments and errors as for
 * inpc_octree_subdivide (at most n_leaves outputs). */
inpc_status inpc_octree_prune(const inpc_octree* tree, const double* q, double tau_p, float* centers_out,
                              int32_t* levels_out, double* p_out, double* q_out, int64_t out_capacity,
                              int64_t* n_out, void* workspace, size_t workspace_bytes, inpc_stream_t stream);

/* ======================================================================== */
/* (f) Batches of views                                                     */
/* ======================================================================== */
/* One view of a batch (all pointers are device memory owned by the caller;
 * nothing in a job is read after inpc_render_batch's work completes).
 *   cam, opts   the view's camera and rasterizer options (head mode,
 *               n_channels = 4 * grid levels; tile sizes may differ per view)
 *   view_id     the view's Philox stream of the batch's seed (Sec. 3.2)
 *   n_samples   points drawn for this view
 *   leaf_idx, pos, h   [n] int32, [n, 3] float32, [n, n_channels] of
 *               opts.feat_dtype (= the grid's out_dtype): sampled points and
 *               their features
 *   image, T_final, n_contrib   the forward's outputs, as for
 *               inpc_rasterize_fwd
 *   d_image     float32 [H, W, n_channels] upstream image gradient, or NULL
 *               for a forward-only view
 *   sample_ws   inpc_sample_workspace_size(n_leaves, n_samples) bytes
 *   raster_ws   inpc_rasterize_bwd_hashgrid_workspace_size(...) bytes */
typedef struct {
  inpc_camera cam;
  inpc_raster_opts opts;
  uint32_t view_id;
  int64_t n_samples;
  int32_t* leaf_idx;
  float* pos;
  void* h;
  void* image;
  float* T_final;
  int32_t* n_contrib;
  const float* d_image;
  void* sample_ws;
  size_t sample_ws_bytes;
  void* raster_ws;
  size_t raster_ws_bytes;
} inpc_view_job;

/* A batch of views of one scene (the paper renders one viewpoint per
 * training iteration, Sec. 4.1; a batch of independent views is this
 * library's throughput form and has no counterpart in the paper): every
 * view samples the shared octree, queries the
 * shared grid `table`, rasterizes, and, when its d_image is given, runs the
 * fused backward, adding into the shared FP32 `grad_table` (atomic, so
 * views may run concurrently; the caller zeroes it).  Each view is exactly
 * the sequence inpc_sample_octree -> inpc_query_hashgrid ->
 * inpc_rasterize_fwd -> inpc_rasterize_bwd_hashgrid.
 * Views are spread round-robin over `streams` (n_streams >= 1, distinct):
 * the call forks them from streams[0] and joins them back into it, so all
 * of the batch is ordered after earlier work on streams[0] and before later
 * work there, and one stream capture on streams[0] records the whole batch
 * as one CUDA graph (replayed as one launch per step).
 * Errors: INPC_ERR_INVALID_ARG (null or bad arguments, repeated streams),
 * or the first error of a view's call (the remaining views are not
 * enqueued; the streams are still joined). */
inpc_status inpc_render_batch(const inpc_octree* tree, uint64_t seed, const inpc_hashgrid_desc* grid,
                              const void* table, const inpc_view_job* views, int32_t n_views, float* grad_table,
                              const inpc_stream_t* streams, int32_t n_streams);

/* ------------------------------------------------------------------------ */
/* Persistent front end of a batch of views (many camera views per launch:  */
/* the paper renders one view at a time, Sec. 4.1 and Table 2 time it).    */
/* ------------------------------------------------------------------------ */
/* One view of inpc_sample_query_batch:
 *   view_id    the view's Philox stream of the batch's seed (Sec. 3.2)
 *   n_samples  points drawn for the view, in [0, 2^29]
 *   leaf_idx   int32 [n_samples], pos float32 [n_samples, 3]: as
 *              inpc_sample_octree's outputs
 *   h          [n_samples, 4 * n_levels] of the grid's out_dtype: as
 *              inpc_query_hashgrid's output (16-byte aligned for FP32,
 *              8-byte for BF16) */
typedef struct {
  uint32_t view_id;
  int64_t n_samples;
  int32_t* leaf_idx;
  float* pos;
  void* h;
} inpc_front_view;

/* Workspace bytes of inpc_sample_query_batch for a tree of n_leaves and a
 * batch of n_views views.  Errors: INPC_ERR_CAPACITY (n_leaves outside
 * [1, 2^24], n_views outside [1, 64]). */
inpc_status inpc_sample_query_batch_workspace_size(int64_t n_leaves, int32_t n_views, size_t* bytes);

/* The sampling (Sec. 3.2, exactly inpc_sample_octree's definition) and the
 * grid query (Sec. 3.3, exactly inpc_query_hashgrid's) of n_views views of
 * one octree and one table in two launches: the sampling of every view in
 * ONE persistent kernel, whose CTAs take work items (stage, view, tile) from
 * a queue in the workspace and wait for the items an item depends on; then
 * the query of every view in one more launch.  The leaf CDF is built once
 * for the batch.  Outputs are bit-identical to inpc_sample_octree followed
 * by inpc_query_hashgrid for each view.
 *   max_wait_us  bound of every wait, in microseconds of the GPU's global
 *                timer, in [1, 6e7]; a wait that runs out sets
 *                INPC_DEV_TIMEOUT in the workspace's status word (read with
 *                inpc_read_device_status), every CTA then returns, and the
 *                outputs are undefined.  No wait is longer than its bound.
 * Device status bits as inpc_sample_octree (bad and all-zero weights) plus
 * INPC_DEV_TIMEOUT.  The workspace must not be shared by calls whose GPU
 * work overlaps.  Errors: INPC_ERR_INVALID_ARG (null pointer, misaligned
 * output, workspace too small, max_wait_us out of range), INPC_ERR_CAPACITY
 * (sizes), INPC_ERR_UNSUPPORTED (grid options), INPC_ERR_CUDA. */
inpc_status inpc_sample_query_batch(const inpc_octree* tree, uint64_t seed, const inpc_hashgrid_desc* grid,
                                    const void* table, const inpc_front_view* views, int32_t n_views,
                                    int64_t max_wait_us, void* workspace, size_t workspace_bytes,
                                    inpc_stream_t stream);

/* inpc_render_batch with the sampling and query of all views through
 * inpc_sample_query_batch (up to 64 views per call, on streams[0], before
 * the fork), then each view's rasterizer
 * forward and fused backward over the streams as in inpc_render_batch.  The
 * jobs' sample_ws are not used; front_workspace holds
 * inpc_sample_query_batch_workspace_size(n_leaves, min(n_views, 64)) bytes.
 * Outputs are bit-identical to inpc_render_batch's (the table gradient up
 * to the order of its atomic additions).  max_wait_us and the device status
 * (in front_workspace) as for inpc_sample_query_batch.  Errors as for
 * inpc_render_batch and inpc_sample_query_batch. */
inpc_status inpc_render_batch_persistent(const inpc_octree* tree, uint64_t seed, const inpc_hashgrid_desc* grid,
                                         const void* table, const inpc_view_job* views, int32_t n_views,
                                         float* grad_table, const inpc_stream_t* streams, int32_t n_streams,
                                         void* front_workspace, size_t front_workspace_bytes, int64_t max_wait_us);

/* Host-side fault injection for failure tests (no counterpart in the
 * paper).  spec (NULL or "" disarms):
 *   "workspace_overflow"  every *_workspace_size query returns
 *                         INPC_ERR_CAPACITY, as if the sizes overflowed
 *   "corrupt_args"        every compute entry point sees its first array
 *                         argument as NULL; its own validation must then
 *                         return INPC_ERR_INVALID_ARG before enqueuing
 *                         anything
 *   "queue_short"         the next inpc_sample_query_batch launch waits for
 *                         one more draw tile of its first view than exists,
 *                         so that wait runs out (INPC_DEV_TIMEOUT) and the
 *                         kernel returns; disarmed by that launch
 * The INPC_FAULT environment variable, read at the library's first use,
 * arms the same faults.  Nothing is injected on the device.  Errors:
 * INPC_ERR_INVALID_ARG (unknown spec). */
inpc_status inpc_set_fault(const char* spec);

/* Calibration for roofline reporting (no counterpart in the paper): the
 * rate at which this GPU performs the operation that bounds the grid
 * adjoint's table-gradient additions (the adjoint of the Sec. 3.3 query in
 * the App. A.6 backward), 16-byte FP32 vector reductions
 * (red.global.add.v4.f32) into uniformly random rows of an L2-resident
 * region.  Every SM runs 8 CTAs of 256 threads, each thread 128 reductions
 * per launch; two launches warm up, five are timed with CUDA events on
 * `stream`, and the call waits for them.
 *   buf      device float32 [rows, 4], 16-byte aligned, owned by the caller;
 *            its contents are overwritten (sums of ones)
 *   rows     a power of two in [2^10, 2^26] (the region: rows * 16 bytes)
 *   paired   0: every lane reduces into its own random row; 1: lanes 2j and
 *            2j + 1 reduce into the two rows of one 32-byte sector, as the
 *            adjoint's x-vertex pairs do
 *   gops     out: rows reduced per second / 1e9 (lane reductions)
 * Errors: INPC_ERR_INVALID_ARG (null pointers, misaligned buf, rows not a
 * power of two in range), INPC_ERR_CUDA. */
inpc_status inpc_l2_reduction_rate(float* buf, int64_t rows, int32_t paired, double* gops, inpc_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* INPC_H */
