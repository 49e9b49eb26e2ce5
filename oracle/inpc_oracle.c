/*
 * inpc_oracle.c -- plain, slow, FP64 CPU oracle for the INPC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke check
 * and the benchmark's CPU-baseline leg may load this library.  It shares no
 * code, header, table or helper with the CUDA path; it is written directly
 * from the paper's definitions, one function per step, in the paper's order:
 *
 *   sampling      Sec. 3.2 "Viewpoint-Specific Sampling" (multinomial sampling
 *                 with replacement, uniform position in the chosen leaf), with
 *                 the precision remark of Sec. 3.1 "Subdivision";
 *   hash query    Sec. 3.3 and App. A.5 (multi-resolution grid, trilinear
 *                 interpolation per level, features concatenated);
 *   rasterizer    Sec. 3.4 (Eq. 5 projection, Eq. 6 bilinear opacity),
 *                 Eq. 1 front-to-back alpha blending, App. A.6 early stop at
 *                 transmittance 1e-4 and Algorithm 1's stage order;
 *   backward      App. A.6 "During optimization ..." (per-splat gradients
 *                 combined into per-point gradients), written here as the
 *                 plain analytic derivative of the forward definition;
 *   octree        Sec. 3.1 "Probability Updates" (Eq. 2, Eq. 3, with the
 *                 per-point blending weights of App. A.6), "Subdivision" and
 *                 "Pruning", App. A.4 leaf layout;
 *   view sampling Sec. 3.2 "Viewpoint-Specific Sampling" (Eq. 4) with App.
 *                 A.4 "Depth Calculation" and "Ensuring Sample Count";
 *   pre-extraction Sec. 3.2 "Viewpoint-Independent Sampling" (Eq. 4 without
 *                 visibility and depth, multinomial counts, 3D Halton
 *                 positions);
 *   SH head       Sec. 3.3: spherical contraction of the query positions,
 *                 opacity from the first feature, degree-2 spherical
 *                 harmonics on the next 36 features giving a 4D
 *                 view-dependent color per point, and its derivative.
 *
 * Readings where the paper is silent (all listed in the design notes):
 *   - leaf weights are quantised to integers q_i = rint(w_i / max w * 2^29)
 *     and the CDF is their exact prefix sum (FP64 holds every partial sum
 *     exactly while the leaf count stays below 2^24, the paper's 256^3 cap);
 *   - the leaf drawn for a 53-bit uniform integer b is the smallest i with
 *     cdf_i > floor(b * Q / 2^53), Q = sum q (zero-weight leaves never drawn);
 *   - the sampled list of leaf indices is emitted grouped by leaf, in
 *     ascending leaf order (the draws fix only how many samples each leaf
 *     gets); positions are drawn per output slot;
 *   - random numbers come from Philox4x32-10 (Salmon et al., SC'11) keyed by
 *     the 64-bit seed, counter (sample lo, sample hi, view, purpose);
 *   - a level-l leaf spans center +- root_size * 2^-l / 2, half-open;
 *   - grid level l has resolution N_l; vertex coordinates 0..N_l; the level is
 *     stored densely iff (N_l+1)^3 <= T, else through the spatial hash
 *     x*1 ^ y*2654435761 ^ z*805459861 (mod T); levels start on multiples of
 *     16 table rows;
 *   - the projection (Eq. 5) is evaluated in the kernel's FP32 arithmetic with
 *     a fixed operation order, because it decides integer pixel indices and
 *     the depth order; everything downstream of it is FP64 here;
 *   - pixel (i, j) has its center at (i + 0.5, j + 0.5);
 *   - per-pixel order: ascending (FP32 depth, point id);
 *   - alpha = min(alpha_h * w, alpha_max); blending stops after the fragment
 *     whose update takes T below t_min (that fragment is included);
 *   - a point's feature gradient is the plain sum of its splat gradients; its
 *     opacity gradient sums the splat gradients times dalpha/dalpha_h;
 *   - a point's blending weight for the octree updates is the sum of its
 *     splats' T_k alpha_k weighted by their bilinear weights (App. A.6); a
 *     splat that is not blended contributes 0, a culled point has weight 0;
 *   - Eq. 2/3 range over all points drawn from the leaf in the step; a leaf
 *     without points only decays; subdivision replaces a leaf by its 8
 *     children in place (x fastest, then y, then z: Morton order within the
 *     parent) and happens only if the resulting leaf count stays below the
 *     cap; pruning keeps the order of the surviving leaves;
 *   - a leaf is visible unless all 8 corners of its cube lie outside one
 *     plane of the view frustum (near < z < far, 0 <= u < W, 0 <= v < H),
 *     in FP64 camera coordinates with a fixed operation order; d_i uses the
 *     leaf center's view-space z; the level factor 2^(l lambda_l) is exp2;
 *   - a sample is in view when its FP32 position projects (the rasterizer's
 *     FP32 projection) strictly between near and far and into [0, W) x [0, H);
 *     round r of the re-sampling redraws every sample not in view, in place,
 *     with Philox purposes 2 + 2r (leaf) and 3 + 2r (position);
 *   - pre-extraction: the k-th sample of a leaf (k = 0, 1, ...) sits at
 *     c + (h - 1/2) * edge with h the Halton point of index k + 1 in bases
 *     (2, 3, 5) (index 0 would be the cube's corner); each radical inverse
 *     is an exact fraction n / b^m divided once in FP64;
 *   - contraction (mip-NeRF 360): y = (x - center) / radius, contract(y) = y
 *     for |y| <= 1, else (2 - 1/|y|) y / |y|; query position contract(y)/4 +
 *     1/2 in [0, 1]^3.  Evaluated in FP32 with a fixed operation order on both
 *     sides, since it decides the grid cells;
 *   - SH head: direction d = (x - camera center) / |x - camera center|; real
 *     orthonormal SH of degree 2, Y_0 = sqrt(1/(4 pi)); Y_1..3 = sqrt(3/(4 pi))
 *     (y, z, x); Y_4..8 = sqrt(15/(4 pi)) xy, sqrt(15/(4 pi)) yz,
 *     sqrt(5/(16 pi)) (3 z^2 - 1), sqrt(15/(4 pi)) xz, sqrt(15/(16 pi))
 *     (x^2 - y^2); color channel c = sum_k Y_k(d) h[1 + 9 c + k].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_ARG -1
#define ORACLE_ERR_WEIGHTS -2
#define ORACLE_ERR_NOMEM -3

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,       */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).  One round maps   */
/* the 4-word counter through two 32x32->64 multiplications whose high      */
/* halves are xored with the other two words and the round key; the key is  */
/* advanced by the Weyl constants between rounds.                           */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_MUL_A = 0xD2511F53u;
static const uint32_t PHILOX_MUL_B = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL_A = 0x9E3779B9u;
static const uint32_t PHILOX_WEYL_B = 0xBB67AE85u;

void oracle_philox4x32_10(const uint32_t key_in[2], const uint32_t ctr_in[4], uint32_t out[4]) {
  uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_WEYL_A;
      k1 += PHILOX_WEYL_B;
    }
    uint64_t pa = (uint64_t)PHILOX_MUL_A * (uint64_t)x0;
    uint64_t pb = (uint64_t)PHILOX_MUL_B * (uint64_t)x2;
    uint32_t pa_hi = (uint32_t)(pa >> 32), pa_lo = (uint32_t)pa;
    uint32_t pb_hi = (uint32_t)(pb >> 32), pb_lo = (uint32_t)pb;
    uint32_t y0 = pb_hi ^ x1 ^ k0;
    uint32_t y1 = pb_lo;
    uint32_t y2 = pa_hi ^ x3 ^ k1;
    uint32_t y3 = pa_lo;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Bulk form for statistical tests: out[4*i..] = Philox(key, (i + ctr0, ctr1, ctr2, ctr3)). */
void oracle_philox_stream(uint64_t seed, uint32_t ctr1, uint32_t ctr2, uint32_t ctr3,
                          int64_t n, uint32_t* out) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t i = 0; i < n; ++i) {
    uint32_t ctr[4] = {(uint32_t)i, ctr1, ctr2, ctr3};
    oracle_philox4x32_10(key, ctr, out + 4 * i);
  }
}

/* ------------------------------------------------------------------------ */
/* Sampling (Sec. 3.2): multinomial sampling with replacement over leaves,  */
/* then a uniform position inside the chosen leaf.                          */
/* ------------------------------------------------------------------------ */

/* Quantised weights and their inclusive prefix sum.  Returns Q (the total)
 * through *total.  Errors: negative, NaN or infinite weight, or no positive
 * weight. */
int oracle_build_cdf(const double* w, int64_t n_leaves, double* cdf, double* total) {
  if (n_leaves <= 0 || n_leaves > (1ll << 24)) return ORACLE_ERR_ARG;
  double wmax = 0.0;
  for (int64_t i = 0; i < n_leaves; ++i) {
    if (!(w[i] >= 0.0) || isinf(w[i])) return ORACLE_ERR_WEIGHTS;
    if (w[i] > wmax) wmax = w[i];
  }
  if (!(wmax > 0.0)) return ORACLE_ERR_WEIGHTS;
  double run = 0.0;
  for (int64_t i = 0; i < n_leaves; ++i) {
    double q = rint(ldexp(w[i] / wmax, 29));
    run += q; /* exact: every partial sum is an integer below 2^53 */
    cdf[i] = run;
  }
  *total = run;
  return ORACLE_OK;
}

/* Smallest i with cdf[i] > r (cdf non-decreasing, r < cdf[n-1]). */
int64_t oracle_search_cdf(const double* cdf, int64_t n_leaves, double r) {
  int64_t lo = 0, hi = n_leaves - 1;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (cdf[mid] > r) hi = mid; else lo = mid + 1;
  }
  return lo;
}

/* r = floor(b * Q / 2^53) for a 53-bit b, in exact 128-bit integer arithmetic. */
uint64_t oracle_scale_draw(uint64_t b53, uint64_t Q) {
  unsigned __int128 p = (unsigned __int128)b53 * (unsigned __int128)Q;
  return (uint64_t)(p >> 53);
}

/* Leaf of draw s: smallest i with cdf_i > floor(b * Q / 2^53), b the low 53
 * bits of Philox(key = seed, counter = (s lo, s hi, view, 0)) words 1:0. */
static int64_t draw_leaf(const uint32_t key[2], const double* cdf, int64_t n_leaves, uint64_t Q,
                         int64_t s, uint32_t view_id) {
  uint32_t ctr[4] = {(uint32_t)s, (uint32_t)((uint64_t)s >> 32), view_id, 0u};
  uint32_t r4[4];
  oracle_philox4x32_10(key, ctr, r4);
  uint64_t b = ((uint64_t)(r4[1] & 0x1FFFFFu) << 32) | (uint64_t)r4[0];
  uint64_t r = oracle_scale_draw(b, Q);
  return oracle_search_cdf(cdf, n_leaves, (double)r);
}

/* Per-draw leaf indices in draw order (exposed for tests). */
int oracle_draw_leaves(const double* weights, int64_t n_leaves, uint64_t seed, uint32_t view_id,
                       int64_t n_samples, int32_t* leaf_of_draw) {
  double* cdf = (double*)malloc(sizeof(double) * (size_t)(n_leaves > 0 ? n_leaves : 1));
  if (!cdf) return ORACLE_ERR_NOMEM;
  double Qd = 0.0;
  int st = oracle_build_cdf(weights, n_leaves, cdf, &Qd);
  if (st != ORACLE_OK) { free(cdf); return st; }
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < n_samples; ++s)
    leaf_of_draw[s] = (int32_t)draw_leaf(key, cdf, n_leaves, (uint64_t)Qd, s, view_id);
  free(cdf);
  return ORACLE_OK;
}

/* Full sampling step (Sec. 3.2): N draws with replacement give the per-leaf
 * counts; the list of leaf indices is emitted in ascending leaf order (leaf
 * i occupies slots start_i .. start_i + count_i - 1), and the sample in slot
 * k gets the uniform position c + (u - 1/2) * root_size * 2^-l with
 * u_d = (word_d >> 8) * 2^-24 from Philox(counter = (k lo, k hi, view, 1)).
 * pos_out is FP64 and exact (u is a 24-bit dyadic fraction).
 * counts_out (optional) receives count_i per leaf. */
int oracle_sample_octree(const float* centers, const int32_t* levels, const double* weights,
                         int64_t n_leaves, double root_size, uint64_t seed, uint32_t view_id,
                         int64_t n_samples, int32_t* leaf_out, double* pos_out, int64_t* counts_out) {
  if (n_samples < 0) return ORACLE_ERR_ARG;
  int32_t* draws = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_samples > 0 ? n_samples : 1));
  int64_t* count = (int64_t*)calloc((size_t)(n_leaves > 0 ? n_leaves : 1), sizeof(int64_t));
  if (!draws || !count) { free(draws); free(count); return ORACLE_ERR_NOMEM; }
  int st = oracle_draw_leaves(weights, n_leaves, seed, view_id, n_samples, draws);
  if (st != ORACLE_OK) { free(draws); free(count); return st; }
  for (int64_t s = 0; s < n_samples; ++s) count[draws[s]]++;
  free(draws);
  int64_t k = 0;
  for (int64_t i = 0; i < n_leaves; ++i)
    for (int64_t c = 0; c < count[i]; ++c) leaf_out[k++] = (int32_t)i;
  if (counts_out) for (int64_t i = 0; i < n_leaves; ++i) counts_out[i] = count[i];
  free(count);
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
  for (int64_t slot = 0; slot < n_samples; ++slot) {
    int64_t leaf = leaf_out[slot];
    uint32_t ctr[4] = {(uint32_t)slot, (uint32_t)((uint64_t)slot >> 32), view_id, 1u};
    uint32_t r4[4];
    oracle_philox4x32_10(key, ctr, r4);
    double edge = ldexp(root_size, -levels[leaf]);
    for (int d = 0; d < 3; ++d) {
      double u = ldexp((double)(r4[d] >> 8), -24);
      pos_out[3 * slot + d] = (double)centers[3 * leaf + d] + (u - 0.5) * edge;
    }
  }
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Multi-resolution hash grid (Sec. 3.3, App. A.5 / Listing 1).             */
/* ------------------------------------------------------------------------ */

static int level_is_dense(int64_t res, int64_t T) {
  int64_t side = res + 1;
  return side * side * side <= T;
}

static int64_t level_entries(int64_t res, int64_t T) {
  int64_t side = res + 1;
  int64_t dense = side * side * side;
  return dense <= T ? dense : T;
}

/* Table rows per level and their level-major offsets; returns the total.
 * Storage layout (not fixed by the paper): each level starts on a multiple
 * of 16 rows and the total is rounded up to 16; padding rows are unused. */
int64_t oracle_hash_layout(int32_t n_levels, const int32_t* res, int32_t log2_T, int64_t* offsets) {
  int64_t T = 1ll << log2_T;
  int64_t off = 0;
  for (int l = 0; l < n_levels; ++l) {
    off = (off + 15) / 16 * 16;
    if (offsets) offsets[l] = off;
    off += level_entries(res[l], T);
  }
  return (off + 15) / 16 * 16;
}

/* Row of the table (within its level) that holds grid vertex (vx, vy, vz). */
int64_t oracle_hash_vertex_index(int64_t res, int32_t log2_T, int64_t vx, int64_t vy, int64_t vz) {
  int64_t T = 1ll << log2_T;
  if (level_is_dense(res, T)) {
    int64_t side = res + 1;
    return vx + vy * side + vz * side * side;
  }
  uint32_t h = ((uint32_t)vx * 1u) ^ ((uint32_t)vy * 2654435761u) ^ ((uint32_t)vz * 805459861u);
  return (int64_t)(h & (uint32_t)(T - 1));
}

/* Cell and fractional offset of coordinate x on a level of resolution res:
 * x is clamped to [0,1]; cell = min(floor(x*res), res-1); frac = x*res - cell. */
static void grid_cell(double x, int64_t res, int64_t* cell, double* frac) {
  if (!(x >= 0.0)) x = 0.0; /* also maps NaN to 0 */
  if (x > 1.0) x = 1.0;
  double s = x * (double)res;
  double c = floor(s);
  if (c > (double)(res - 1)) c = (double)(res - 1);
  *cell = (int64_t)c;
  *frac = s - c;
}

/* h[n, l*F + f] = sum over the 8 cell corners of trilinear weight * table[row, f];
 * abs_out (optional) receives the sum of absolute terms. */
int oracle_hash_fwd(int32_t n_levels, const int32_t* res, int32_t log2_T, int32_t n_feats,
                    const double* table, const double* pos, int64_t n, double* h_out, double* abs_out) {
  int64_t* offsets = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_levels);
  if (!offsets) return ORACLE_ERR_NOMEM;
  oracle_hash_layout(n_levels, res, log2_T, offsets);
  int64_t C = (int64_t)n_levels * n_feats;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p) {
    for (int l = 0; l < n_levels; ++l) {
      int64_t cell[3];
      double fr[3];
      for (int d = 0; d < 3; ++d) grid_cell(pos[3 * p + d], res[l], &cell[d], &fr[d]);
      for (int f = 0; f < n_feats; ++f) h_out[p * C + l * n_feats + f] = 0.0;
      if (abs_out) for (int f = 0; f < n_feats; ++f) abs_out[p * C + l * n_feats + f] = 0.0;
      for (int corner = 0; corner < 8; ++corner) {
        int bx = corner & 1, by = (corner >> 1) & 1, bz = (corner >> 2) & 1;
        double w = (bx ? fr[0] : 1.0 - fr[0]) * (by ? fr[1] : 1.0 - fr[1]) * (bz ? fr[2] : 1.0 - fr[2]);
        int64_t row = offsets[l] + oracle_hash_vertex_index(res[l], log2_T, cell[0] + bx, cell[1] + by, cell[2] + bz);
        for (int f = 0; f < n_feats; ++f) {
          h_out[p * C + l * n_feats + f] += w * table[row * n_feats + f];
          if (abs_out) abs_out[p * C + l * n_feats + f] += fabs(w * table[row * n_feats + f]);
        }
      }
    }
  }
  free(offsets);
  return ORACLE_OK;
}

/* grad_table[row, f] += weight * dh[n, l*F + f]; abs_out (optional) receives
 * the sum of weight * |dh| (or weight * dh_abs, the caller's own absolute-term
 * sums for dh, when given), used as the condition-aware scale. */
int oracle_hash_bwd(int32_t n_levels, const int32_t* res, int32_t log2_T, int32_t n_feats,
                    const double* pos, const double* dh, int64_t n, double* grad_out, double* abs_out,
                    const double* dh_abs) {
  int64_t* offsets = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_levels);
  if (!offsets) return ORACLE_ERR_NOMEM;
  oracle_hash_layout(n_levels, res, log2_T, offsets);
  int64_t C = (int64_t)n_levels * n_feats;
  /* levels own disjoint row ranges, so they can be accumulated independently
   * and in point order (deterministic). */
#pragma omp parallel for schedule(dynamic, 1)
  for (int l = 0; l < n_levels; ++l) {
    for (int64_t p = 0; p < n; ++p) {
      int64_t cell[3];
      double fr[3];
      for (int d = 0; d < 3; ++d) grid_cell(pos[3 * p + d], res[l], &cell[d], &fr[d]);
      for (int corner = 0; corner < 8; ++corner) {
        int bx = corner & 1, by = (corner >> 1) & 1, bz = (corner >> 2) & 1;
        double w = (bx ? fr[0] : 1.0 - fr[0]) * (by ? fr[1] : 1.0 - fr[1]) * (bz ? fr[2] : 1.0 - fr[2]);
        int64_t row = offsets[l] + oracle_hash_vertex_index(res[l], log2_T, cell[0] + bx, cell[1] + by, cell[2] + bz);
        for (int f = 0; f < n_feats; ++f) {
          double term = w * dh[p * C + l * n_feats + f];
          grad_out[row * n_feats + f] += term;
          if (abs_out) abs_out[row * n_feats + f] += w * (dh_abs ? dh_abs[p * C + l * n_feats + f] : fabs(dh[p * C + l * n_feats + f]));
        }
      }
    }
  }
  free(offsets);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Rasterizer (Sec. 3.4, Eq. 1, Eq. 5, Eq. 6, App. A.6, Algorithm 1).        */
/* ------------------------------------------------------------------------ */

typedef struct {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  float near_plane, far_plane;
} oracle_camera;

/* Eq. 5 in FP32 with a fixed operation order:
 *   x_c = fma(R[2], z, fma(R[1], y, fma(R[0], x, t[0])))   (same for y_c, z_c)
 *   u = fma(fx, x_c / z_c, cx),  v = fma(fy, y_c / z_c, cy),  d = z_c.
 * Returns 1 if the point lies strictly between the near and far planes. */
int oracle_project(const oracle_camera* cam, const float* p, float* u, float* v, float* d) {
  float xc = fmaf(cam->R[2], p[2], fmaf(cam->R[1], p[1], fmaf(cam->R[0], p[0], cam->t[0])));
  float yc = fmaf(cam->R[5], p[2], fmaf(cam->R[4], p[1], fmaf(cam->R[3], p[0], cam->t[1])));
  float zc = fmaf(cam->R[8], p[2], fmaf(cam->R[7], p[1], fmaf(cam->R[6], p[0], cam->t[2])));
  *d = zc;
  if (!(zc > cam->near_plane && zc < cam->far_plane)) return 0;
  float qx = xc / zc;
  float qy = yc / zc;
  *u = fmaf(cam->fx, qx, cam->cx);
  *v = fmaf(cam->fy, qy, cam->cy);
  return 1;
}

/* The four bilinear splats of a projected point (Eq. 6): pixel centers at
 * (i + 1/2, j + 1/2); the 2x2 nearest centers are i0 = floor(u - 1/2) + {0,1}
 * and j0 = floor(v - 1/2) + {0,1}; weight (1 - |u - u_i|)(1 - |v - v_j|).
 * Writes pixel columns/rows and weights for the four corners (a + 2b order). */
void oracle_splat_corners(double u, double v, int64_t* pi, int64_t* pj, double* w) {
  double fu = u - 0.5, fv = v - 0.5;
  double i0 = floor(fu), j0 = floor(fv);
  for (int b = 0; b < 2; ++b)
    for (int a = 0; a < 2; ++a) {
      int k = a + 2 * b;
      double uc = i0 + a + 0.5, vc = j0 + b + 0.5;
      pi[k] = (int64_t)i0 + a;
      pj[k] = (int64_t)j0 + b;
      w[k] = (1.0 - fabs(u - uc)) * (1.0 - fabs(v - vc));
    }
}

typedef struct {
  float depth;
  int32_t id;
  int32_t corner;
} frag_rec;

static int frag_cmp(const void* pa, const void* pb) {
  const frag_rec* a = (const frag_rec*)pa;
  const frag_rec* b = (const frag_rec*)pb;
  if (a->depth < b->depth) return -1;
  if (a->depth > b->depth) return 1;
  if (a->id < b->id) return -1;
  if (a->id > b->id) return 1;
  return 0;
}

typedef struct {
  int64_t n_pix;
  int64_t* start;   /* [n_pix + 1] */
  frag_rec* frags;  /* sorted per pixel */
  double* fu;       /* per point projected u, v (FP64 copies of the FP32 values) */
  double* fv;
  int8_t* visible;
} frag_lists;

static void free_lists(frag_lists* L) {
  free(L->start); free(L->frags); free(L->fu); free(L->fv); free(L->visible);
}

/* Algorithm 1, ProjectAndCull + BilinearSplatting + per-pixel depth order. */
static int build_lists(const oracle_camera* cam, const float* pos, int64_t n, frag_lists* L) {
  int64_t W = cam->width, H = cam->height;
  L->n_pix = W * H;
  L->start = (int64_t*)calloc((size_t)(W * H + 1), sizeof(int64_t));
  L->fu = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  L->fv = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  L->visible = (int8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  L->frags = NULL;
  if (!L->start || !L->fu || !L->fv || !L->visible) return ORACLE_ERR_NOMEM;
  int64_t* count = L->start + 1;
  for (int64_t p = 0; p < n; ++p) {
    float u, v, d;
    if (!oracle_project(cam, pos + 3 * p, &u, &v, &d)) continue;
    L->visible[p] = 1;
    L->fu[p] = (double)u;
    L->fv[p] = (double)v;
    if (!(L->fu[p] >= -0.5 && L->fu[p] < (double)W + 0.5 && L->fv[p] >= -0.5 && L->fv[p] < (double)H + 0.5)) {
      L->visible[p] = 0;
      continue;
    }
    int64_t pi[4], pj[4];
    double w[4];
    oracle_splat_corners(L->fu[p], L->fv[p], pi, pj, w);
    for (int k = 0; k < 4; ++k)
      if (pi[k] >= 0 && pi[k] < W && pj[k] >= 0 && pj[k] < H) count[pj[k] * W + pi[k]]++;
  }
  for (int64_t q = 0; q < W * H; ++q) L->start[q + 1] += L->start[q];
  int64_t total = L->start[W * H];
  L->frags = (frag_rec*)malloc(sizeof(frag_rec) * (size_t)(total > 0 ? total : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(W * H > 0 ? W * H : 1));
  if (!L->frags || !fill) { free(fill); return ORACLE_ERR_NOMEM; }
  memcpy(fill, L->start, sizeof(int64_t) * (size_t)(W * H));
  for (int64_t p = 0; p < n; ++p) {
    if (!L->visible[p]) continue;
    float u, v, d;
    oracle_project(cam, pos + 3 * p, &u, &v, &d);
    int64_t pi[4], pj[4];
    double w[4];
    oracle_splat_corners(L->fu[p], L->fv[p], pi, pj, w);
    for (int k = 0; k < 4; ++k)
      if (pi[k] >= 0 && pi[k] < W && pj[k] >= 0 && pj[k] < H) {
        frag_rec r = {d, (int32_t)p, k};
        L->frags[fill[pj[k] * W + pi[k]]++] = r;
      }
  }
  free(fill);
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t q = 0; q < W * H; ++q) {
    int64_t m = L->start[q + 1] - L->start[q];
    if (m > 1) qsort(L->frags + L->start[q], (size_t)m, sizeof(frag_rec), frag_cmp);
  }
  return ORACLE_OK;
}

typedef struct {
  int32_t opacity_from_ch0; /* 0: opacity given per point; 1: alpha_h = 1 - exp(-exp(feat[:,0])) */
  int32_t n_channels;
  double t_min;
  double alpha_max;
  double ambiguity_rel;     /* relative band around t_min flagged as ambiguous */
} oracle_raster_opts;

/* Point opacity alpha_h (Sec. 3.3 activation in head mode). */
static double point_alpha(const oracle_raster_opts* o, const double* opacity, const double* feat, int64_t p) {
  if (o->opacity_from_ch0) return 1.0 - exp(-exp(feat[p * o->n_channels]));
  return opacity[p];
}

/* Blended color vector of a point: its features, with channel 0 replaced
 * by 1 in head mode (so image channel 0 carries the accumulated alpha). */
static double point_color(const oracle_raster_opts* o, const double* feat, int64_t p, int c) {
  if (o->opacity_from_ch0 && c == 0) return 1.0;
  return feat[p * o->n_channels + c];
}

/* Magnitude of a blended color channel for the condition-aware tolerance:
 * |c|, or feat_abs (the caller's own sum of absolute terms that produced the
 * feature, e.g. the grid query's sum |w t|) when given; 1 for the constant
 * channel 0 in head mode. */
static double color_scale(const oracle_raster_opts* o, const double* feat, const double* feat_abs, int64_t p, int c) {
  if (o->opacity_from_ch0 && c == 0) return 1.0;
  if (feat_abs) return feat_abs[p * o->n_channels + c];
  return fabs(feat[p * o->n_channels + c]);
}

/* Forward: image[H,W,F], T_final[H,W], n_contrib[H,W], n_frags[H,W] (all
 * fragments of the pixel), flags[H,W] bit 0 = stopping decision within the
 * ambiguity band of t_min; abs_out[H,W,F] (optional) = sum T alpha |c|
 * (|c| from feat_abs when given). */
int oracle_raster_fwd(const oracle_camera* cam, const oracle_raster_opts* o, const float* pos,
                      const double* opacity, const double* feat, int64_t n,
                      double* image, double* T_final, int32_t* n_contrib, int32_t* n_frags,
                      uint8_t* flags, double* abs_out, const double* feat_abs) {
  frag_lists L;
  int st = build_lists(cam, pos, n, &L);
  if (st != ORACLE_OK) { free_lists(&L); return st; }
  int F = o->n_channels;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t q = 0; q < L.n_pix; ++q) {
    double* C = image + q * F;
    for (int c = 0; c < F; ++c) C[c] = 0.0;
    if (abs_out) for (int c = 0; c < F; ++c) abs_out[q * F + c] = 0.0;
    double T = 1.0;
    int32_t cnt = 0;
    uint8_t flag = 0;
    double band = o->ambiguity_rel * o->t_min;
    for (int64_t k = L.start[q]; k < L.start[q + 1]; ++k) {
      const frag_rec* r = &L.frags[k];
      int64_t pi[4], pj[4];
      double w[4];
      oracle_splat_corners(L.fu[r->id], L.fv[r->id], pi, pj, w);
      double a = point_alpha(o, opacity, feat, r->id) * w[r->corner];
      if (a > o->alpha_max) a = o->alpha_max;
      for (int c = 0; c < F; ++c) {
        double term = T * a * point_color(o, feat, r->id, c);
        C[c] += term;
        if (abs_out) abs_out[q * F + c] += T * a * color_scale(o, feat, feat_abs, r->id, c);
      }
      double Tn = T * (1.0 - a);
      ++cnt;
      if (fabs(Tn - o->t_min) <= band) flag |= 1;
      T = Tn;
      if (T < o->t_min) break;
    }
    T_final[q] = T;
    n_contrib[q] = cnt;
    if (n_frags) n_frags[q] = (int32_t)(L.start[q + 1] - L.start[q]);
    if (flags) flags[q] = flag;
  }
  free_lists(&L);
  return ORACLE_OK;
}

/* Backward of oracle_raster_fwd for upstream gradient d_image[H,W,F].
 * Per pixel with blended fragments k = 0..n-1, T_k = prod_{i<k} (1 - alpha_i):
 *   dL/dc_k     = T_k alpha_k g
 *   dL/dalpha_k = T_k (c_k . g) - sum_{j>k} [prod_{i<j, i!=k} (1 - alpha_i)] alpha_j (c_j . g)
 * (the second form is the derivative of T_j with respect to alpha_k written
 * without division).  Per point: d_feat = sum of its dL/dc_k; d_alpha_h =
 * sum of w_k dL/dalpha_k over unclamped splats; in head mode d_feat[:,0] =
 * d_alpha_h * exp(h0) * exp(-exp(h0)) and channel 0 of dL/dc is dropped.
 * d_opacity (given mode) and d_feat are written (not accumulated);
 * abs_feat (optional) receives sum |terms| of d_feat for the tolerance. */
int oracle_raster_bwd(const oracle_camera* cam, const oracle_raster_opts* o, const float* pos,
                      const double* opacity, const double* feat, int64_t n, const double* d_image,
                      double* d_opacity, double* d_feat, double* abs_feat, double* abs_opacity,
                      const double* feat_abs) {
  frag_lists L;
  int st = build_lists(cam, pos, n, &L);
  if (st != ORACLE_OK) { free_lists(&L); return st; }
  int F = o->n_channels;
  int64_t total = L.start[L.n_pix];
  /* per-fragment scalars: a_k = T_k alpha_k, da_k = dL/dalpha_k, used flag */
  double* fa = (double*)calloc((size_t)(total > 0 ? total : 1), sizeof(double));
  double* fda = (double*)calloc((size_t)(total > 0 ? total : 1), sizeof(double));
  double* fdaabs = (double*)calloc((size_t)(total > 0 ? total : 1), sizeof(double));
  if (!fa || !fda || !fdaabs) { free(fa); free(fda); free(fdaabs); free_lists(&L); return ORACLE_ERR_NOMEM; }
#pragma omp parallel
  {
    int64_t cap = 64;
    double* al = (double*)malloc(sizeof(double) * (size_t)cap);
    double* dot = (double*)malloc(sizeof(double) * (size_t)cap);
    double* dotabs = (double*)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 256)
    for (int64_t q = 0; q < L.n_pix; ++q) {
      int64_t b0 = L.start[q], m = L.start[q + 1] - L.start[q];
      if (m == 0) continue;
      if (m > cap) {
        cap = m;
        al = (double*)realloc(al, sizeof(double) * (size_t)cap);
        dot = (double*)realloc(dot, sizeof(double) * (size_t)cap);
        dotabs = (double*)realloc(dotabs, sizeof(double) * (size_t)cap);
      }
      const double* g = d_image + q * F;
      /* forward replay to find the blended prefix */
      double T = 1.0;
      int64_t nb = 0;
      for (int64_t k = 0; k < m; ++k) {
        const frag_rec* r = &L.frags[b0 + k];
        int64_t pi[4], pj[4];
        double w[4];
        oracle_splat_corners(L.fu[r->id], L.fv[r->id], pi, pj, w);
        double a = point_alpha(o, opacity, feat, r->id) * w[r->corner];
        if (a > o->alpha_max) a = o->alpha_max;
        al[k] = a;
        double s = 0.0, sa = 0.0;
        for (int c = 0; c < F; ++c) {
          s += point_color(o, feat, r->id, c) * g[c];
          sa += color_scale(o, feat, feat_abs, r->id, c) * fabs(g[c]);
        }
        dot[k] = s;
        dotabs[k] = sa;
        ++nb;
        T = T * (1.0 - a);
        if (T < o->t_min) break;
      }
      for (int64_t k = 0; k < nb; ++k) {
        double Tk = 1.0;
        for (int64_t i = 0; i < k; ++i) Tk *= (1.0 - al[i]);
        double da = Tk * dot[k];
        double daabs = Tk * dotabs[k];
        /* prod = prod_{i<j, i!=k} (1 - alpha_i), grown one factor per j */
        double prod = Tk;
        for (int64_t j = k + 1; j < nb; ++j) {
          da -= prod * al[j] * dot[j];
          daabs += prod * al[j] * dotabs[j];
          prod *= (1.0 - al[j]);
        }
        fa[b0 + k] = Tk * al[k];
        fda[b0 + k] = da;
        fdaabs[b0 + k] = daabs;
      }
    }
    free(al);
    free(dot);
    free(dotabs);
  }
  /* per-point accumulation, serial and in (pixel, depth) order */
  double* dah = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* dahabs = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (!dah || !dahabs) { free(dah); free(dahabs); free(fa); free(fda); free(fdaabs); free_lists(&L); return ORACLE_ERR_NOMEM; }
  for (int64_t p = 0; p < n * F; ++p) d_feat[p] = 0.0;
  if (abs_feat) for (int64_t p = 0; p < n * F; ++p) abs_feat[p] = 0.0;
  for (int64_t q = 0; q < L.n_pix; ++q) {
    const double* g = d_image + q * F;
    for (int64_t k = L.start[q]; k < L.start[q + 1]; ++k) {
      const frag_rec* r = &L.frags[k];
      if (fa[k] == 0.0 && fda[k] == 0.0) continue;
      for (int c = 0; c < F; ++c) {
        d_feat[(int64_t)r->id * F + c] += fa[k] * g[c];
        if (abs_feat) abs_feat[(int64_t)r->id * F + c] += fabs(fa[k] * g[c]);
      }
      int64_t pi[4], pj[4];
      double w[4];
      oracle_splat_corners(L.fu[r->id], L.fv[r->id], pi, pj, w);
      double ah = point_alpha(o, opacity, feat, r->id);
      double dadah = (ah * w[r->corner] > o->alpha_max) ? 0.0 : w[r->corner];
      dah[r->id] += dadah * fda[k];
      dahabs[r->id] += fabs(dadah) * fdaabs[k];
    }
  }
  for (int64_t p = 0; p < n; ++p) {
    if (o->opacity_from_ch0) {
      double h0 = feat[p * F];
      double dh0 = exp(h0) * exp(-exp(h0));
      d_feat[p * F] = dah[p] * dh0;
      if (abs_feat) abs_feat[p * F] = dahabs[p] * dh0;
    } else {
      if (d_opacity) d_opacity[p] = dah[p];
      if (abs_opacity) abs_opacity[p] = dahabs[p];
    }
  }
  free(dah); free(dahabs); free(fa); free(fda); free(fdaabs);
  free_lists(&L);
  return ORACLE_OK;
}

/* Per-pixel sorted fragment lists, exposed for tests: writes the number of
 * fragments per pixel (count[H*W]) and, if ids/corners are given, the point
 * ids and corner indices in blending order (size = total). Returns total. */
int64_t oracle_fragment_lists(const oracle_camera* cam, const float* pos, int64_t n,
                              int64_t* count, int32_t* ids, int32_t* corners, float* depths) {
  frag_lists L;
  if (build_lists(cam, pos, n, &L) != ORACLE_OK) { free_lists(&L); return -1; }
  for (int64_t q = 0; q < L.n_pix; ++q) count[q] = L.start[q + 1] - L.start[q];
  int64_t total = L.start[L.n_pix];
  for (int64_t k = 0; k < total; ++k) {
    if (ids) ids[k] = L.frags[k].id;
    if (corners) corners[k] = L.frags[k].corner;
    if (depths) depths[k] = L.frags[k].depth;
  }
  free_lists(&L);
  return total;
}

/* ------------------------------------------------------------ octree ---- */

/* Per-point blending weights for the probability updates (Sec. 3.1 Eq. 2/3
 * use b_j = T_j alpha_j; App. A.6 combines a point's four splat weights by
 * their bilinear weights): b[p] = sum_k w_k T_k alpha_k over the point's
 * blended splats.  pix_sum (optional, [H*W]) = sum over the pixel's blended
 * fragments of T_k alpha_k (which telescopes to 1 - T_final). */
int oracle_point_weights(const oracle_camera* cam, const oracle_raster_opts* o, const float* pos,
                         const double* opacity, const double* feat, int64_t n, double* b, double* pix_sum) {
  frag_lists L;
  int st = build_lists(cam, pos, n, &L);
  if (st != ORACLE_OK) { free_lists(&L); return st; }
  for (int64_t p = 0; p < n; ++p) b[p] = 0.0;
  for (int64_t q = 0; q < L.n_pix; ++q) {
    double T = 1.0, sum = 0.0;
    for (int64_t k = L.start[q]; k < L.start[q + 1]; ++k) {
      const frag_rec* r = &L.frags[k];
      int64_t pi[4], pj[4];
      double w[4];
      oracle_splat_corners(L.fu[r->id], L.fv[r->id], pi, pj, w);
      double a = point_alpha(o, opacity, feat, r->id) * w[r->corner];
      if (a > o->alpha_max) a = o->alpha_max;
      b[r->id] += w[r->corner] * (T * a);
      sum += T * a;
      T = T * (1.0 - a);
      if (T < o->t_min) break;
    }
    if (pix_sum) pix_sum[q] = sum;
  }
  free_lists(&L);
  return ORACLE_OK;
}

/* Eq. 2 and Eq. 3 for one step: for every leaf i, with B_i the weights b of
 * the points drawn from it,
 *   p_i = max(lambda_u p_i, max B_i),  q_i = max(lambda_u q_i, max B_i - min B_i);
 * a leaf with no point only decays.  The b are FP32 values (the
 * rasterizer's output type); max, min and their difference are taken in
 * FP64. */
int oracle_octree_update(const int32_t* leaf_idx, const float* b, int64_t n, double* p, double* q,
                         int64_t n_leaves, double lambda_u) {
  double* bmax = (double*)malloc(sizeof(double) * (size_t)(n_leaves > 0 ? n_leaves : 1));
  double* bmin = (double*)malloc(sizeof(double) * (size_t)(n_leaves > 0 ? n_leaves : 1));
  uint8_t* seen = (uint8_t*)calloc((size_t)(n_leaves > 0 ? n_leaves : 1), 1);
  if (!bmax || !bmin || !seen) { free(bmax); free(bmin); free(seen); return ORACLE_ERR_NOMEM; }
  for (int64_t j = 0; j < n; ++j) {
    int64_t i = leaf_idx[j];
    if (i < 0 || i >= n_leaves) { free(bmax); free(bmin); free(seen); return ORACLE_ERR_ARG; }
    double v = (double)b[j];
    if (!seen[i]) { bmax[i] = v; bmin[i] = v; seen[i] = 1; }
    else {
      if (v > bmax[i]) bmax[i] = v;
      if (v < bmin[i]) bmin[i] = v;
    }
  }
  for (int64_t i = 0; i < n_leaves; ++i) {
    double dp = lambda_u * p[i], dq = lambda_u * q[i];
    if (seen[i]) {
      double spread = bmax[i] - bmin[i];
      p[i] = bmax[i] > dp ? bmax[i] : dp;
      q[i] = spread > dq ? spread : dq;
    } else {
      p[i] = dp;
      q[i] = dq;
    }
  }
  free(bmax); free(bmin); free(seen);
  return ORACLE_OK;
}

/* Subdivision (Sec. 3.1): every leaf with q_i > tau_s is replaced, in place,
 * by its 8 children (level l + 1, centers c + (d - 1/2) * root * 2^-(l+1)
 * per axis for d in {0, 1}, child k = dx + 2 dy + 4 dz), which inherit p_i
 * and start with q = 0 -- unless the resulting leaf count would reach
 * max_leaves, in which case nothing is subdivided.  Outputs need room for
 * 8 n_leaves entries; returns the new leaf count (negative on error). */
int64_t oracle_octree_subdivide(const float* centers, const int32_t* levels, const double* p, const double* q,
                                int64_t n_leaves, double root_size, double tau_s, int64_t max_leaves,
                                float* centers_out, int32_t* levels_out, double* p_out, double* q_out) {
  int64_t n_split = 0;
  for (int64_t i = 0; i < n_leaves; ++i) if (q[i] > tau_s) ++n_split;
  int split = n_leaves + 7 * n_split < max_leaves;
  int64_t o = 0;
  for (int64_t i = 0; i < n_leaves; ++i) {
    if (!(split && q[i] > tau_s)) {
      for (int d = 0; d < 3; ++d) centers_out[3 * o + d] = centers[3 * i + d];
      levels_out[o] = levels[i];
      p_out[o] = p[i];
      q_out[o] = q[i];
      ++o;
      continue;
    }
    double child = root_size * ldexp(1.0, -(levels[i] + 1));  /* child edge */
    for (int k = 0; k < 8; ++k) {
      int dxyz[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
      for (int d = 0; d < 3; ++d)
        centers_out[3 * o + d] = (float)((double)centers[3 * i + d] + ((double)dxyz[d] - 0.5) * child);
      levels_out[o] = levels[i] + 1;
      p_out[o] = p[i];
      q_out[o] = 0.0;
      ++o;
    }
  }
  return o;
}

/* Pruning (Sec. 3.1): leaves with p_i < tau_p are removed; the others keep
 * their order.  Returns the new leaf count. */
int64_t oracle_octree_prune(const float* centers, const int32_t* levels, const double* p, const double* q,
                            int64_t n_leaves, double tau_p, float* centers_out, int32_t* levels_out,
                            double* p_out, double* q_out) {
  int64_t o = 0;
  for (int64_t i = 0; i < n_leaves; ++i) {
    if (p[i] < tau_p) continue;
    for (int d = 0; d < 3; ++d) centers_out[3 * o + d] = centers[3 * i + d];
    levels_out[o] = levels[i];
    p_out[o] = p[i];
    q_out[o] = q[i];
    ++o;
  }
  return o;
}

/* ------------------------------------------------- view-specific sampling */

/* Camera coordinates of a world point in FP64, evaluated left to right. */
static void cam_space(const oracle_camera* cam, const double x[3], double xc[3]) {
  for (int k = 0; k < 3; ++k)
    xc[k] = (double)cam->R[3 * k] * x[0] + (double)cam->R[3 * k + 1] * x[1] + (double)cam->R[3 * k + 2] * x[2] +
            (double)cam->t[k];
}

/* Frustum culling of a leaf cube (center c, edge e): culled iff all corners
 * are outside one of the six planes. */
static int box_visible(const oracle_camera* cam, const float* c, double e) {
  int out[6] = {1, 1, 1, 1, 1, 1};
  for (int k = 0; k < 8; ++k) {
    double x[3] = {(double)c[0] + ((k & 1) ? 0.5 : -0.5) * e, (double)c[1] + ((k & 2) ? 0.5 : -0.5) * e,
                   (double)c[2] + ((k & 4) ? 0.5 : -0.5) * e};
    double xc[3];
    cam_space(cam, x, xc);
    if (!(xc[2] <= (double)cam->near_plane)) out[0] = 0;
    if (!(xc[2] >= (double)cam->far_plane)) out[1] = 0;
    if (!((double)cam->fx * xc[0] + (double)cam->cx * xc[2] < 0.0)) out[2] = 0;
    if (!((double)cam->fx * xc[0] + ((double)cam->cx - (double)cam->width) * xc[2] >= 0.0)) out[3] = 0;
    if (!((double)cam->fy * xc[1] + (double)cam->cy * xc[2] < 0.0)) out[4] = 0;
    if (!((double)cam->fy * xc[1] + ((double)cam->cy - (double)cam->height) * xc[2] >= 0.0)) out[5] = 0;
  }
  for (int i = 0; i < 6; ++i) if (out[i]) return 0;
  return 1;
}

/* Eq. 4: w_i = 1_visible p_i / (d_i 2^(l_i lambda_l)) with the view depth
 * d_i = max(|z_view - near| / far, tau_d) (App. A.4). */
int oracle_view_weights(const float* centers, const int32_t* levels, const double* p, int64_t n_leaves,
                        double root_size, const oracle_camera* cam, double lambda_l, double tau_d, double* w_out) {
  for (int64_t i = 0; i < n_leaves; ++i) {
    double e = ldexp(root_size, -levels[i]);
    if (!box_visible(cam, centers + 3 * i, e)) { w_out[i] = 0.0; continue; }
    double c[3] = {(double)centers[3 * i], (double)centers[3 * i + 1], (double)centers[3 * i + 2]};
    double xc[3];
    cam_space(cam, c, xc);
    double d = fabs(xc[2] - (double)cam->near_plane) / (double)cam->far_plane;
    if (d < tau_d) d = tau_d;
    w_out[i] = p[i] / (d * exp2((double)levels[i] * lambda_l));
  }
  return ORACLE_OK;
}

/* A sample is in view when the rasterizer's FP32 projection keeps it and it
 * falls inside the image rectangle. */
int oracle_point_in_view(const oracle_camera* cam, const float* p) {
  float u, v, d;
  if (!oracle_project(cam, p, &u, &v, &d)) return 0;
  return u >= 0.0f && u < (float)cam->width && v >= 0.0f && v < (float)cam->height;
}

/* App. A.4 "Ensuring Sample Count": up to max_rounds rounds; in round r every
 * sample j not in view gets a new leaf (draw with Philox counter (j, view,
 * 2 + 2r) over the CDF of w) and a new position (counter (j, view, 3 + 2r)),
 * in place.  n_left receives the number of samples still not in view. */
int oracle_resample_view(const float* centers, const int32_t* levels, const double* w, int64_t n_leaves,
                         double root_size, const oracle_camera* cam, uint64_t seed, uint32_t view_id, int64_t n,
                         int32_t max_rounds, int32_t* leaf, float* pos, int64_t* n_left) {
  double* cdf = (double*)malloc(sizeof(double) * (size_t)(n_leaves > 0 ? n_leaves : 1));
  if (!cdf) return ORACLE_ERR_NOMEM;
  double Qd = 0.0;
  int st = oracle_build_cdf(w, n_leaves, cdf, &Qd);
  if (st != ORACLE_OK) { free(cdf); return st; }
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int32_t r = 0; r < max_rounds; ++r) {
    int64_t redrawn = 0;
    for (int64_t j = 0; j < n; ++j) {
      if (oracle_point_in_view(cam, pos + 3 * j)) continue;
      uint32_t c0[4] = {(uint32_t)j, (uint32_t)((uint64_t)j >> 32), view_id, 2u + 2u * (uint32_t)r};
      uint32_t r4[4];
      oracle_philox4x32_10(key, c0, r4);
      uint64_t b = ((uint64_t)(r4[1] & 0x1FFFFFu) << 32) | (uint64_t)r4[0];
      int64_t i = oracle_search_cdf(cdf, n_leaves, (double)oracle_scale_draw(b, (uint64_t)Qd));
      uint32_t c1[4] = {(uint32_t)j, (uint32_t)((uint64_t)j >> 32), view_id, 3u + 2u * (uint32_t)r};
      oracle_philox4x32_10(key, c1, r4);
      double edge = ldexp(root_size, -levels[i]);
      for (int d = 0; d < 3; ++d)
        pos[3 * j + d] = (float)((double)centers[3 * i + d] + (ldexp((double)(r4[d] >> 8), -24) - 0.5) * edge);
      leaf[j] = (int32_t)i;
      ++redrawn;
    }
    if (redrawn == 0) break;
  }
  int64_t left = 0;
  for (int64_t j = 0; j < n; ++j) left += !oracle_point_in_view(cam, pos + 3 * j);
  *n_left = left;
  free(cdf);
  return ORACLE_OK;
}

/* ------------------------------------------------------ pre-extraction --- */

/* Eq. 4 without the visibility indicator and the depth: w_i = p_i / 2^(l_i lambda_l). */
int oracle_level_weights(const int32_t* levels, const double* p, int64_t n_leaves, double lambda_l, double* w_out) {
  for (int64_t i = 0; i < n_leaves; ++i) w_out[i] = p[i] / exp2((double)levels[i] * lambda_l);
  return ORACLE_OK;
}

/* Radical inverse of i in base b (the van der Corput sequence): the digits
 * of i mirrored behind the radix point, as the exact fraction num / b^m,
 * divided once. */
double oracle_radical_inverse(uint32_t b, uint64_t i) {
  uint64_t num = 0, den = 1;
  while (i > 0) {
    num = num * b + i % b;
    den *= b;
    i /= b;
  }
  return (double)num / (double)den;
}

/* Viewpoint-independent pre-extraction: the per-leaf counts of N draws with
 * replacement from w (the same draws as oracle_sample_octree: Philox purpose
 * 0), leaf-grouped output, and Halton positions (see the readings above),
 * rounded once from FP64 to FP32. */
int oracle_sample_halton(const float* centers, const int32_t* levels, const double* w, int64_t n_leaves,
                         double root_size, uint64_t seed, int64_t n_samples, int32_t* leaf_out, float* pos_out) {
  int64_t* counts = (int64_t*)calloc((size_t)(n_leaves > 0 ? n_leaves : 1), sizeof(int64_t));
  double* dummy = (double*)malloc(sizeof(double) * 3 * (size_t)(n_samples > 0 ? n_samples : 1));
  if (!counts || !dummy) { free(counts); free(dummy); return ORACLE_ERR_NOMEM; }
  int st = oracle_sample_octree(centers, levels, w, n_leaves, root_size, seed, 0u, n_samples, leaf_out, dummy,
                                counts);
  free(dummy);
  if (st != ORACLE_OK) { free(counts); return st; }
  int64_t slot = 0;
  const uint32_t bases[3] = {2u, 3u, 5u};
  for (int64_t i = 0; i < n_leaves; ++i) {
    double edge = ldexp(root_size, -levels[i]);
    for (int64_t k = 0; k < counts[i]; ++k, ++slot)
      for (int d = 0; d < 3; ++d)
        pos_out[3 * slot + d] =
            (float)((double)centers[3 * i + d] + (oracle_radical_inverse(bases[d], (uint64_t)k + 1) - 0.5) * edge);
  }
  free(counts);
  return ORACLE_OK;
}

/* --------------------------------------------------------------- SH head --- */

/* Spherical contraction (mip-NeRF 360) in FP32, fixed order:
 * y = (x - center) / radius; r = sqrt(fma(y2, y2, fma(y1, y1, y0 * y0)));
 * s = r <= 1 ? 1 : (2 - 1 / r) / r; q = fma(y * s, 1/4, 1/2). */
int oracle_contract(const float* pos, int64_t n, const float* center, float radius, float* out) {
  for (int64_t p = 0; p < n; ++p) {
    float y[3];
    for (int d = 0; d < 3; ++d) y[d] = (pos[3 * p + d] - center[d]) / radius;
    float r = sqrtf(fmaf(y[2], y[2], fmaf(y[1], y[1], y[0] * y[0])));
    float sc = 1.0f;
    if (r > 1.0f) sc = (2.0f - 1.0f / r) / r;
    for (int d = 0; d < 3; ++d) out[3 * p + d] = fmaf(y[d] * sc, 0.25f, 0.5f);
  }
  return ORACLE_OK;
}

/* The 9 real orthonormal SH of degree <= 2 at the unit vector d. */
void oracle_sh_basis(const double* d, double* Y) {
  const double pi = acos(-1.0);
  double x = d[0], y = d[1], z = d[2];
  Y[0] = sqrt(1.0 / (4.0 * pi));
  double c1 = sqrt(3.0 / (4.0 * pi));
  Y[1] = c1 * y;
  Y[2] = c1 * z;
  Y[3] = c1 * x;
  double c2 = sqrt(15.0 / (4.0 * pi));
  Y[4] = c2 * x * y;
  Y[5] = c2 * y * z;
  Y[6] = sqrt(5.0 / (16.0 * pi)) * (3.0 * z * z - 1.0);
  Y[7] = c2 * x * z;
  Y[8] = sqrt(15.0 / (16.0 * pi)) * (x * x - y * y);
}

/* Absolute-term version of the basis for the condition-aware tolerance:
 * every polynomial with its terms taken in absolute value (3z^2 + 1,
 * x^2 + y^2), so that cancellation inside a basis function is covered. */
static void sh_basis_abs(const double* d, double* Y) {
  const double pi = acos(-1.0);
  double x = fabs(d[0]), y = fabs(d[1]), z = fabs(d[2]);
  Y[0] = sqrt(1.0 / (4.0 * pi));
  double c1 = sqrt(3.0 / (4.0 * pi));
  Y[1] = c1 * y;
  Y[2] = c1 * z;
  Y[3] = c1 * x;
  double c2 = sqrt(15.0 / (4.0 * pi));
  Y[4] = c2 * x * y;
  Y[5] = c2 * y * z;
  Y[6] = sqrt(5.0 / (16.0 * pi)) * (3.0 * z * z + 1.0);
  Y[7] = c2 * x * z;
  Y[8] = sqrt(15.0 / (16.0 * pi)) * (x * x + y * y);
}

static void view_dir(const oracle_camera* cam, const float* p, double* d) {
  /* camera center o = -R^T t */
  double o[3];
  for (int k = 0; k < 3; ++k)
    o[k] = -((double)cam->R[k] * cam->t[0] + (double)cam->R[3 + k] * cam->t[1] + (double)cam->R[6 + k] * cam->t[2]);
  double v[3] = {(double)p[0] - o[0], (double)p[1] - o[1], (double)p[2] - o[2]};
  double len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int k = 0; k < 3; ++k) d[k] = len > 0.0 ? v[k] / len : (k == 2 ? 1.0 : 0.0);
}

/* Head forward (Sec. 3.3): alpha = 1 - exp(-exp(h0)); color_c = sum_k Y_k h[1 + 9c + k]
 * (c < 4); abs_out (optional) = sum_k |Y|_k |h[1 + 9c + k]| with the
 * absolute-term basis |Y| (see sh_basis_abs).  h is [n, F], F >= 37. */
int oracle_sh_head_fwd(const oracle_camera* cam, const float* pos, const double* h, int64_t n, int32_t F,
                       double* alpha, double* color, double* abs_out) {
  if (F < 37) return ORACLE_ERR_ARG;
  for (int64_t p = 0; p < n; ++p) {
    double d[3], Y[9], Ya[9];
    view_dir(cam, pos + 3 * p, d);
    oracle_sh_basis(d, Y);
    sh_basis_abs(d, Ya);
    alpha[p] = 1.0 - exp(-exp(h[p * F]));
    for (int c = 0; c < 4; ++c) {
      double s = 0.0, a = 0.0;
      for (int k = 0; k < 9; ++k) {
        s += Y[k] * h[p * F + 1 + 9 * c + k];
        a += Ya[k] * fabs(h[p * F + 1 + 9 * c + k]);
      }
      color[4 * p + c] = s;
      if (abs_out) abs_out[4 * p + c] = a;
    }
  }
  return ORACLE_OK;
}

/* Head backward: dh[0] = d_alpha exp(h0) exp(-exp(h0)); dh[1 + 9c + k] =
 * Y_k d_color_c; every other channel 0.  abs_out (optional): |dh[0]| and
 * |Y|_k |d_color_c|. */
int oracle_sh_head_bwd(const oracle_camera* cam, const float* pos, const double* h, int64_t n, int32_t F,
                       const double* d_alpha, const double* d_color, double* dh, double* abs_out) {
  if (F < 37) return ORACLE_ERR_ARG;
  for (int64_t p = 0; p < n; ++p) {
    double d[3], Y[9], Ya[9];
    view_dir(cam, pos + 3 * p, d);
    oracle_sh_basis(d, Y);
    sh_basis_abs(d, Ya);
    for (int f = 0; f < F; ++f) dh[p * F + f] = 0.0;
    double e = exp(h[p * F]);
    dh[p * F] = d_alpha[p] * e * exp(-e);
    for (int c = 0; c < 4; ++c)
      for (int k = 0; k < 9; ++k) dh[p * F + 1 + 9 * c + k] = Y[k] * d_color[4 * p + c];
    if (abs_out) {
      for (int f = 0; f < F; ++f) abs_out[p * F + f] = 0.0;
      abs_out[p * F] = fabs(dh[p * F]);
      for (int c = 0; c < 4; ++c)
        for (int k = 0; k < 9; ++k) abs_out[p * F + 1 + 9 * c + k] = Ya[k] * fabs(d_color[4 * p + c]);
    }
  }
  return ORACLE_OK;
}
