/*
 * ddgs_oracle.h -- plain CPU oracle for DDGS-CT DRR splatting.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may include, link or
 * call this code: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it. It shares no code, header or constant table with the
 * CUDA library.
 *
 * Two parts:
 *   1. An FP64 renderer (render_f64.c): Eq. 1 of the paper evaluated for every
 *      Gaussian at every requested pixel, with no tiling, plus the analytic
 *      FP64 gradient of Eq. 1 / Eq. 3 with respect to every Gaussian
 *      parameter, the shared bases and the per-view pose.
 *   2. An FP32 binning reference (binning_f32.c): the integer decisions of the
 *      tiled renderer (culling, screen rectangle, tiles touched, depth key,
 *      stable depth order per tile) taken in IEEE single precision with one
 *      fixed operation order, so that a GPU implementation of the same
 *      definition can be compared with it bit for bit.
 *
 * Conventions (shared with the library by definition, not by code):
 *   Gaussians  [0, n_iso) are isotropic (Eq. 3, c = sigmoid(b_iso . f)),
 *              [n_iso, n) are direction-dependent
 *              (Eq. 3, c = sigmoid(Y_1..L(d) . B_dir f)).
 *   Variants   (ablations of Sec. 4.4 / Table 3 and the ray-angle reading of
 *              Eq. 3): "entangled" gives every Gaussian both terms,
 *              c = sigmoid(b_iso . f + Y(d) . B_dir f) ("direct-entangled",
 *              co-located as in usual spherical-harmonic splatting);
 *              "per_pixel" takes d as the direction of the pixel's own ray
 *              (source to pixel centre) instead of source to the Gaussian's
 *              mean, so c varies across the Gaussian's footprint.
 *   Pose       world -> camera rigid transform [R | t], 3x4 row-major. The
 *              X-ray source sits at the camera origin; the detector plane is
 *              z = sdd; pixel (row i, col j) has centre (j + 1/2, i + 1/2).
 *   Detector   per view: sdd, pitch_u, pitch_v, off_u, off_v; focal lengths
 *              f_u = sdd / pitch_u, f_v = sdd / pitch_v; principal point
 *              (W/2 + off_u, H/2 + off_v).
 */
#ifndef DDGS_ORACLE_H
#define DDGS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------- FP64 renderer ---------------- */

typedef struct {
  int32_t n, n_iso, k, L;        /* k <= 64 features; degree 1 <= L <= 4, k_L = L(L+2) */
  const double *means;           /* [n][3] */
  const double *log_scales;      /* [n][3] */
  const double *quats;           /* [n][4] (w, x, y, z), any non-zero norm */
  const double *opacity_logits;  /* [n] */
  const double *feat;            /* [n][k]; row i is f_iso if i < n_iso else f_dir */
  const double *b_iso;           /* [k] */
  const double *B_dir;           /* [k_L][k] row-major, rows ordered (l, m = -l..l) */
  int32_t entangled;             /* 1: every Gaussian carries both terms of Eq. 3 */
  int32_t per_pixel;             /* 1: d is the pixel's ray direction */
} or_scene;

typedef struct {
  int32_t n_views, height, width;
  const double *world_to_cam;    /* [V][3][4] */
  const double *detector;        /* [V][5]: sdd, pitch_u, pitch_v, off_u, off_v */
} or_views;

typedef struct {
  int32_t tile;
  double dilation, near_plane, alpha_min, alpha_max, t_min, q_max;
} or_config;

/* Flags raised per pixel when a decision of the cutoffs lies close to its
 * threshold, where a binary32 renderer may take it the other way. The q,
 * alpha_min and t_min decisions are "flagged decisions": the walk numbers them
 * and can invert any subset (flip mask), so a test can enumerate every
 * legitimate outcome. The clamp is continuous in the image and only flagged
 * (its derivative jumps). */
enum {
  OR_NEAR_Q = 1,        /* |q - q_max| < 2e-3 and the Gaussian would pass alpha_min */
  OR_NEAR_ALPHA_MIN = 2,/* |sigma - alpha_min| < 1e-3 alpha_min */
  OR_NEAR_CLAMP = 4,    /* |alpha G - alpha_max| < 1e-5 */
  OR_NEAR_TMIN = 8,     /* |T' - t_min| < 1e-4 t_min */
  OR_NEAR_CULL = 16     /* a Gaussian's depth within 1e-6 (relative) of near/far */
};

/* Forward. pix == NULL renders every pixel of every view in (v, row, col)
 * order (n_pix must then be V*H*W); otherwise pix is [n_pix][3] = (v, row, col).
 * depth32 [V][n] is the FP32 depth of the binning reference, used to order the
 * Gaussians (ascending depth, ties by ascending index).
 * flip_masks [n_pix] (nullable = all 0): bit d inverts the d-th flagged
 * decision of that pixel's walk.
 * Outputs per requested pixel (each nullable): image C, final transmittance T,
 * id of the last Gaussian added (-1 if none), number of Gaussians added,
 * flags, number of flagged decisions met. */
int or_render(const or_scene *s, const or_views *vw, const or_config *cfg,
              const float *depth32, int64_t n_pix, const int32_t *pix,
              const uint32_t *flip_masks, double *image, double *t_final,
              int32_t *last_id, int32_t *n_contrib, int32_t *flags,
              int32_t *n_flagged, int n_threads);

/* Backward of L = sum_p dL_dC[p] * C(p) over the requested pixels.
 * flip_masks [n_pix] (nullable = all 0): the walk differentiated at each
 * pixel is the forward's walk with the same mask (bit d inverts the d-th
 * flagged decision), so a pixel can be differentiated along the outcome a
 * binary32 renderer actually took near a cutoff.
 * Every output pointer may be NULL (skip). Outputs are overwritten. */
int or_render_backward(const or_scene *s, const or_views *vw,
                       const or_config *cfg, const float *depth32,
                       int64_t n_pix, const int32_t *pix, const uint32_t *flip_masks,
                       const double *dL_dC,
                       double *g_means, double *g_log_scales, double *g_quats,
                       double *g_opacity_logits, double *g_feat,
                       double *g_b_iso, double *g_B_dir,
                       double *g_pose /* [V][12] */,
                       double *g_2d /* [V][n][7 + k_L]: u, v, conic a, b, c, alpha,
                                       logit z, then sum of dL/dz Y_m (= dL/dh_m) */,
                       int n_threads);

/* Per requested pixel: the number of projected Gaussians with q <= q_max at
 * the pixel centre, over the whole list (no early termination, no alpha_min):
 * the pixel-Gaussian pairs inside the cutoff ellipse. */
int or_count_inside(const or_scene *s, const or_views *vw, const or_config *cfg,
                    const float *depth32, int64_t n_pix, const int32_t *pix,
                    int32_t *n_inside, int n_threads);

/* Per (view, Gaussian) projected quantities, FP64, for tests:
 * out [V][n][9] = u, v, conic a, b, c, alpha, color, depth, valid. */
int or_project(const or_scene *s, const or_views *vw, const or_config *cfg,
               double *out);

/* ---------------- FP32 binning reference ---------------- */

typedef struct {
  int32_t n;
  const float *means, *log_scales, *quats; /* as above, float32 */
} or_geom32;

typedef struct {
  int32_t n_views, height, width;
  const float *world_to_cam, *detector;
} or_views32;

typedef struct {
  int32_t tile;
  float dilation, near_plane, q_max;
} or_config32;

/* exp in binary32 using only correctly rounded +, -, *, rint and an exact
 * power-of-two scaling (Cody-Waite reduction, degree-7 Taylor polynomial). */
float or_exp32(float x);

/* Per (v, i): depth (camera z), tiles touched, and the inclusive tile
 * rectangle rect[v][i] = (tx0, ty0, tx1, ty1) (-1s when culled).
 * Also the FP32 mean and 2D covariance diagonal (for tests): aux [V][n][4] =
 * (u, v, cov_a, cov_c); aux may be NULL. */
int or32_project(const or_geom32 *g, const or_views32 *vw, const or_config32 *cfg,
                 float *depth, uint32_t *tiles_touched, int32_t *rect, float *aux);

/* Emission + stable sort + tile ranges. keys[m] = (global tile << 32) |
 * bits(depth) where global tile = v * tiles_x * tiles_y + ty * tiles_x + tx;
 * vals[m] = Gaussian index. ranges [V * tiles][2] = [start, end), (0, 0) when
 * empty. m_total must equal the sum of tiles_touched. */
int or32_bin(const or_views32 *vw, const or_config32 *cfg, int32_t n,
             const float *depth, const uint32_t *tiles_touched,
             const int32_t *rect, int64_t m_total, uint64_t *keys,
             uint32_t *vals, uint32_t *ranges);

#ifdef __cplusplus
}
#endif
#endif
