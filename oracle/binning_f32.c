/*
 * binning_f32.c -- FP32 binning reference of the oracle.
 *
 * TEST INFRASTRUCTURE ONLY (see ddgs_oracle.h). Compile with
 * -ffp-contract=off: every float operation below is one correctly rounded
 * IEEE binary32 operation, evaluated in the order written.
 *
 * What it decides. Eq. 1 multiplies, for the j-th Gaussian "on the ray",
 * the transmittance of every Gaussian in front of it, so a renderer must fix
 * an order; the image-plane projections of Eq. 1's text (mu-hat, Sigma-hat)
 * fix where a Gaussian can reach. The tiled renderer turns those into integer
 * decisions: is the Gaussian culled, which tiles does its q <= q_max ellipse
 * touch, and in which depth order does each tile list it. This file takes
 * those decisions in binary32, by the operation order G1..G15 below, which the
 * GPU preprocess follows from the same written definition.
 *
 *   G1  s_j = exp32(log_s_j)
 *   G2  n2 = ((w*w + x*x) + y*y) + z*z;  r = sqrt(n2);  w, x, y, z each / r
 *   G3  R from the unit quaternion, e.g. R00 = 1 - 2*(yy + zz),
 *       R01 = 2*(xy - wz), with xy = x*y etc. (products rounded first)
 *   G4  M_ij = R_ij * s_j
 *   G5  Sigma_ij = (M_i0*M_j0 + M_i1*M_j1) + M_i2*M_j2
 *   G6  xc_r = ((W_r0*mu_0 + W_r1*mu_1) + W_r2*mu_2) + t_r
 *   G7  culled unless near < z < sdd            (z = xc_2)
 *   G8  fu = sdd/pitch_u, fv = sdd/pitch_v, cu = 0.5*W + off_u,
 *       cv = 0.5*H + off_v, xz = x/z, yz = y/z, u = fu*xz + cu, v = fv*yz + cv
 *   G9  j00 = fu/z, j11 = fv/z, j02 = -(j00*xz), j12 = -(j11*yz)
 *   G10 A_0k = j00*W_0k + j02*W_2k,  A_1k = j11*W_1k + j12*W_2k
 *   G11 B_rk = (A_r0*Sigma_0k + A_r1*Sigma_1k) + A_r2*Sigma_2k
 *   G12 a = ((B_00*A_00 + B_01*A_01) + B_02*A_02) + d
 *       b =  (B_00*A_10 + B_01*A_11) + B_02*A_12
 *       c = ((B_10*A_10 + B_11*A_11) + B_12*A_12) + d
 *   G13 det = a*c - b*b; culled unless det > 0
 *   G14 ex = sqrt(q_max*a), ey = sqrt(q_max*c);
 *       ex' = ex*(1 + 2^-10) + 2^-10 (same for ey); culled if u, v, ex', ey'
 *       is not a number
 *   G15 columns lo = ceil((u - ex') - 0.5), hi = floor((u + ex') - 0.5),
 *       clamped to [0, W-1] (rows likewise with v, ey', H); culled if lo > hi;
 *       tiles tx0 = lo / tile, tx1 = hi / tile (integers);
 *       tiles touched = (tx1 - tx0 + 1) * (ty1 - ty0 + 1)
 *
 * The q <= q_max ellipse of the 2D covariance [[a, b], [b, c]] spans exactly
 * +-sqrt(q_max * a) in u and +-sqrt(q_max * c) in v; G14's small widening keeps
 * the rectangle a superset of every pixel whose FP32 or FP64 q is <= q_max.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "ddgs_oracle.h"

/* Cody & Waite (1980) argument reduction: ln 2 = LN2_HI + LN2_LO with LN2_HI
 * short enough that k * LN2_HI is exact for |k| < 2^15. */
#define OR_LN2_HI 0.693359375f
#define OR_LN2_LO (-2.12194440e-4f)
#define OR_LOG2E 1.44269504f

static float pow2i(int k) {
  /* 2^k for k in [-126, 127], built from its exponent field (exact). */
  uint32_t bits = (uint32_t)(k + 127) << 23;
  float f;
  memcpy(&f, &bits, sizeof f);
  return f;
}

float or_exp32(float x) {
  if (x != x) return x;
  if (x > 88.0f) return INFINITY;
  if (x < -87.0f) return 0.0f;
  float kf = rintf(x * OR_LOG2E);
  int k = (int)kf;
  float r = (x - kf * OR_LN2_HI) - kf * OR_LN2_LO; /* |r| <= ~0.35 */
  /* Taylor series of e^r to degree 7, Horner form, coefficients 1/n!. */
  float p = (float)(1.0 / 5040.0);
  p = p * r + (float)(1.0 / 720.0);
  p = p * r + (float)(1.0 / 120.0);
  p = p * r + (float)(1.0 / 24.0);
  p = p * r + (float)(1.0 / 6.0);
  p = p * r + 0.5f;
  p = p * r + 1.0f;
  p = p * r + 1.0f;
  return p * pow2i(k);
}

/* One Gaussian in one view; returns tiles touched (0 = culled). */
static uint32_t project_one(const float *mu, const float *ls, const float *qt,
                            const float *Wt, const float *det_params, int H,
                            int Wd, const or_config32 *cfg, float *depth_out,
                            int32_t rect[4], float aux[4]) {
  rect[0] = rect[1] = rect[2] = rect[3] = -1;
  /* G1 */
  float s0 = or_exp32(ls[0]), s1 = or_exp32(ls[1]), s2 = or_exp32(ls[2]);
  /* G2 */
  float w = qt[0], x = qt[1], y = qt[2], z = qt[3];
  float n2 = ((w * w + x * x) + y * y) + z * z;
  float rn = sqrtf(n2);
  w = w / rn; x = x / rn; y = y / rn; z = z / rn;
  /* G3 */
  float xx = x * x, yy = y * y, zz = z * z;
  float xy = x * y, xz = x * z, yz = y * z;
  float wx = w * x, wy = w * y, wz = w * z;
  float R[3][3];
  R[0][0] = 1.0f - 2.0f * (yy + zz);
  R[0][1] = 2.0f * (xy - wz);
  R[0][2] = 2.0f * (xz + wy);
  R[1][0] = 2.0f * (xy + wz);
  R[1][1] = 1.0f - 2.0f * (xx + zz);
  R[1][2] = 2.0f * (yz - wx);
  R[2][0] = 2.0f * (xz - wy);
  R[2][1] = 2.0f * (yz + wx);
  R[2][2] = 1.0f - 2.0f * (xx + yy);
  /* G4 */
  float M[3][3];
  for (int i = 0; i < 3; ++i) {
    M[i][0] = R[i][0] * s0;
    M[i][1] = R[i][1] * s1;
    M[i][2] = R[i][2] * s2;
  }
  /* G5 */
  float S[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      float v = (M[i][0] * M[j][0] + M[i][1] * M[j][1]) + M[i][2] * M[j][2];
      S[i][j] = v;
      S[j][i] = v;
    }
  /* G6: Wt is [3][4] row-major (R | t) */
  float xc[3];
  for (int r = 0; r < 3; ++r)
    xc[r] = ((Wt[4 * r + 0] * mu[0] + Wt[4 * r + 1] * mu[1]) +
             Wt[4 * r + 2] * mu[2]) + Wt[4 * r + 3];
  float zc = xc[2];
  *depth_out = zc;
  /* G7 */
  float sdd = det_params[0];
  if (!(zc > cfg->near_plane && zc < sdd)) return 0;
  /* G8 */
  float fu = sdd / det_params[1];
  float fv = sdd / det_params[2];
  float cu = 0.5f * (float)Wd + det_params[3];
  float cv = 0.5f * (float)H + det_params[4];
  float xzr = xc[0] / zc, yzr = xc[1] / zc;
  float u = fu * xzr + cu;
  float v = fv * yzr + cv;
  /* G9 */
  float j00 = fu / zc, j11 = fv / zc;
  float j02 = -(j00 * xzr), j12 = -(j11 * yzr);
  /* G10 */
  float A[2][3];
  for (int k = 0; k < 3; ++k) {
    A[0][k] = j00 * Wt[0 + k] + j02 * Wt[8 + k];
    A[1][k] = j11 * Wt[4 + k] + j12 * Wt[8 + k];
  }
  /* G11 */
  float B[2][3];
  for (int r = 0; r < 2; ++r)
    for (int k = 0; k < 3; ++k)
      B[r][k] = (A[r][0] * S[0][k] + A[r][1] * S[1][k]) + A[r][2] * S[2][k];
  /* G12 */
  float d = cfg->dilation;
  float ca = ((B[0][0] * A[0][0] + B[0][1] * A[0][1]) + B[0][2] * A[0][2]) + d;
  float cb = (B[0][0] * A[1][0] + B[0][1] * A[1][1]) + B[0][2] * A[1][2];
  float cc = ((B[1][0] * A[1][0] + B[1][1] * A[1][1]) + B[1][2] * A[1][2]) + d;
  if (aux) { aux[0] = u; aux[1] = v; aux[2] = ca; aux[3] = cc; }
  /* G13 */
  float det = ca * cc - cb * cb;
  if (!(det > 0.0f)) return 0;
  /* G14 */
  float ex = sqrtf(cfg->q_max * ca), ey = sqrtf(cfg->q_max * cc);
  ex = ex * 1.0009765625f + 0.0009765625f;
  ey = ey * 1.0009765625f + 0.0009765625f;
  if (u != u || v != v || ex != ex || ey != ey) return 0;
  /* G15 */
  float xlo = ceilf((u - ex) - 0.5f), xhi = floorf((u + ex) - 0.5f);
  float ylo = ceilf((v - ey) - 0.5f), yhi = floorf((v + ey) - 0.5f);
  xlo = fmaxf(xlo, 0.0f); xhi = fminf(xhi, (float)(Wd - 1));
  ylo = fmaxf(ylo, 0.0f); yhi = fminf(yhi, (float)(H - 1));
  if (xlo > xhi || ylo > yhi) return 0;
  int t = cfg->tile;
  int tx0 = (int)xlo / t, tx1 = (int)xhi / t;
  int ty0 = (int)ylo / t, ty1 = (int)yhi / t;
  rect[0] = tx0; rect[1] = ty0; rect[2] = tx1; rect[3] = ty1;
  return (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
}

int or32_project(const or_geom32 *g, const or_views32 *vw, const or_config32 *cfg,
                 float *depth, uint32_t *tiles_touched, int32_t *rect, float *aux) {
  if (!g || !vw || !cfg || cfg->tile <= 0) return 1;
  const int64_t n = g->n;
#pragma omp parallel for schedule(static)
  for (int64_t vi = 0; vi < (int64_t)vw->n_views * n; ++vi) {
    int64_t v = vi / n, i = vi % n;
    float a4[4];
    tiles_touched[vi] = project_one(
        g->means + 3 * i, g->log_scales + 3 * i, g->quats + 4 * i,
        vw->world_to_cam + 12 * v, vw->detector + 5 * v, vw->height, vw->width,
        cfg, &depth[vi], &rect[4 * vi], a4);
    if (aux) memcpy(aux + 4 * vi, a4, sizeof a4);
  }
  return 0;
}

typedef struct {
  uint64_t key;
  uint32_t val;
} kv;

static int cmp_kv(const void *pa, const void *pb) {
  const kv *a = (const kv *)pa, *b = (const kv *)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  if (a->val != b->val) return a->val < b->val ? -1 : 1;
  return 0;
}

int or32_bin(const or_views32 *vw, const or_config32 *cfg, int32_t n,
             const float *depth, const uint32_t *tiles_touched,
             const int32_t *rect, int64_t m_total, uint64_t *keys,
             uint32_t *vals, uint32_t *ranges) {
  const int t = cfg->tile;
  const int64_t tiles_x = (vw->width + t - 1) / t;
  const int64_t tiles_y = (vw->height + t - 1) / t;
  const int64_t tiles = tiles_x * tiles_y;
  kv *buf = (kv *)malloc(sizeof(kv) * (size_t)(m_total > 0 ? m_total : 1));
  if (!buf) return 2;
  int64_t m = 0;
  /* Emission in (view, Gaussian index, tile row, tile column) order. */
  for (int64_t v = 0; v < vw->n_views; ++v)
    for (int64_t i = 0; i < n; ++i) {
      int64_t vi = v * n + i;
      if (tiles_touched[vi] == 0) continue;
      const int32_t *r = rect + 4 * vi;
      uint32_t dbits;
      memcpy(&dbits, &depth[vi], sizeof dbits);
      for (int64_t ty = r[1]; ty <= r[3]; ++ty)
        for (int64_t tx = r[0]; tx <= r[2]; ++tx) {
          if (m >= m_total) { free(buf); return 3; }
          uint64_t gt = (uint64_t)(v * tiles + ty * tiles_x + tx);
          buf[m].key = (gt << 32) | (uint64_t)dbits;
          buf[m].val = (uint32_t)i;
          ++m;
        }
    }
  if (m != m_total) { free(buf); return 3; }
  /* Equal keys come from distinct Gaussians of one view, emitted in ascending
   * index order, so ordering by (key, index) is the stable sort by key. */
  qsort(buf, (size_t)m, sizeof(kv), cmp_kv);
  memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)(vw->n_views * tiles));
  for (int64_t j = 0; j < m; ++j) {
    keys[j] = buf[j].key;
    vals[j] = buf[j].val;
    uint64_t gt = buf[j].key >> 32;
    if (j == 0 || (buf[j - 1].key >> 32) != gt) ranges[2 * gt] = (uint32_t)j;
    if (j == m - 1 || (buf[j + 1].key >> 32) != gt) ranges[2 * gt + 1] = (uint32_t)(j + 1);
  }
  free(buf);
  return 0;
}
