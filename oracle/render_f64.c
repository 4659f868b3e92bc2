/*
 * render_f64.c -- FP64 renderer of the oracle (forward and analytic backward).
 *
 * TEST INFRASTRUCTURE ONLY (see ddgs_oracle.h).
 *
 * What it computes, step by step, with the paper's notation:
 *   - Gaussian g_i = {mu_i, Sigma_i, alpha_i, f_i} (Sec. 3.1). Sigma_i is
 *     built from a scale and a rotation, Sigma = R S S^T R^T with
 *     S = diag(exp(log_s)) and R the rotation of the normalised quaternion;
 *     alpha_i = sigmoid(opacity logit).
 *   - Radiosity (Eq. 3): isotropic Gaussians c = sigmoid(b_iso . f_i);
 *     direction-dependent Gaussians c = sigmoid(Y_1..L(theta, phi) . B_dir f_j)
 *     with Y the real spherical harmonics of degrees 1..L (no degree 0), so
 *     k_L = L(L+2). The ray angles are those of the unit direction from the
 *     X-ray source to the Gaussian's mean, in world coordinates.
 *     Written per pair (pixel p, Gaussian j) as c = sigmoid(z), z = a_j +
 *     Y(d) . h_j with a_j = b_iso . f_j for a Gaussian with an isotropic
 *     term (else 0) and h_j = B_dir f_j for one with a directional term (else
 *     0). Variants: "entangled" gives every Gaussian both terms (the
 *     direct-entangled ablation of Table 3); "per_pixel" takes d as the unit
 *     direction of pixel p's ray (source to pixel centre) rather than of the
 *     Gaussian's mean.
 *   - Image-plane projections mu-hat, Sigma-hat (text of Eq. 1): perspective
 *     projection of the mean onto the detector and the local affine
 *     (Jacobian) projection of Sigma, plus a dilation d on the diagonal.
 *   - Eq. 1: C(p) = sum_j c_j sigma_j prod_{l<j} (1 - sigma_l) with
 *     sigma = alpha exp(-q/2), q = (p - mu-hat)^T Sigma-hat^-1 (p - mu-hat),
 *     over the Gaussians in ascending depth, with the cutoffs q <= q_max,
 *     sigma = min(alpha_max, alpha G) >= alpha_min, and the walk stopping before
 *     a Gaussian that would bring the transmittance below t_min. Every
 *     Gaussian is tested at every pixel: no tiles, no bounding boxes.
 *   - Appendix A.1: prod (1 - sigma_l) is the Beer-Lambert transmittance;
 *     the image is monochrome (one channel); background 0.
 *   - Appendix A.2: isotropic and direction-dependent Gaussians are sorted
 *     and blended together in one list.
 *   - Backward: the exact derivative of the above (Sec. 3.1 relies on the
 *     renderer being differentiable; Sec. 4.3 differentiates with respect to
 *     the pose), written with small dense matrix products.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "ddgs_oracle.h"

#define KMAX 64
#define LMAX 4
#define KLMAX (LMAX * (LMAX + 2))
#define OR_PI 3.14159265358979323846

/* ---- real spherical harmonics of degrees 1..L (Eq. 3's Y without degree 0) ----
 * For a unit direction (x, y, z), degree l, order m (-l..l):
 *   Y_lm = (-1)^m N_l|m| sqrt(2)^[m != 0] D^|m| P_l(z) * { Re (x+iy)^|m|  (m > 0)
 *                                                        { 1              (m = 0)
 *                                                        { Im (x+iy)^|m|  (m < 0)
 * with P_l the Legendre polynomial, D^m its m-th derivative, and
 * N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!). sin^m(theta) e^{i m phi} =
 * (x+iy)^m on the unit sphere, so this is the usual real harmonic with the
 * Condon-Shortley sign (-1)^m; at l = 1 it is sqrt(3/(4 pi)) (-y, z, -x).
 * Index of (l, m): l^2 - 1 + (m + l). The functions are polynomials in (x, y, z);
 * dY[j][c] is their derivative along component c. */
static void legendre_coeffs(int l, double c[LMAX + 1]) {
  double p0[LMAX + 1] = {0}, p1[LMAX + 1] = {0}, p2[LMAX + 1];
  p0[0] = 1.0;
  p1[1] = 1.0;
  if (l == 0) { memcpy(c, p0, sizeof p0); return; }
  for (int n = 1; n < l; ++n) {  /* (n+1) P_{n+1} = (2n+1) z P_n - n P_{n-1} */
    for (int i = 0; i <= LMAX; ++i) {
      double zp = i > 0 ? p1[i - 1] : 0.0;
      p2[i] = ((2 * n + 1) * zp - n * p0[i]) / (n + 1);
    }
    memcpy(p0, p1, sizeof p0);
    memcpy(p1, p2, sizeof p1);
  }
  memcpy(c, p1, sizeof p1);
}

static double poly_deriv_eval(const double c[LMAX + 1], int m, double z) {
  /* value at z of the m-th derivative of sum_i c_i z^i */
  double acc = 0.0, zp = 1.0;
  for (int i = m; i <= LMAX; ++i) {
    double f = 1.0;
    for (int j = 0; j < m; ++j) f *= (i - j);
    acc += c[i] * f * zp;
    zp *= z;
  }
  return acc;
}

static double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

static void real_sh(int L, const double d[3], double *Y, double (*dY)[3]) {
  const double x = d[0], y = d[1], z = d[2];
  /* Re/Im of (x + i y)^m and their derivatives */
  double re[LMAX + 1], im[LMAX + 1];
  re[0] = 1.0; im[0] = 0.0;
  for (int m = 1; m <= LMAX; ++m) {
    re[m] = re[m - 1] * x - im[m - 1] * y;
    im[m] = re[m - 1] * y + im[m - 1] * x;
  }
  for (int l = 1; l <= L; ++l) {
    double c[LMAX + 1];
    legendre_coeffs(l, c);
    for (int m = -l; m <= l; ++m) {
      const int am = m < 0 ? -m : m;
      const double N = sqrt((2.0 * l + 1.0) / (4.0 * OR_PI) * factorial(l - am) / factorial(l + am)) *
                       (am ? sqrt(2.0) : 1.0) * ((am & 1) ? -1.0 : 1.0);
      const double Q = poly_deriv_eval(c, am, z), dQ = poly_deriv_eval(c, am + 1, z);
      double A, dAx, dAy;
      if (m > 0) { A = re[am]; dAx = am * re[am - 1]; dAy = -am * im[am - 1]; }
      else if (m < 0) { A = im[am]; dAx = am * im[am - 1]; dAy = am * re[am - 1]; }
      else { A = 1.0; dAx = 0.0; dAy = 0.0; }
      const int j = l * l - 1 + (m + l);
      Y[j] = N * Q * A;
      if (dY) {
        dY[j][0] = N * Q * dAx;
        dY[j][1] = N * Q * dAy;
        dY[j][2] = N * dQ * A;
      }
    }
  }
}

typedef struct {
  int valid, near_cull;
  double qn[4], qnorm, s[3], R[3][3], M[3][3], Sig[3][3];
  double W[3][3], t[3], xc[3], fu, fv;
  double J[2][3], A[2][3], cov[3], det, conic[3];
  double u, v, alpha, color;  /* color: per-Gaussian direction only */
  int has_iso, has_dir;
  double a;                   /* isotropic logit b_iso . f (0 without that term) */
  double d[3], dnorm, dhat[3], Y[KLMAX], h[KLMAX], dY[KLMAX][3];
} g64;

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* Forward projection of Gaussian i into view v, keeping intermediates. */
static void project64(const or_scene *sc, const or_views *vw,
                      const or_config *cfg, int64_t v, int64_t i, g64 *g) {
  memset(g, 0, sizeof *g);
  const double *mu = sc->means + 3 * i;
  const double *q = sc->quats + 4 * i;
  const double *T = vw->world_to_cam + 12 * v;
  const double *dp = vw->detector + 5 * v;
  const int k = sc->k;

  for (int j = 0; j < 3; ++j) g->s[j] = exp(sc->log_scales[3 * i + j]);
  g->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int j = 0; j < 4; ++j) g->qn[j] = q[j] / g->qnorm;
  double w = g->qn[0], x = g->qn[1], y = g->qn[2], z = g->qn[3];
  double (*R)[3] = g->R;
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) g->M[a][b] = R[a][b] * g->s[b];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double acc = 0;
      for (int c = 0; c < 3; ++c) acc += g->M[a][c] * g->M[b][c];
      g->Sig[a][b] = acc;
    }
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) g->W[r][c] = T[4 * r + c];
    g->t[r] = T[4 * r + 3];
  }
  for (int r = 0; r < 3; ++r)
    g->xc[r] = g->W[r][0] * mu[0] + g->W[r][1] * mu[1] + g->W[r][2] * mu[2] + g->t[r];

  /* opacity and radiosity do not depend on culling */
  g->alpha = sigmoid(sc->opacity_logits[i]);
  const double *f = sc->feat + (int64_t)k * i;
  g->has_iso = sc->entangled || i < sc->n_iso;
  g->has_dir = sc->entangled || i >= sc->n_iso;
  double zl = 0;
  if (g->has_iso) {
    for (int n = 0; n < k; ++n) g->a += sc->b_iso[n] * f[n];
    zl = g->a;
  }
  if (g->has_dir) {
    const int kL = sc->L * (sc->L + 2);
    for (int m = 0; m < kL; ++m) {
      double hm = 0;
      for (int n = 0; n < k; ++n) hm += sc->B_dir[m * k + n] * f[n];
      g->h[m] = hm;
    }
    if (!sc->per_pixel) {
      /* source position S = -W^T t; direction mu - S = mu + W^T t */
      for (int c = 0; c < 3; ++c)
        g->d[c] = mu[c] + g->W[0][c] * g->t[0] + g->W[1][c] * g->t[1] + g->W[2][c] * g->t[2];
      g->dnorm = sqrt(g->d[0] * g->d[0] + g->d[1] * g->d[1] + g->d[2] * g->d[2]);
      for (int c = 0; c < 3; ++c) g->dhat[c] = g->d[c] / g->dnorm;
      real_sh(sc->L, g->dhat, g->Y, g->dY);
      for (int m = 0; m < kL; ++m) zl += g->Y[m] * g->h[m];
    }
  }
  /* with per-pixel directions a directional Gaussian has no single colour */
  g->color = (g->has_dir && sc->per_pixel) ? NAN : sigmoid(zl);

  double zc = g->xc[2], sdd = dp[0];
  double tol_n = 1e-6 * fabs(cfg->near_plane) + 1e-12, tol_f = 1e-6 * sdd;
  if (fabs(zc - cfg->near_plane) < tol_n || fabs(zc - sdd) < tol_f) g->near_cull = 1;
  if (!(zc > cfg->near_plane && zc < sdd)) return;
  g->fu = sdd / dp[1];
  g->fv = sdd / dp[2];
  double cu = 0.5 * vw->width + dp[3], cv = 0.5 * vw->height + dp[4];
  g->u = g->fu * g->xc[0] / zc + cu;
  g->v = g->fv * g->xc[1] / zc + cv;
  g->J[0][0] = g->fu / zc; g->J[0][1] = 0; g->J[0][2] = -g->fu * g->xc[0] / (zc * zc);
  g->J[1][0] = 0; g->J[1][1] = g->fv / zc; g->J[1][2] = -g->fv * g->xc[1] / (zc * zc);
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c)
      g->A[r][c] = g->J[r][0] * g->W[0][c] + g->J[r][1] * g->W[1][c] + g->J[r][2] * g->W[2][c];
  double C2[2][2];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c) {
      double acc = 0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) acc += g->A[r][a] * g->Sig[a][b] * g->A[c][b];
      C2[r][c] = acc;
    }
  g->cov[0] = C2[0][0] + cfg->dilation;
  g->cov[1] = 0.5 * (C2[0][1] + C2[1][0]);
  g->cov[2] = C2[1][1] + cfg->dilation;
  g->det = g->cov[0] * g->cov[2] - g->cov[1] * g->cov[1];
  if (!(g->det > 0)) return;
  g->conic[0] = g->cov[2] / g->det;
  g->conic[1] = -g->cov[1] / g->det;
  g->conic[2] = g->cov[0] / g->det;
  g->valid = 1;
}

/* Back-propagate the 2D gradient gg[7 + k_L] = d/d(u, v, conic a, b, c,
 * alpha), the summed gradient of the colour logit z, and dL/dh_m (the sums of
 * dL/dz Y_m over the pixels) of Gaussian i in view v into parameter and pose
 * gradients. */
typedef struct {
  double mu[3], ls[3], q[4], logit, f[KMAX];
  double b_iso[KMAX], B_dir[KLMAX * KMAX];
  double pose[12];
} grad_acc;

static void backprop64(const or_scene *sc, int64_t i, const g64 *g,
                       const double gg[7], grad_acc *out) {
  const int k = sc->k;
  const double *mu = sc->means + 3 * i;
  const double *f = sc->feat + (int64_t)k * i;
  double dW[3][3] = {{0}}, dt[3] = {0}, dmu[3] = {0};

  /* radiosity, Eq. 3: z = a + Y(d) . h, a = b_iso . f, h = B_dir f */
  const double dzl = gg[6];
  if (g->has_iso) {
    for (int n = 0; n < k; ++n) {
      out->f[n] += dzl * sc->b_iso[n];
      out->b_iso[n] += dzl * f[n];
    }
  }
  if (g->has_dir) {
    const int kL = sc->L * (sc->L + 2);
    const double *dh = gg + 7;
    for (int m = 0; m < kL; ++m)
      for (int n = 0; n < k; ++n) {
        out->B_dir[m * k + n] += dh[m] * f[n];
        out->f[n] += sc->B_dir[m * k + n] * dh[m];
      }
  }
  if (g->has_dir && !sc->per_pixel) {
    /* the direction of the mean: d = mu - S */
    const int kL = sc->L * (sc->L + 2);
    double dY[KLMAX];
    for (int m = 0; m < kL; ++m) dY[m] = dzl * g->h[m];
    double ddh[3] = {0, 0, 0};
    for (int m = 0; m < kL; ++m)
      for (int c3 = 0; c3 < 3; ++c3) ddh[c3] += dY[m] * g->dY[m][c3];
    double dot = ddh[0] * g->dhat[0] + ddh[1] * g->dhat[1] + ddh[2] * g->dhat[2];
    double dd[3];
    for (int c = 0; c < 3; ++c) dd[c] = (ddh[c] - g->dhat[c] * dot) / g->dnorm;
    /* d = mu + W^T t */
    for (int c = 0; c < 3; ++c) dmu[c] += dd[c];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        dW[r][c] += g->t[r] * dd[c];
        dt[r] += g->W[r][c] * dd[c];
      }
  }
  /* opacity */
  out->logit += gg[5] * g->alpha * (1 - g->alpha);

  if (g->valid) {
    /* conic = inverse of the 2D covariance */
    double K[2][2] = {{g->conic[0], g->conic[1]}, {g->conic[1], g->conic[2]}};
    double GK[2][2] = {{gg[2], 0.5 * gg[3]}, {0.5 * gg[3], gg[4]}};
    double GS[2][2];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 2; ++c) {
        double acc = 0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) acc += K[r][a] * GK[a][b] * K[b][c];
        GS[r][c] = -acc;
      }
    /* cov2 = A Sigma A^T: dA = 2 GS A Sigma, dSigma = A^T GS A */
    double dA[2][3], dSig[3][3];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c) {
        double acc = 0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 3; ++b) acc += GS[r][a] * g->A[a][b] * g->Sig[b][c];
        dA[r][c] = 2 * acc;
      }
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double acc = 0;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) acc += g->A[a][r] * GS[a][b] * g->A[b][c];
        dSig[r][c] = acc;
      }
    /* A = J W */
    double dJ[2][3];
    for (int r = 0; r < 2; ++r)
      for (int c = 0; c < 3; ++c) {
        double acc = 0;
        for (int b = 0; b < 3; ++b) acc += dA[r][b] * g->W[c][b];
        dJ[r][c] = acc;
      }
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        dW[r][c] += g->J[0][r] * dA[0][c] + g->J[1][r] * dA[1][c];
    /* J(xc) and the projected mean */
    double x = g->xc[0], y = g->xc[1], z = g->xc[2], fu = g->fu, fv = g->fv;
    double dxc[3] = {0, 0, 0};
    dxc[0] += dJ[0][2] * (-fu / (z * z));
    dxc[1] += dJ[1][2] * (-fv / (z * z));
    dxc[2] += dJ[0][0] * (-fu / (z * z)) + dJ[0][2] * (2 * fu * x / (z * z * z)) +
              dJ[1][1] * (-fv / (z * z)) + dJ[1][2] * (2 * fv * y / (z * z * z));
    dxc[0] += gg[0] * fu / z;
    dxc[2] += -gg[0] * fu * x / (z * z);
    dxc[1] += gg[1] * fv / z;
    dxc[2] += -gg[1] * fv * y / (z * z);
    /* xc = W mu + t */
    for (int c = 0; c < 3; ++c)
      dmu[c] += g->W[0][c] * dxc[0] + g->W[1][c] * dxc[1] + g->W[2][c] * dxc[2];
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) dW[r][c] += dxc[r] * mu[c];
      dt[r] += dxc[r];
    }
    /* Sigma = M M^T: dM = 2 dSigma M */
    double dM[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double acc = 0;
        for (int a = 0; a < 3; ++a) acc += (dSig[r][a] + dSig[a][r]) * g->M[a][c];
        dM[r][c] = acc;
      }
    /* M = R diag(s) */
    double dR[3][3], ds[3] = {0, 0, 0};
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        dR[r][c] = dM[r][c] * g->s[c];
        ds[c] += dM[r][c] * g->R[r][c];
      }
    for (int c = 0; c < 3; ++c) out->ls[c] += ds[c] * g->s[c];
    /* R(unit quaternion) */
    double w = g->qn[0], qx = g->qn[1], qy = g->qn[2], qz = g->qn[3];
    double dqn[4];
    dqn[0] = 2 * (-qz * dR[0][1] + qy * dR[0][2] + qz * dR[1][0] - qx * dR[1][2] -
                  qy * dR[2][0] + qx * dR[2][1]);
    dqn[1] = 2 * (qy * dR[0][1] + qz * dR[0][2] + qy * dR[1][0] - 2 * qx * dR[1][1] -
                  w * dR[1][2] + qz * dR[2][0] + w * dR[2][1] - 2 * qx * dR[2][2]);
    dqn[2] = 2 * (-2 * qy * dR[0][0] + qx * dR[0][1] + w * dR[0][2] + qx * dR[1][0] +
                  qz * dR[1][2] - w * dR[2][0] + qz * dR[2][1] - 2 * qy * dR[2][2]);
    dqn[3] = 2 * (-2 * qz * dR[0][0] - w * dR[0][1] + qx * dR[0][2] + w * dR[1][0] -
                  2 * qz * dR[1][1] + qy * dR[1][2] + qx * dR[2][0] + qy * dR[2][1]);
    double dot = dqn[0] * w + dqn[1] * qx + dqn[2] * qy + dqn[3] * qz;
    for (int c = 0; c < 4; ++c) out->q[c] += (dqn[c] - g->qn[c] * dot) / g->qnorm;
  }
  for (int c = 0; c < 3; ++c) out->mu[c] += dmu[c];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) out->pose[4 * r + c] += dW[r][c];
    out->pose[4 * r + 3] += dt[r];
  }
}

/* ---- per-view depth order ---- */

typedef struct {
  float z;
  int32_t i;
} zi;

static int cmp_zi(const void *pa, const void *pb) {
  const zi *a = (const zi *)pa, *b = (const zi *)pb;
  if (a->z != b->z) return a->z < b->z ? -1 : 1;
  return (a->i > b->i) - (a->i < b->i);
}

typedef struct {
  g64 *g;        /* [n] projections of this view */
  int32_t *order;/* valid Gaussians by ascending (FP32 depth, index) */
  int64_t n_order;
  int near_cull;
} view_cache;

static int build_view(const or_scene *sc, const or_views *vw, const or_config *cfg,
                      const float *depth32, int64_t v, view_cache *vc) {
  const int64_t n = sc->n;
  vc->g = (g64 *)malloc(sizeof(g64) * (size_t)(n > 0 ? n : 1));
  zi *tmp = (zi *)malloc(sizeof(zi) * (size_t)(n > 0 ? n : 1));
  vc->order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!vc->g || !tmp || !vc->order) return 2;
  vc->near_cull = 0;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) project64(sc, vw, cfg, v, i, &vc->g[i]);
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) {
    vc->near_cull |= vc->g[i].near_cull;
    if (!vc->g[i].valid) continue;
    tmp[m].z = depth32[v * n + i];
    tmp[m].i = (int32_t)i;
    ++m;
  }
  qsort(tmp, (size_t)m, sizeof(zi), cmp_zi);
  for (int64_t j = 0; j < m; ++j) vc->order[j] = tmp[j].i;
  vc->n_order = m;
  free(tmp);
  return 0;
}

static void free_view(view_cache *vc) {
  free(vc->g);
  free(vc->order);
}

/* One pixel's walk through Eq. 1.
 *
 * Decisions close to a cutoff (q vs q_max, sigma vs alpha_min, T' vs t_min)
 * can go either way in a binary32 renderer, so each one taken within a window
 * of its threshold is "flagged" and numbered in the order met; bit d of
 * flip_mask inverts the d-th flagged decision. flip_mask = 0 is the plain FP64
 * walk; enumerating masks gives every result a renderer that rounds
 * differently near those thresholds may legitimately produce.
 * Windows: W_Q absolute on q, W_A relative on sigma, W_T relative on T'.
 * When rec != NULL it records, per added Gaussian, (index, sigma, G, T before,
 * clamped, dx, dy). Returns the number of Gaussians added. */
#define W_Q 2e-3
#define W_A 1e-3
#define W_T 1e-4
#define W_CLAMP 1e-5
typedef struct {
  int32_t i;
  int clamped;
  double sigma, G, T, dx, dy, color;
} contrib;

/* Colour of Gaussian g at a pixel: Yp = Y(pixel ray) with per-pixel
 * directions, NULL otherwise. */
static double pair_color(const g64 *g, const double *Yp, int kL) {
  if (!Yp || !g->has_dir) return g->color;
  double z = g->a;
  for (int m = 0; m < kL; ++m) z += Yp[m] * g->h[m];
  return sigmoid(z);
}

static int64_t walk_pixel(const view_cache *vc, const or_config *cfg, double px,
                          double py, const double *Yp, int kL, unsigned flip_mask,
                          double *C_out, double *T_out, int32_t *last_out,
                          int32_t *flags_out, int32_t *nflag_out, contrib *rec) {
  double T = 1.0, C = 0.0;
  int32_t last = -1, flags = vc->near_cull ? OR_NEAR_CULL : 0;
  int nflag = 0;
  int64_t cnt = 0;
#define DECIDE(natural) \
  ((nflag < 31 && ((flip_mask >> nflag) & 1u)) ? (nflag++, !(natural)) : (nflag++, (natural)))
  for (int64_t j = 0; j < vc->n_order; ++j) {
    const g64 *g = &vc->g[vc->order[j]];
    double dx = g->u - px, dy = g->v - py;
    double q = g->conic[0] * dx * dx + 2 * g->conic[1] * dx * dy + g->conic[2] * dy * dy;
    int keep_q = q <= cfg->q_max && q >= 0;
    if (fabs(q - cfg->q_max) < W_Q && q >= 0) {
      /* the decision only matters if the Gaussian would then pass alpha_min */
      double s_in = fmin(cfg->alpha_max, g->alpha * exp(-0.5 * q));
      if (s_in >= cfg->alpha_min * (1 - W_A)) {
        flags |= OR_NEAR_Q;
        keep_q = DECIDE(keep_q);
      }
    }
    if (!keep_q) continue;
    double G = exp(-0.5 * q);
    double a = g->alpha * G;
    if (fabs(a - cfg->alpha_max) < W_CLAMP) flags |= OR_NEAR_CLAMP;
    int clamped = a > cfg->alpha_max;
    double sigma = clamped ? cfg->alpha_max : a;
    int keep_a = sigma >= cfg->alpha_min;
    if (fabs(sigma - cfg->alpha_min) < W_A * cfg->alpha_min) {
      flags |= OR_NEAR_ALPHA_MIN;
      keep_a = DECIDE(keep_a);
    }
    if (!keep_a) continue;
    double Tn = T * (1 - sigma);
    int stop = Tn < cfg->t_min;
    if (fabs(Tn - cfg->t_min) < W_T * cfg->t_min) {
      flags |= OR_NEAR_TMIN;
      stop = DECIDE(stop);
    }
    if (stop) break;
    const double color = pair_color(g, Yp, kL);
    if (rec) {
      rec[cnt].i = vc->order[j];
      rec[cnt].clamped = clamped;
      rec[cnt].sigma = sigma;
      rec[cnt].G = G;
      rec[cnt].T = T;
      rec[cnt].dx = dx;
      rec[cnt].dy = dy;
      rec[cnt].color = color;
    }
    C += color * sigma * T;
    T = Tn;
    last = vc->order[j];
    ++cnt;
  }
#undef DECIDE
  if (C_out) *C_out = C;
  if (T_out) *T_out = T;
  if (last_out) *last_out = last;
  if (flags_out) *flags_out = flags;
  if (nflag_out) *nflag_out = nflag;
  return cnt;
}

/* Unit direction (world frame) of the ray from the source through the centre
 * (px, py) of a detector pixel of view v: in camera coordinates the pixel
 * sits at rc = ((px - c_u) pitch_u, (py - c_v) pitch_v, sdd); the world
 * direction is W^T rc. Also returns rc and |W^T rc| for the backward pass. */
static void pixel_ray(const or_views *vw, int64_t v, double px, double py,
                      double rc[3], double dhat[3], double *dnorm) {
  const double *T = vw->world_to_cam + 12 * v;
  const double *dp = vw->detector + 5 * v;
  rc[0] = (px - (0.5 * vw->width + dp[3])) * dp[1];
  rc[1] = (py - (0.5 * vw->height + dp[4])) * dp[2];
  rc[2] = dp[0];
  double d[3];
  for (int c = 0; c < 3; ++c) d[c] = T[c] * rc[0] + T[4 + c] * rc[1] + T[8 + c] * rc[2];
  *dnorm = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int c = 0; c < 3; ++c) dhat[c] = d[c] / *dnorm;
}

/* Pixel list helpers: either explicit (v,row,col) triples or all pixels. */
static void pixel_at(const or_views *vw, const int32_t *pix, int64_t p,
                     int64_t *v, int64_t *row, int64_t *col) {
  if (pix) {
    *v = pix[3 * p]; *row = pix[3 * p + 1]; *col = pix[3 * p + 2];
  } else {
    int64_t hw = (int64_t)vw->height * vw->width;
    *v = p / hw;
    *row = (p % hw) / vw->width;
    *col = p % vw->width;
  }
}

static int check_args(const or_scene *sc, const or_views *vw, int64_t n_pix,
                      const int32_t *pix) {
  if (!sc || !vw) return 1;
  if (sc->k < 1 || sc->k > KMAX || sc->L < 1 || sc->L > LMAX) return 1;
  if (sc->n_iso < 0 || sc->n_iso > sc->n) return 1;
  if (!pix && n_pix != (int64_t)vw->n_views * vw->height * vw->width) return 1;
  for (int64_t p = 0; pix && p < n_pix; ++p)
    if (pix[3 * p] < 0 || pix[3 * p] >= vw->n_views || pix[3 * p + 1] < 0 ||
        pix[3 * p + 1] >= vw->height || pix[3 * p + 2] < 0 || pix[3 * p + 2] >= vw->width)
      return 1;
  return 0;
}

#ifdef _OPENMP
#include <omp.h>
#define SET_THREADS(nt) do { if ((nt) > 0) omp_set_num_threads(nt); } while (0)
#else
#define SET_THREADS(nt) do { (void)(nt); } while (0)
#endif

int or_project(const or_scene *sc, const or_views *vw, const or_config *cfg,
               double *out) {
  if (check_args(sc, vw, (int64_t)vw->n_views * vw->height * vw->width, NULL)) return 1;
  for (int64_t v = 0; v < vw->n_views; ++v)
    for (int64_t i = 0; i < sc->n; ++i) {
      g64 g;
      project64(sc, vw, cfg, v, i, &g);
      double *o = out + 9 * (v * sc->n + i);
      o[0] = g.u; o[1] = g.v; o[2] = g.conic[0]; o[3] = g.conic[1]; o[4] = g.conic[2];
      o[5] = g.alpha; o[6] = g.color; o[7] = g.xc[2]; o[8] = g.valid;
    }
  return 0;
}

int or_render(const or_scene *sc, const or_views *vw, const or_config *cfg,
              const float *depth32, int64_t n_pix, const int32_t *pix,
              const uint32_t *flip_masks, double *image, double *t_final,
              int32_t *last_id, int32_t *n_contrib, int32_t *flags,
              int32_t *n_flagged, int n_threads) {
  if (check_args(sc, vw, n_pix, pix)) return 1;
  SET_THREADS(n_threads);
  const int kL = sc->L * (sc->L + 2);
  for (int64_t v = 0; v < vw->n_views; ++v) {
    view_cache vc;
    if (build_view(sc, vw, cfg, depth32, v, &vc)) return 2;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < n_pix; ++p) {
      int64_t pv, row, col;
      pixel_at(vw, pix, p, &pv, &row, &col);
      if (pv != v) continue;
      double C, T;
      int32_t last, fl, nf;
      unsigned mask = flip_masks ? flip_masks[p] : 0u;
      double Yp[KLMAX], rc[3], dh[3], dn;
      if (sc->per_pixel) {
        pixel_ray(vw, v, col + 0.5, row + 0.5, rc, dh, &dn);
        real_sh(sc->L, dh, Yp, NULL);
      }
      int64_t cnt = walk_pixel(&vc, cfg, col + 0.5, row + 0.5, sc->per_pixel ? Yp : NULL, kL,
                               mask, &C, &T, &last, &fl, &nf, NULL);
      if (image) image[p] = C;
      if (t_final) t_final[p] = T;
      if (last_id) last_id[p] = last;
      if (n_contrib) n_contrib[p] = (int32_t)cnt;
      if (flags) flags[p] = fl;
      if (n_flagged) n_flagged[p] = nf;
    }
    free_view(&vc);
  }
  return 0;
}

int or_render_backward(const or_scene *sc, const or_views *vw,
                       const or_config *cfg, const float *depth32,
                       int64_t n_pix, const int32_t *pix, const uint32_t *flip_masks,
                       const double *dL_dC,
                       double *g_means, double *g_log_scales, double *g_quats,
                       double *g_opacity_logits, double *g_feat,
                       double *g_b_iso, double *g_B_dir, double *g_pose,
                       double *g_2d, int n_threads) {
  if (check_args(sc, vw, n_pix, pix)) return 1;
  SET_THREADS(n_threads);
  const int64_t n = sc->n;
  const int k = sc->k;
  const int kL = sc->L * (sc->L + 2), G2 = 7 + kL;
  const int64_t V = vw->n_views;
  /* 2D gradients per (view, Gaussian) */
  double *g2 = (double *)calloc((size_t)(V * n * G2 + 1), sizeof(double));
  /* pose gradient through the per-pixel ray directions */
  double *pose_ray = (double *)calloc((size_t)(V * 12 + 1), sizeof(double));
  if (!g2 || !pose_ray) { free(g2); free(pose_ray); return 2; }
  for (int64_t v = 0; v < vw->n_views; ++v) {
    view_cache vc;
    if (build_view(sc, vw, cfg, depth32, v, &vc)) { free(g2); return 2; }
    int fail = 0;
#pragma omp parallel
    {
      contrib *rec = (contrib *)malloc(sizeof(contrib) * (size_t)(vc.n_order + 1));
      if (!rec) {
#pragma omp atomic write
        fail = 1;
      }
#pragma omp for schedule(dynamic, 16)
      for (int64_t p = 0; p < n_pix; ++p) {
        if (!rec) continue;
        int64_t pv, row, col;
        pixel_at(vw, pix, p, &pv, &row, &col);
        if (pv != v || dL_dC[p] == 0.0) continue;
        double Yp[KLMAX], dYp[KLMAX][3], rc[3], dhat[3], dn, gY[KLMAX] = {0};
        if (sc->per_pixel) {
          pixel_ray(vw, v, col + 0.5, row + 0.5, rc, dhat, &dn);
          real_sh(sc->L, dhat, Yp, dYp);
        }
        /* the same walk as the forward, with this pixel's flipped decisions */
        const unsigned mask = flip_masks ? flip_masks[p] : 0u;
        int64_t cnt = walk_pixel(&vc, cfg, col + 0.5, row + 0.5, sc->per_pixel ? Yp : NULL, kL,
                                 mask, NULL, NULL, NULL, NULL, NULL, rec);
        double gC = dL_dC[p];
        /* S = sum over later Gaussians of c sigma T (suffix sum) */
        double S = 0.0;
        for (int64_t j = cnt - 1; j >= 0; --j) {
          const contrib *r = &rec[j];
          const g64 *g = &vc.g[r->i];
          const double c = r->color;
          double dC_dc = r->sigma * r->T;
          double dC_dsigma = c * r->T - S / (1 - r->sigma);
          S += c * r->sigma * r->T;
          double gs = gC * dC_dsigma;
          /* colour logit z = a + Y(d) . h */
          const double dz = gC * dC_dc * c * (1 - c);
          double gg[7 + KLMAX] = {0, 0, 0, 0, 0, 0, dz};
          if (g->has_dir) {
            const double *Y = sc->per_pixel ? Yp : g->Y;
            for (int m = 0; m < kL; ++m) gg[7 + m] = dz * Y[m];
            if (sc->per_pixel)
              for (int m = 0; m < kL; ++m) gY[m] += dz * g->h[m];
          }
          if (!r->clamped) {
            gg[5] = gs * r->G;
            double gq = gs * g->alpha * r->G * -0.5;
            double dx = r->dx, dy = r->dy;
            gg[0] = gq * (2 * g->conic[0] * dx + 2 * g->conic[1] * dy);
            gg[1] = gq * (2 * g->conic[1] * dx + 2 * g->conic[2] * dy);
            gg[2] = gq * dx * dx;
            gg[3] = gq * 2 * dx * dy;
            gg[4] = gq * dy * dy;
          }
          double *dst = g2 + G2 * (v * n + r->i);
          for (int e = 0; e < G2; ++e) {
#pragma omp atomic
            dst[e] += gg[e];
          }
        }
        if (sc->per_pixel && cnt > 0) {
          /* Y(dhat), dhat = d / |d|, d = W^T rc: dL/dW[r][c] = rc[r] dL/dd[c] */
          double ddh[3] = {0, 0, 0};
          for (int m = 0; m < kL; ++m)
            for (int c3 = 0; c3 < 3; ++c3) ddh[c3] += gY[m] * dYp[m][c3];
          double dot = ddh[0] * dhat[0] + ddh[1] * dhat[1] + ddh[2] * dhat[2];
          for (int r = 0; r < 3; ++r)
            for (int c3 = 0; c3 < 3; ++c3) {
#pragma omp atomic
              pose_ray[12 * v + 4 * r + c3] += rc[r] * (ddh[c3] - dhat[c3] * dot) / dn;
            }
        }
      }
      free(rec);
    }
    free_view(&vc);
    if (fail) { free(g2); free(pose_ray); return 2; }
  }
  if (g_2d) memcpy(g_2d, g2, sizeof(double) * (size_t)(V * n * G2));

  /* chain rule per Gaussian (summed over views) and per view (over Gaussians) */
  double *pose = pose_ray;
  double *gb = (double *)calloc((size_t)((1 + kL) * k), sizeof(double));
  if (!gb) { free(g2); free(pose); return 2; }
#pragma omp parallel
  {
    double *pose_l = (double *)calloc((size_t)(V * 12 + 1), sizeof(double));
    double *gb_l = (double *)calloc((size_t)((1 + kL) * k), sizeof(double));
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      grad_acc acc;
      memset(&acc, 0, sizeof acc);
      for (int64_t v = 0; v < V; ++v) {
        const double *gg = g2 + G2 * (v * n + i);
        int any = 0;
        for (int e = 0; e < G2; ++e) any |= gg[e] != 0.0;
        if (!any) continue;
        g64 g;
        project64(sc, vw, cfg, v, i, &g);
        memset(acc.pose, 0, sizeof acc.pose);
        backprop64(sc, i, &g, gg, &acc);
        for (int c = 0; c < 12; ++c) pose_l[12 * v + c] += acc.pose[c];
      }
      if (g_means) for (int c = 0; c < 3; ++c) g_means[3 * i + c] = acc.mu[c];
      if (g_log_scales) for (int c = 0; c < 3; ++c) g_log_scales[3 * i + c] = acc.ls[c];
      if (g_quats) for (int c = 0; c < 4; ++c) g_quats[4 * i + c] = acc.q[c];
      if (g_opacity_logits) g_opacity_logits[i] = acc.logit;
      if (g_feat) for (int c = 0; c < k; ++c) g_feat[(int64_t)k * i + c] = acc.f[c];
      for (int c = 0; c < k; ++c) gb_l[c] += acc.b_iso[c];
      for (int c = 0; c < kL * k; ++c) gb_l[k + c] += acc.B_dir[c];
    }
#pragma omp critical
    {
      for (int64_t c = 0; c < V * 12; ++c) pose[c] += pose_l[c];
      for (int c = 0; c < (1 + kL) * k; ++c) gb[c] += gb_l[c];
    }
    free(pose_l);
    free(gb_l);
  }
  if (g_pose) memcpy(g_pose, pose, sizeof(double) * (size_t)(V * 12));
  if (g_b_iso) memcpy(g_b_iso, gb, sizeof(double) * (size_t)k);
  if (g_B_dir) memcpy(g_B_dir, gb + k, sizeof(double) * (size_t)(kL * k));
  free(pose);
  free(gb);
  free(g2);
  return 0;
}

int or_count_inside(const or_scene *sc, const or_views *vw, const or_config *cfg,
                    const float *depth32, int64_t n_pix, const int32_t *pix,
                    int32_t *n_inside, int n_threads) {
  if (check_args(sc, vw, n_pix, pix) || !n_inside) return 1;
  SET_THREADS(n_threads);
  for (int64_t v = 0; v < vw->n_views; ++v) {
    view_cache vc;
    if (build_view(sc, vw, cfg, depth32, v, &vc)) return 2;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < n_pix; ++p) {
      int64_t pv, row, col;
      pixel_at(vw, pix, p, &pv, &row, &col);
      if (pv != v) continue;
      double px = col + 0.5, py = row + 0.5;
      int32_t cnt = 0;
      for (int64_t j = 0; j < vc.n_order; ++j) {
        const g64 *g = &vc.g[vc.order[j]];
        double dx = g->u - px, dy = g->v - py;
        double q = g->conic[0] * dx * dx + 2 * g->conic[1] * dx * dy + g->conic[2] * dy * dy;
        cnt += (q <= cfg->q_max && q >= 0);
      }
      n_inside[p] = cnt;
    }
    free_view(&vc);
  }
  return 0;
}
