// preprocess.cu -- per (view, Gaussian) projection, key emission, and the
// backward chain from 2D gradients to Gaussian, basis and pose gradients.
//
// Forward (K1): for each Gaussian, once: Sigma = R S S^T R^T from the scale
// and quaternion (Sec. 3.1), alpha = sigmoid(logit), and the view-independent
// part of the radiosity (Eq. 3); then for each view: the perspective
// projection of the mean, the Jacobian projection of Sigma (the image-plane
// projections mu-hat, Sigma-hat of Eq. 1), its conic, the direction-dependent
// radiosity at the source-to-mean direction (Eq. 3), and the screen tiles
// reached by the q <= q_max ellipse. One thread handles one Gaussian for all
// views, so a Gaussian is read from HBM once per batch of views.
//
// The steps that decide integers (culling, tile rectangle, depth key) use
// one correctly rounded binary32 operation each, in the fixed order G1..G15
// (G1 scales; G2-G3 normalised quaternion and rotation; G4-G5 the 3D
// covariance; then per view G6 the camera transform, G7 the depth test, G8 the
// projection of the mean, G9-G12 the Jacobian and the 2D covariance, G13 its
// determinant, G14 the ellipse extents, G15 the tile rectangle), so they can
// be compared bit for bit with a CPU reference that follows the same
// definition.
#include "ddgs_internal.cuh"

namespace ddgs {
namespace {

// exp in binary32 from correctly rounded operations only: Cody & Waite (1980)
// reduction x = k ln2 + r with ln 2 split into a short head and a tail, then the
// Taylor series of e^r to degree 7 (coefficients 1/n!), then an exact scaling
// by 2^k built from the exponent field.
__device__ __forceinline__ float exp32(float x) {
  if (x != x) return x;
  if (x > 88.0f) return __int_as_float(0x7f800000);
  if (x < -87.0f) return 0.0f;
  const float kf = rintf(mulr(x, 1.44269504f));
  const int k = (int)kf;
  const float r = subr(subr(x, mulr(kf, 0.693359375f)), mulr(kf, -2.12194440e-4f));
  float p = (float)(1.0 / 5040.0);
  p = addr(mulr(p, r), (float)(1.0 / 720.0));
  p = addr(mulr(p, r), (float)(1.0 / 120.0));
  p = addr(mulr(p, r), (float)(1.0 / 24.0));
  p = addr(mulr(p, r), (float)(1.0 / 6.0));
  p = addr(mulr(p, r), 0.5f);
  p = addr(mulr(p, r), 1.0f);
  p = addr(mulr(p, r), 1.0f);
  return mulr(p, __int_as_float((k + 127) << 23));
}

// Opacity and radiosity sigmoids: they reach the image and the gradients only
// (never the binning), so the approximate reciprocal serves.
__device__ __forceinline__ float sigmoidf_(float x) { return rcp_approx(1.0f + __expf(-x)); }

// View-independent geometry of one Gaussian (steps G1-G5).
struct GaussGeom {
  float s[3], qn[4], qnorm, R[9], M[9], S[6];  // S: xx, xy, xz, yy, yz, zz
};

__device__ __forceinline__ void gauss_geom(const float *ls, const float *q, GaussGeom &g) {
  // G1
  g.s[0] = exp32(ls[0]); g.s[1] = exp32(ls[1]); g.s[2] = exp32(ls[2]);
  // G2
  float w = q[0], x = q[1], y = q[2], z = q[3];
  float n2 = addr(addr(addr(mulr(w, w), mulr(x, x)), mulr(y, y)), mulr(z, z));
  float rn = sqrtr(n2);
  g.qnorm = rn;
  w = divr(w, rn); x = divr(x, rn); y = divr(y, rn); z = divr(z, rn);
  g.qn[0] = w; g.qn[1] = x; g.qn[2] = y; g.qn[3] = z;
  // G3
  float xx = mulr(x, x), yy = mulr(y, y), zz = mulr(z, z);
  float xy = mulr(x, y), xz = mulr(x, z), yz = mulr(y, z);
  float wx = mulr(w, x), wy = mulr(w, y), wz = mulr(w, z);
  float *R = g.R;
  R[0] = subr(1.0f, mulr(2.0f, addr(yy, zz)));
  R[1] = mulr(2.0f, subr(xy, wz));
  R[2] = mulr(2.0f, addr(xz, wy));
  R[3] = mulr(2.0f, addr(xy, wz));
  R[4] = subr(1.0f, mulr(2.0f, addr(xx, zz)));
  R[5] = mulr(2.0f, subr(yz, wx));
  R[6] = mulr(2.0f, subr(xz, wy));
  R[7] = mulr(2.0f, addr(yz, wx));
  R[8] = subr(1.0f, mulr(2.0f, addr(xx, yy)));
  // G4
  float *M = g.M;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    M[3 * r + 0] = mulr(R[3 * r + 0], g.s[0]);
    M[3 * r + 1] = mulr(R[3 * r + 1], g.s[1]);
    M[3 * r + 2] = mulr(R[3 * r + 2], g.s[2]);
  }
  // G5
  g.S[0] = dot3r(M[0], M[1], M[2], M[0], M[1], M[2]);
  g.S[1] = dot3r(M[0], M[1], M[2], M[3], M[4], M[5]);
  g.S[2] = dot3r(M[0], M[1], M[2], M[6], M[7], M[8]);
  g.S[3] = dot3r(M[3], M[4], M[5], M[3], M[4], M[5]);
  g.S[4] = dot3r(M[3], M[4], M[5], M[6], M[7], M[8]);
  g.S[5] = dot3r(M[6], M[7], M[8], M[6], M[7], M[8]);
}

__device__ __forceinline__ float sym(const float *S, int r, int c) {
  // symmetric 3x3 stored as xx, xy, xz, yy, yz, zz
  const int idx[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
  return S[idx[3 * r + c]];
}

// Per-view projection (steps G6-G13) with everything the backward needs.
struct ViewProj {
  float xc[3], xz, yz, u, v, j00, j11, j02, j12, A[6], cov[3], det;
  bool valid;
};

__device__ __forceinline__ void view_proj(const float mu[3], const float S[6], const ViewConst &vc,
                                          float dilation, float near_plane, ViewProj &p) {
  // G6
#pragma unroll
  for (int r = 0; r < 3; ++r)
    p.xc[r] = addr(dot3r(vc.W[3 * r], vc.W[3 * r + 1], vc.W[3 * r + 2], mu[0], mu[1], mu[2]), vc.t[r]);
  const float z = p.xc[2];
  // G7
  p.valid = (z > near_plane && z < vc.sdd);
  if (!p.valid) return;
  // G8
  p.xz = divr(p.xc[0], z);
  p.yz = divr(p.xc[1], z);
  p.u = addr(mulr(vc.fu, p.xz), vc.cu);
  p.v = addr(mulr(vc.fv, p.yz), vc.cv);
  // G9
  p.j00 = divr(vc.fu, z);
  p.j11 = divr(vc.fv, z);
  p.j02 = -mulr(p.j00, p.xz);
  p.j12 = -mulr(p.j11, p.yz);
  // G10: A = J W (rows 0 and 1)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    p.A[k] = addr(mulr(p.j00, vc.W[k]), mulr(p.j02, vc.W[6 + k]));
    p.A[3 + k] = addr(mulr(p.j11, vc.W[3 + k]), mulr(p.j12, vc.W[6 + k]));
  }
  // G11: B = A Sigma
  float B[6];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      B[3 * r + k] = dot3r(p.A[3 * r], p.A[3 * r + 1], p.A[3 * r + 2], sym(S, 0, k), sym(S, 1, k),
                           sym(S, 2, k));
  // G12
  p.cov[0] = addr(dot3r(B[0], B[1], B[2], p.A[0], p.A[1], p.A[2]), dilation);
  p.cov[1] = dot3r(B[0], B[1], B[2], p.A[3], p.A[4], p.A[5]);
  p.cov[2] = addr(dot3r(B[3], B[4], B[5], p.A[3], p.A[4], p.A[5]), dilation);
  // G13
  p.det = subr(mulr(p.cov[0], p.cov[2]), mulr(p.cov[1], p.cov[1]));
  p.valid = p.det > 0.0f;
}

// The same projection for the backward chain, in plain FP32 with contracted
// multiply-adds and one approximate reciprocal of z: no integer decision
// depends on it, and a record reaches the backward only if the forward's
// exact chain kept it (its 2D gradient is non-zero), so it is not culled here.
__device__ __forceinline__ void view_proj_grad(const float mu[3], const float S[6], const ViewConst &vc,
                                               float dilation, ViewProj &p) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
    p.xc[r] = fmaf(vc.W[3 * r + 2], mu[2], fmaf(vc.W[3 * r + 1], mu[1], fmaf(vc.W[3 * r], mu[0], vc.t[r])));
  const float iz = rcp_approx(p.xc[2]);
  p.xz = p.xc[0] * iz;
  p.yz = p.xc[1] * iz;
  p.j00 = vc.fu * iz;
  p.j11 = vc.fv * iz;
  p.j02 = -p.j00 * p.xz;
  p.j12 = -p.j11 * p.yz;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    p.A[k] = fmaf(p.j02, vc.W[6 + k], p.j00 * vc.W[k]);
    p.A[3 + k] = fmaf(p.j12, vc.W[6 + k], p.j11 * vc.W[3 + k]);
  }
  float B[6];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      B[3 * r + k] = fmaf(p.A[3 * r + 2], sym(S, 2, k),
                          fmaf(p.A[3 * r + 1], sym(S, 1, k), p.A[3 * r] * sym(S, 0, k)));
  p.cov[0] = fmaf(B[2], p.A[2], fmaf(B[1], p.A[1], fmaf(B[0], p.A[0], dilation)));
  p.cov[1] = fmaf(B[2], p.A[5], fmaf(B[1], p.A[4], B[0] * p.A[3]));
  p.cov[2] = fmaf(B[5], p.A[5], fmaf(B[4], p.A[4], fmaf(B[3], p.A[3], dilation)));
  p.det = fmaf(p.cov[0], p.cov[2], -p.cov[1] * p.cov[1]);
  p.valid = true;
}

// G14-G15: inclusive tile rectangle; returns tiles touched (0 = none).
__device__ __forceinline__ uint32_t tile_rect(const ViewProj &p, float q_max, int H, int W, int tile,
                                              int &tx0, int &ty0, int &tx1, int &ty1) {
  float ex = sqrtr(mulr(q_max, p.cov[0])), ey = sqrtr(mulr(q_max, p.cov[2]));
  ex = addr(mulr(ex, 1.0009765625f), 0.0009765625f);
  ey = addr(mulr(ey, 1.0009765625f), 0.0009765625f);
  if (p.u != p.u || p.v != p.v || ex != ex || ey != ey) return 0;
  float xlo = ceilf(subr(subr(p.u, ex), 0.5f)), xhi = floorf(subr(addr(p.u, ex), 0.5f));
  float ylo = ceilf(subr(subr(p.v, ey), 0.5f)), yhi = floorf(subr(addr(p.v, ey), 0.5f));
  xlo = fmaxf(xlo, 0.0f); xhi = fminf(xhi, (float)(W - 1));
  ylo = fmaxf(ylo, 0.0f); yhi = fminf(yhi, (float)(H - 1));
  if (xlo > xhi || ylo > yhi) return 0;
  tx0 = (int)xlo / tile; tx1 = (int)xhi / tile;
  ty0 = (int)ylo / tile; ty1 = (int)yhi / tile;
  return (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
}

__device__ __forceinline__ void load_view(const float *pose, const float *det, const ViewTab &vt,
                                          ViewConst &vc) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    vc.W[3 * r] = pose[4 * r];
    vc.W[3 * r + 1] = pose[4 * r + 1];
    vc.W[3 * r + 2] = pose[4 * r + 2];
    vc.t[r] = pose[4 * r + 3];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) vc.wt[c] = vc.W[c] * vc.t[0] + vc.W[3 + c] * vc.t[1] + vc.W[6 + c] * vc.t[2];
  vc.sdd = det[0];
  vc.fu = divr(det[0], det[1]);
  vc.fv = divr(det[0], det[2]);
  vc.cu = addr(mulr(0.5f, (float)vt.W), det[3]);
  vc.cv = addr(mulr(0.5f, (float)vt.H), det[4]);
  vc.H = vt.H;
  vc.Wd = vt.W;
  vc.tiles_x = vt.tiles_x;
  vc.tile_base = vt.tile_base;
  vc.rec_off = vt.rec_off;
}

// Feature row of the request's local Gaussian l.
__device__ __forceinline__ void load_feat(const float *feat_iso, const void *feat_dir, int bf16,
                                          const ReqTab &rq, int64_t l, float f[K]) {
  if (l < rq.n_iso) {
    const float4 *p = reinterpret_cast<const float4 *>(feat_iso + (rq.iso_row + l) * K);
    float4 a = p[0], b = p[1];
    f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w; f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
  } else if (bf16) {
    const uint4 raw = *(reinterpret_cast<const uint4 *>(feat_dir) + (rq.dir_row + l - rq.n_iso));
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      f[2 * k] = __uint_as_float(w[k] << 16);
      f[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
  } else {
    const float4 *p = reinterpret_cast<const float4 *>(static_cast<const float *>(feat_dir) +
                                                       (rq.dir_row + l - rq.n_iso) * K);
    float4 a = p[0], b = p[1];
    f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w; f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
  }
}

// ---- generic radiosity: runtime feature dimension k <= 32, degree L <= 3 ----
constexpr int KG = 32;   // largest feature dimension of the generic kernels
constexpr int KLG = 15;  // largest k_L = L(L+2) (L = 3)

__device__ __forceinline__ float load_feat1(const float *feat_iso, const void *feat_dir, int bf16,
                                            const ReqTab &rq, int64_t l, int K, int k) {
  if (l < rq.n_iso) return feat_iso[(rq.iso_row + l) * K + k];
  const int64_t idx = (rq.dir_row + l - rq.n_iso) * K + k;
  if (bf16) {
    const unsigned short u = static_cast<const unsigned short *>(feat_dir)[idx];
    return __uint_as_float((uint32_t)u << 16);
  }
  return static_cast<const float *>(feat_dir)[idx];
}

// Real spherical harmonics of degrees 1..L for a unit direction, Y_lm =
// (-1)^m N_lm sqrt(2)^[m != 0] D^|m| P_l(z) * (Re (x+iy)^|m| for m > 0, 1 for
// m = 0, Im (x+iy)^|m| for m < 0), N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!),
// ordered (l, m = -l..l). Row j of the table holds m and the coefficients of
// the z polynomial; each block builds it from these definitions.
struct ShTable {
  float c[KLG][4];
  int m[KLG];
};

__device__ void sh_table_row(int j, ShTable &t) {
  int l = 1;
  while ((l + 1) * (l + 1) - 1 <= j) ++l;
  const int m = j - (l * l - 1) - l, am = m < 0 ? -m : m;
  double p0[4] = {1, 0, 0, 0}, p1[4] = {0, 1, 0, 0};
  for (int n = 1; n < l; ++n) {  // (n+1) P_{n+1} = (2n+1) z P_n - n P_{n-1}
    double p2[4];
    for (int i = 0; i < 4; ++i) p2[i] = ((2 * n + 1) * (i ? p1[i - 1] : 0.0) - n * p0[i]) / (n + 1);
    for (int i = 0; i < 4; ++i) { p0[i] = p1[i]; p1[i] = p2[i]; }
  }
  double fl = 1, fh = 1;  // (l-|m|)!, (l+|m|)!
  for (int i = 2; i <= l - am; ++i) fl *= i;
  for (int i = 2; i <= l + am; ++i) fh *= i;
  const double norm = sqrt((2.0 * l + 1.0) / (4.0 * 3.14159265358979323846) * fl / fh) *
                      (am ? 1.4142135623730951 : 1.0) * ((am & 1) ? -1.0 : 1.0);
  for (int i = 0; i < 4; ++i) {
    double d = 0;
    if (i + am < 4) {
      d = p1[i + am];
      for (int q = 0; q < am; ++q) d *= (i + am - q);
    }
    t.c[j][i] = (float)(norm * d);
  }
  t.m[j] = m;
}

// Y[j] and, if dY is given, the derivative of Y[j] along x, y, z.
__device__ __forceinline__ void sh_eval(const ShTable &t, int kL, float x, float y, float z, float *Y,
                                        float (*dY)[3]) {
  const float re[4] = {1.f, x, x * x - y * y, x * (x * x - y * y) - y * (2.f * x * y)};
  const float im[4] = {0.f, y, 2.f * x * y, x * (2.f * x * y) + y * (x * x - y * y)};
#pragma unroll
  for (int j = 0; j < KLG; ++j) {
    if (j >= kL) break;
    const int m = t.m[j], am = m < 0 ? -m : m;
    const float *c = t.c[j];
    const float Q = fmaf(fmaf(fmaf(c[3], z, c[2]), z, c[1]), z, c[0]);
    float A = 1.f, dAx = 0.f, dAy = 0.f;
    if (m > 0) { A = re[am]; dAx = am * re[am - 1]; dAy = -am * im[am - 1]; }
    else if (m < 0) { A = im[am]; dAx = am * im[am - 1]; dAy = am * re[am - 1]; }
    Y[j] = Q * A;
    if (dY) {
      const float dQ = fmaf(fmaf(3.f * c[3], z, 2.f * c[2]), z, c[1]);
      dY[j][0] = Q * dAx;
      dY[j][1] = Q * dAy;
      dY[j][2] = dQ * A;
    }
  }
}

struct PreArgs {
  const float *means, *log_scales, *quats, *logits, *feat_iso;
  const void *feat_dir;
  int feat_dir_bf16;
  const float *b_iso, *B_dir, *world_to_cam, *detector;
  float dilation, near_plane, q_max;
  RenderShape s;
  int K, L;          // feature dimension and harmonic degree
  int entangled;     // every Gaussian carries both terms of Eq. 3
  int per_pixel;     // Y at the pixel rays: write (a, h) to rec2 instead of a colour
  float4 *rec, *rec2;  // rec: two float4 per record
  uint4 *bin_info;  // (rect lo, rect hi, depth bits, tiles touched)
  uint32_t *blk_total;
  unsigned long long *t0;  // batch start (min over blocks of %globaltimer), or null
  int32_t *status;         // device status word: ST_NONFINITE is or-ed in
};

// A parameter that is NaN or +-Inf (fitting by gradient descent, Sec. 3.1, is
// where such values arise). The kernels keep going -- a NaN depth or
// determinant is culled by the binning's comparisons, a NaN opacity or colour
// reaches the image -- and the status word reports it.
__device__ __forceinline__ bool nonfinite(float x) { return !(fabsf(x) <= 3.402823466e38f); }

// One atomic per warp that saw a non-finite value.
__device__ __forceinline__ void flag_nonfinite(bool bad, int32_t *status) {
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0 && status)
    atomicOr(status, ST_NONFINITE);
}

__device__ __forceinline__ uint32_t block_sum_u32(uint32_t x, uint32_t *s_red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  if (lane == 0) s_red[wid] = x;
  __syncthreads();
  uint32_t t = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
  return t;
}

// The request of this block and the thread's local Gaussian index.
struct BlockReq {
  ReqTab rq;
  int r;
  int64_t l;
  bool live;
  __device__ __forceinline__ BlockReq(const RenderShape &s) {
    r = find_request(s.req, s.R, blockIdx.x);
    rq = s.req[r];
    l = ((int64_t)blockIdx.x - rq.blk_base) * PRE_THREADS + threadIdx.x;
    live = l < rq.n;
  }
};

// GEN = false: k = 8, L = 1 (the paper's evaluation setting) with vector
// feature loads; GEN = true: any k <= 32 and L <= 3, and the Eq. 3 variants.
// Generic radiosity: logit z = a + Y(d) . h, a = b_iso . f for a Gaussian with
// the isotropic term (every one of the isotropic range; all when entangled),
// h = B_dir f for one with the directional term. With per-pixel directions
// the record carries (a, h) and the rasteriser evaluates Y per pixel.
// Four resident blocks per SM for the k = 8, L = 1 instance (64 registers, a
// few bytes spilled: 0.38 -> 0.37 ms at 64 poses); the generic one keeps its
// registers.
template <bool GEN>
__global__ void __launch_bounds__(PRE_THREADS, GEN ? 1 : 4) preprocess_fwd_kernel(PreArgs a) {
  constexpr int KS = GEN ? KG : K, KLS = GEN ? KLG : 3;
  const int Kr = GEN ? a.K : K, kL = GEN ? a.L * (a.L + 2) : 3;
  __shared__ ViewConst sv[VIEW_CHUNK];
  __shared__ float s_b[KS], s_B[KLS * KS];
  __shared__ ShTable s_sh;
  __shared__ uint32_t s_red[PRE_THREADS / 32];
  const int tid = threadIdx.x;
  const RenderShape &s = a.s;
  const BlockReq br(s);
  const ReqTab &rq = br.rq;
  const bool live = br.live;
  const int64_t i = rq.g_off + br.l;  // index into the parameter arrays
  if (tid == 0 && a.t0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    atomicMin(a.t0, t);
  }
  bool bad = false;  // a non-finite input seen by this thread
  for (int e = tid; e < Kr; e += PRE_THREADS) {
    s_b[e] = a.b_iso[(int64_t)br.r * Kr + e];
    bad |= nonfinite(s_b[e]);
  }
  for (int e = tid; e < kL * Kr; e += PRE_THREADS) {
    s_B[e] = a.B_dir[(int64_t)br.r * kL * Kr + e];
    bad |= nonfinite(s_B[e]);
  }
  if (GEN && tid < kL) sh_table_row(tid, s_sh);
  __syncthreads();

  GaussGeom gg;
  float mu[3] = {0, 0, 0}, alpha = 0.f, c_iso = 0.f, h[KLS];
#pragma unroll
  for (int m = 0; m < KLS; ++m) h[m] = 0.f;
  bool is_dir = false, has_dir = false;
  if (live) {
    mu[0] = a.means[3 * i]; mu[1] = a.means[3 * i + 1]; mu[2] = a.means[3 * i + 2];
    float ls[3] = {a.log_scales[3 * i], a.log_scales[3 * i + 1], a.log_scales[3 * i + 2]};
    float4 q4 = reinterpret_cast<const float4 *>(a.quats)[i];
    float q[4] = {q4.x, q4.y, q4.z, q4.w};
    gauss_geom(ls, q, gg);
    const float logit = a.logits[i];
    alpha = sigmoidf_(logit);
    bad |= nonfinite(mu[0]) | nonfinite(mu[1]) | nonfinite(mu[2]) | nonfinite(ls[0]) |
           nonfinite(ls[1]) | nonfinite(ls[2]) | nonfinite(q[0]) | nonfinite(q[1]) |
           nonfinite(q[2]) | nonfinite(q[3]) | nonfinite(logit);
    is_dir = br.l >= rq.n_iso;
    if (!GEN) {
      float f[K];
      load_feat(a.feat_iso, a.feat_dir, a.feat_dir_bf16, rq, br.l, f);
#pragma unroll
      for (int k = 0; k < K; ++k) bad |= nonfinite(f[k]);
      if (!is_dir) {
        float zl = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) zl = fmaf(s_b[k], f[k], zl);
        c_iso = sigmoidf_(zl);
      } else {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          float acc = 0.f;
#pragma unroll
          for (int k = 0; k < K; ++k) acc = fmaf(s_B[m * K + k], f[k], acc);
          h[m] = acc;
        }
      }
    } else {
      // c_iso holds the isotropic logit a here
      const bool has_iso = !is_dir || a.entangled;
      has_dir = is_dir || a.entangled;
      float zl = 0.f;
      for (int k = 0; k < Kr; ++k) {
        const float fk = load_feat1(a.feat_iso, a.feat_dir, a.feat_dir_bf16, rq, br.l, Kr, k);
        bad |= nonfinite(fk);
        if (has_iso) zl = fmaf(s_b[k], fk, zl);
        if (has_dir) {
#pragma unroll
          for (int m = 0; m < KLS; ++m)
            if (m < kL) h[m] = fmaf(s_B[m * Kr + k], fk, h[m]);
        }
      }
      c_iso = zl;
    }
  }

  uint32_t total = 0;
  for (int v0 = 0; v0 < rq.n_views; v0 += VIEW_CHUNK) {
    const int nv = min(VIEW_CHUNK, rq.n_views - v0);
    __syncthreads();
    if (tid < nv) {
      const int v = rq.v_off + v0 + tid;
      load_view(a.world_to_cam + 12 * v, a.detector + 5 * v, s.view[v], sv[tid]);
      // the pose and detector of the view: checked by the request's first block
      if (blockIdx.x == rq.blk_base) {
#pragma unroll
        for (int e = 0; e < 12; ++e) bad |= nonfinite(a.world_to_cam[12 * v + e]);
#pragma unroll
        for (int e = 0; e < 5; ++e) bad |= nonfinite(a.detector[5 * v + e]);
      }
    }
    __syncthreads();
    if (!live) continue;
    for (int vv = 0; vv < nv; ++vv) {
      const ViewConst &vc = sv[vv];
      const int64_t rec = vc.rec_off + br.l;
      ViewProj p;
      view_proj(mu, gg.S, vc, a.dilation, a.near_plane, p);
      uint32_t tt = 0;
      int tx0 = 0, ty0 = 0, tx1 = -1, ty1 = -1;
      if (p.valid) tt = tile_rect(p, a.q_max, vc.H, vc.Wd, s.tile, tx0, ty0, tx1, ty1);
      const float depth = p.xc[2];
      a.bin_info[rec] = make_uint4((uint32_t)tx0 | ((uint32_t)ty0 << 16),
                                   (uint32_t)tx1 | ((uint32_t)ty1 << 16), __float_as_uint(depth), tt);
      if (tt == 0) continue;
      total += tt;
      // the record's conic feeds only the rasterisers: approximate reciprocal
      const float idet = rcp_approx(p.det);
      const float ca = p.cov[2] * idet, cb = -p.cov[1] * idet, cc = p.cov[0] * idet;
      float colour = c_iso;
      if (!GEN) {
        if (is_dir) {
          float d0 = mu[0] + vc.wt[0], d1 = mu[1] + vc.wt[1], d2 = mu[2] + vc.wt[2];
          float inv = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
          colour = sigmoidf_(SH_C1 * (-d1 * inv * h[0] + d2 * inv * h[1] - d0 * inv * h[2]));
        }
      } else if (a.per_pixel) {
        a.rec2[rec] = make_float4(c_iso, h[0], h[1], h[2]);  // L = 1: k_L = 3
        colour = 0.f;
      } else {
        float zl = c_iso;
        if (has_dir) {
          float d0 = mu[0] + vc.wt[0], d1 = mu[1] + vc.wt[1], d2 = mu[2] + vc.wt[2];
          float inv = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
          float Y[KLS];
          sh_eval(s_sh, kL, d0 * inv, d1 * inv, d2 * inv, Y, nullptr);
#pragma unroll
          for (int m = 0; m < KLS; ++m)
            if (m < kL) zl = fmaf(Y[m], h[m], zl);
        }
        colour = sigmoidf_(zl);
      }
      // the conic in the rasterisers' units, (a', 2b', c') (see eval_pair)
      a.rec[2 * rec] = make_float4(p.u, p.v, ca * CONIC_SCALE, (2.f * CONIC_SCALE) * cb);
      a.rec[2 * rec + 1] = make_float4(cc * CONIC_SCALE, alpha, colour, box_halfwidths(p.cov, a.q_max));
    }
  }
  flag_nonfinite(bad, a.status);
  uint32_t bt = block_sum_u32(total, s_red);
  if (tid == 0) a.blk_total[blockIdx.x] = bt;
}

// ---------------------------------------------------------------------------
// Backward (K8)
// ---------------------------------------------------------------------------

// 16-byte asynchronous global -> shared copies (the thread that issues them
// waits for them with cp_async_wait).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

struct PreBwdArgs {
  const float *means, *log_scales, *quats, *logits, *feat_iso;
  const void *feat_dir;
  int feat_dir_bf16;
  const float *b_iso, *B_dir, *world_to_cam, *detector;
  float dilation, near_plane;
  RenderShape s;
  int K, L;
  int entangled, per_pixel;
  float4 *grad2d;        // consumed records are cleared (left all-zero for the next backward)
  float4 *grad_h;        // per_pixel: dL/dh summed over pixels (cleared the same way)
  ddgs_grads out;
  int want_param, want_basis, want_pose;
};

// Sum 16 per-lane values over the warp with 15 shuffles; returns the
// component held by this lane (lanes with bit 0 clear and set both hold it).
__device__ __forceinline__ int warp_reduce16(float v[16]) {
  const int lane = threadIdx.x & 31;
  bool hi = lane & 16;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float send = hi ? v[k] : v[k + 8];
    float keep = hi ? v[k + 8] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  hi = lane & 8;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float send = hi ? v[k] : v[k + 4];
    float keep = hi ? v[k + 4] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  hi = lane & 4;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    float send = hi ? v[k] : v[k + 2];
    float keep = hi ? v[k + 2] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  hi = lane & 2;
  {
    float send = hi ? v[0] : v[1];
    float keep = hi ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

// POSE = true: only the pose gradient is wanted (a registration step,
// Sec. 4.3); the per-Gaussian accumulators are left out.
template <bool GEN, bool POSE = false>
__global__ void __launch_bounds__(PRE_THREADS, GEN ? 2 : 3) preprocess_bwd_kernel(PreBwdArgs a) {
  constexpr int KS = GEN ? KG : K, KLS = GEN ? KLG : 3;
  // views whose gradient records are in flight ahead of the one being used
  constexpr int AHEAD = GEN ? 2 : 4;
  const int Kr = GEN ? a.K : K, kL = GEN ? a.L * (a.L + 2) : 3;
  __shared__ ViewConst sv[VIEW_CHUNK];
  __shared__ float s_pose[VIEW_CHUNK][12];
  // each thread's own 2D-gradient records (and dL/dh with per-pixel rays) for
  // the next AHEAD views, copied asynchronously; only the copying thread reads
  // its slots, so its own wait on the copies is enough
  __shared__ float4 s_gr[AHEAD][GEN ? 3 : 2][PRE_THREADS];
  __shared__ float s_b[KS], s_B[KLS * KS], s_basis[(1 + KLS) * KS];
  __shared__ ShTable s_sh;
  const int tid = threadIdx.x, lane = tid & 31;
  const RenderShape &s = a.s;
  const BlockReq br(s);
  const ReqTab &rq = br.rq;
  const bool live = br.live;
  const int64_t i = rq.g_off + br.l;
  for (int e = tid; e < Kr; e += PRE_THREADS) s_b[e] = a.b_iso[(int64_t)br.r * Kr + e];
  for (int e = tid; e < kL * Kr; e += PRE_THREADS) s_B[e] = a.B_dir[(int64_t)br.r * kL * Kr + e];
  for (int e = tid; e < (1 + kL) * Kr; e += PRE_THREADS) s_basis[e] = 0.f;
  if (GEN && tid < kL) sh_table_row(tid, s_sh);
  __syncthreads();

  GaussGeom gg;
  constexpr int KF = GEN ? 1 : K;  // features kept in registers (fast path only)
  float mu[3] = {0, 0, 0}, alpha = 0.f, c_iso = 0.f, h[KLS], f[KF];
  bool is_dir = false, has_iso = false, has_dir = false;
#pragma unroll
  for (int k = 0; k < KF; ++k) f[k] = 0.f;
#pragma unroll
  for (int m = 0; m < KLS; ++m) h[m] = 0.f;
  if (live) {
    mu[0] = a.means[3 * i]; mu[1] = a.means[3 * i + 1]; mu[2] = a.means[3 * i + 2];
    float ls[3] = {a.log_scales[3 * i], a.log_scales[3 * i + 1], a.log_scales[3 * i + 2]};
    float4 q4 = reinterpret_cast<const float4 *>(a.quats)[i];
    float q[4] = {q4.x, q4.y, q4.z, q4.w};
    gauss_geom(ls, q, gg);
    alpha = sigmoidf_(a.logits[i]);
    is_dir = br.l >= rq.n_iso;
    if (!GEN) {
      load_feat(a.feat_iso, a.feat_dir, a.feat_dir_bf16, rq, br.l, f);
      if (!is_dir) {
        float zl = 0.f;
#pragma unroll
        for (int k = 0; k < KF; ++k) zl = fmaf(s_b[k], f[k], zl);
        c_iso = sigmoidf_(zl);
      } else {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          float acc = 0.f;
#pragma unroll
          for (int k = 0; k < KF; ++k) acc = fmaf(s_B[m * KF + k], f[k], acc);
          h[m] = acc;
        }
      }
    } else {
      // c_iso holds the isotropic logit a here
      has_iso = !is_dir || a.entangled;
      has_dir = is_dir || a.entangled;
      float zl = 0.f;
      for (int k = 0; k < Kr; ++k) {
        const float fk = load_feat1(a.feat_iso, a.feat_dir, a.feat_dir_bf16, rq, br.l, Kr, k);
        if (has_iso) zl = fmaf(s_b[k], fk, zl);
        if (has_dir) {
#pragma unroll
          for (int m = 0; m < KLS; ++m)
            if (m < kL) h[m] = fmaf(s_B[m * Kr + k], fk, h[m]);
        }
      }
      c_iso = zl;
    }
  }

  float dSig[6] = {0, 0, 0, 0, 0, 0}, dmu[3] = {0, 0, 0};
  float dz_iso = 0.f, dh[KLS], galpha = 0.f;
#pragma unroll
  for (int m = 0; m < KLS; ++m) dh[m] = 0.f;

  for (int v0 = 0; v0 < rq.n_views; v0 += VIEW_CHUNK) {
    const int nv = min(VIEW_CHUNK, rq.n_views - v0);
    __syncthreads();
    if (tid < nv) {
      const int v = rq.v_off + v0 + tid;
      load_view(a.world_to_cam + 12 * v, a.detector + 5 * v, s.view[v], sv[tid]);
    }
    for (int e = tid; e < nv * 12; e += blockDim.x) (&s_pose[0][0])[e] = 0.f;
    __syncthreads();
    const bool with_h = GEN && a.per_pixel;
    auto fetch = [&](int vv) {  // one commit group per view, empty past the chunk
      if (live && vv < nv) {
        const int64_t rec = sv[vv].rec_off + br.l;
        float4 *slot = &s_gr[vv % AHEAD][0][tid];
        cp_async16(slot, a.grad2d + 2 * rec);
        cp_async16(slot + PRE_THREADS, a.grad2d + 2 * rec + 1);
        if (GEN && with_h) cp_async16(slot + 2 * PRE_THREADS, a.grad_h + rec);
      }
      cp_async_commit();
    };
#pragma unroll
    for (int vv = 0; vv < AHEAD; ++vv) fetch(vv);
    for (int vv = 0; vv < nv; ++vv) {
      const ViewConst &vc = sv[vv];
      float dW[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, dt[3] = {0, 0, 0};
      bool any = false;
      cp_async_wait<AHEAD - 1>();  // this thread's copies of view vv have landed
      const float4 g0 = s_gr[vv % AHEAD][0][tid], g1 = s_gr[vv % AHEAD][1][tid];
      const float4 gh = with_h ? s_gr[vv % AHEAD][GEN ? 2 : 0][tid] : make_float4(0.f, 0.f, 0.f, 0.f);
      fetch(vv + AHEAD);  // reuses the slot just read
      if (live) {
        any = (g0.x != 0.f) | (g0.y != 0.f) | (g0.z != 0.f) | (g0.w != 0.f) | (g1.x != 0.f) |
              (g1.y != 0.f) | (g1.z != 0.f) | (gh.x != 0.f) | (gh.y != 0.f) | (gh.z != 0.f);
        if (any) {  // leave the record zero for the next backward
          const int64_t rec = vc.rec_off + br.l;
          a.grad2d[2 * rec] = make_float4(0.f, 0.f, 0.f, 0.f);
          a.grad2d[2 * rec + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (with_h) a.grad_h[rec] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        ViewProj p;
        if (any) view_proj_grad(mu, gg.S, vc, a.dilation, p);
        if (any) {
          const float gu = g0.x, gv = g0.y, gca = g0.z, gcb = g0.w, gcc = g1.x;
          if (!POSE) galpha += g1.y;
          // radiosity (Eq. 3); dir_grad: the colour depends on the mean's direction
          bool dir_grad = false;
          float d[3], inv = 0.f, dh_[3], ddh[3] = {0.f, 0.f, 0.f};
          if (!GEN) {
            if (!is_dir) {
              if (!POSE) dz_iso += g1.z * c_iso * (1.f - c_iso);
            } else {
              dir_grad = true;
              d[0] = mu[0] + vc.wt[0]; d[1] = mu[1] + vc.wt[1]; d[2] = mu[2] + vc.wt[2];
              inv = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
              dh_[0] = d[0] * inv; dh_[1] = d[1] * inv; dh_[2] = d[2] * inv;
              float Y[3] = {-SH_C1 * dh_[1], SH_C1 * dh_[2], -SH_C1 * dh_[0]};
              float c = sigmoidf_(Y[0] * h[0] + Y[1] * h[1] + Y[2] * h[2]);
              float dz = g1.z * c * (1.f - c);
              if (!POSE) { dh[0] += dz * Y[0]; dh[1] += dz * Y[1]; dh[2] += dz * Y[2]; }
              float dY[3] = {dz * h[0], dz * h[1], dz * h[2]};
              ddh[0] = -SH_C1 * dY[2]; ddh[1] = -SH_C1 * dY[0]; ddh[2] = SH_C1 * dY[1];
            }
          } else if (a.per_pixel) {
            // the rasteriser summed dL/dz (g1.z) and dL/dh (gh) over the pixels
            if (has_iso) dz_iso += g1.z;
            if (has_dir) { dh[0] += gh.x; dh[1] += gh.y; dh[2] += gh.z; }
          } else {
            float zl = c_iso, Y[KLS], dYd[KLS][3];
            if (has_dir) {
              d[0] = mu[0] + vc.wt[0]; d[1] = mu[1] + vc.wt[1]; d[2] = mu[2] + vc.wt[2];
              inv = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
              dh_[0] = d[0] * inv; dh_[1] = d[1] * inv; dh_[2] = d[2] * inv;
              sh_eval(s_sh, kL, dh_[0], dh_[1], dh_[2], Y, dYd);
#pragma unroll
              for (int m = 0; m < KLS; ++m)
                if (m < kL) zl = fmaf(Y[m], h[m], zl);
            }
            const float c = sigmoidf_(zl);
            const float dz = g1.z * c * (1.f - c);
            if (has_iso) dz_iso += dz;
            if (has_dir) {
              dir_grad = true;
#pragma unroll
              for (int m = 0; m < KLS; ++m) {
                if (m >= kL) break;
                dh[m] += dz * Y[m];
                const float w = dz * h[m];
                ddh[0] = fmaf(w, dYd[m][0], ddh[0]);
                ddh[1] = fmaf(w, dYd[m][1], ddh[1]);
                ddh[2] = fmaf(w, dYd[m][2], ddh[2]);
              }
            }
          }
          if (dir_grad) {
            float dot = ddh[0] * dh_[0] + ddh[1] * dh_[1] + ddh[2] * dh_[2];
            float dd[3] = {(ddh[0] - dh_[0] * dot) * inv, (ddh[1] - dh_[1] * dot) * inv,
                           (ddh[2] - dh_[2] * dot) * inv};
#pragma unroll
            for (int c3 = 0; c3 < 3; ++c3) {
              if (!POSE) dmu[c3] += dd[c3];
#pragma unroll
              for (int r = 0; r < 3; ++r) dW[3 * r + c3] += vc.t[r] * dd[c3];
            }
#pragma unroll
            for (int r = 0; r < 3; ++r)
              dt[r] += vc.W[3 * r] * dd[0] + vc.W[3 * r + 1] * dd[1] + vc.W[3 * r + 2] * dd[2];
          }
          // conic = inverse 2D covariance: GS = -K GK K
          const float idet = rcp_approx(p.det);
          const float k0 = p.cov[2] * idet, k1 = -p.cov[1] * idet, k2 = p.cov[0] * idet;
          const float hb = 0.5f * gcb;
          const float m00 = k0 * gca + k1 * hb, m01 = k0 * hb + k1 * gcc;
          const float m10 = k1 * gca + k2 * hb, m11 = k1 * hb + k2 * gcc;
          const float GS00 = -(m00 * k0 + m01 * k1), GS01 = -(m00 * k1 + m01 * k2),
                      GS11 = -(m10 * k1 + m11 * k2);
          // P = A Sigma
          float P[6];
#pragma unroll
          for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k)
              P[3 * r + k] = p.A[3 * r] * sym(gg.S, 0, k) + p.A[3 * r + 1] * sym(gg.S, 1, k) +
                             p.A[3 * r + 2] * sym(gg.S, 2, k);
          // dA = 2 GS P ; Q = GS A ; dSigma += A^T Q
          float dA[6], Q[6];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            dA[k] = 2.f * (GS00 * P[k] + GS01 * P[3 + k]);
            dA[3 + k] = 2.f * (GS01 * P[k] + GS11 * P[3 + k]);
            Q[k] = GS00 * p.A[k] + GS01 * p.A[3 + k];
            Q[3 + k] = GS01 * p.A[k] + GS11 * p.A[3 + k];
          }
          if (!POSE) {
            dSig[0] += p.A[0] * Q[0] + p.A[3] * Q[3];
            dSig[1] += p.A[0] * Q[1] + p.A[3] * Q[4];
            dSig[2] += p.A[0] * Q[2] + p.A[3] * Q[5];
            dSig[3] += p.A[1] * Q[1] + p.A[4] * Q[4];
            dSig[4] += p.A[1] * Q[2] + p.A[4] * Q[5];
            dSig[5] += p.A[2] * Q[2] + p.A[5] * Q[5];
          }
          // A = J W: dJ = dA W^T (entries 00, 02, 11, 12), dW += J^T dA
          const float dJ00 = dA[0] * vc.W[0] + dA[1] * vc.W[1] + dA[2] * vc.W[2];
          const float dJ02 = dA[0] * vc.W[6] + dA[1] * vc.W[7] + dA[2] * vc.W[8];
          const float dJ11 = dA[3] * vc.W[3] + dA[4] * vc.W[4] + dA[5] * vc.W[5];
          const float dJ12 = dA[3] * vc.W[6] + dA[4] * vc.W[7] + dA[5] * vc.W[8];
#pragma unroll
          for (int c3 = 0; c3 < 3; ++c3) {
            dW[c3] += p.j00 * dA[c3];
            dW[3 + c3] += p.j11 * dA[3 + c3];
            dW[6 + c3] += p.j02 * dA[c3] + p.j12 * dA[3 + c3];
          }
          // J(x_c) and the projected mean
          const float iz = rcp_approx(p.xc[2]);
          float dxc[3];
          dxc[0] = -dJ02 * p.j00 * iz + gu * p.j00;
          dxc[1] = -dJ12 * p.j11 * iz + gv * p.j11;
          dxc[2] = -(dJ00 * p.j00 + dJ11 * p.j11) * iz - 2.f * (dJ02 * p.j02 + dJ12 * p.j12) * iz +
                   gu * p.j02 + gv * p.j12;
          // x_c = W mu + t
          if (!POSE) {
#pragma unroll
            for (int c3 = 0; c3 < 3; ++c3)
              dmu[c3] += vc.W[c3] * dxc[0] + vc.W[3 + c3] * dxc[1] + vc.W[6 + c3] * dxc[2];
          }
#pragma unroll
          for (int r = 0; r < 3; ++r) {
#pragma unroll
            for (int c3 = 0; c3 < 3; ++c3) dW[3 * r + c3] += dxc[r] * mu[c3];
            dt[r] += dxc[r];
          }
        }
      }
      if (a.want_pose) {
        const bool warp_any = __any_sync(0xffffffffu, any);
        if (warp_any) {
          float v16[16] = {dW[0], dW[1], dW[2], dt[0], dW[3], dW[4], dW[5], dt[1],
                           dW[6], dW[7], dW[8], dt[2], 0.f, 0.f, 0.f, 0.f};
          const int comp = warp_reduce16(v16);
          if ((lane & 1) == 0 && comp < 12) atomicAdd(&s_pose[vv][comp], v16[0]);
        }
      }
    }
    if (a.want_pose) {
      __syncthreads();
      for (int e = tid; e < nv * 12; e += blockDim.x) {
        float x = (&s_pose[0][0])[e];
        if (x != 0.f) atomicAdd(a.out.world_to_cam + 12 * (int64_t)(rq.v_off + v0) + e, x);
      }
    }
  }

  // per-Gaussian outputs
  if (!POSE && live && a.want_param) {
    if (a.out.opacity_logits) a.out.opacity_logits[i] = galpha * alpha * (1.f - alpha);
    if (a.out.means) {
      a.out.means[3 * i] = dmu[0]; a.out.means[3 * i + 1] = dmu[1]; a.out.means[3 * i + 2] = dmu[2];
    }
    if (!GEN) {
      float gf[K];
      if (!is_dir) {
#pragma unroll
        for (int k = 0; k < K; ++k) gf[k] = dz_iso * s_b[k];
        if (a.out.feat_iso) {
          float4 *o = reinterpret_cast<float4 *>(a.out.feat_iso + (rq.iso_row + br.l) * K);
          o[0] = make_float4(gf[0], gf[1], gf[2], gf[3]);
          o[1] = make_float4(gf[4], gf[5], gf[6], gf[7]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) gf[k] = s_B[k] * dh[0] + s_B[K + k] * dh[1] + s_B[2 * K + k] * dh[2];
        if (a.out.feat_dir) {
          float4 *o = reinterpret_cast<float4 *>(a.out.feat_dir + (rq.dir_row + br.l - rq.n_iso) * K);
          o[0] = make_float4(gf[0], gf[1], gf[2], gf[3]);
          o[1] = make_float4(gf[4], gf[5], gf[6], gf[7]);
        }
      }
    } else {
      // f feeds a = b_iso . f and/or h = B_dir f; the row lives in the
      // Gaussian's own range
      float *dst = !is_dir ? (a.out.feat_iso ? a.out.feat_iso + (rq.iso_row + br.l) * Kr : nullptr)
                           : (a.out.feat_dir ? a.out.feat_dir + (rq.dir_row + br.l - rq.n_iso) * Kr
                                             : nullptr);
      if (dst)
        for (int k = 0; k < Kr; ++k) {
          float acc = has_iso ? dz_iso * s_b[k] : 0.f;
          if (has_dir) {
#pragma unroll
            for (int m = 0; m < KLS; ++m)
              if (m < kL) acc = fmaf(s_B[m * Kr + k], dh[m], acc);
          }
          dst[k] = acc;
        }
    }
    if (a.out.log_scales || a.out.quats) {
      // Sigma = M M^T: dM = 2 dSigma M ; M = R diag(s)
      float dM[9];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c3 = 0; c3 < 3; ++c3)
          dM[3 * r + c3] = 2.f * (sym(dSig, r, 0) * gg.M[c3] + sym(dSig, r, 1) * gg.M[3 + c3] +
                                  sym(dSig, r, 2) * gg.M[6 + c3]);
      float dR[9], ds[3] = {0, 0, 0};
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c3 = 0; c3 < 3; ++c3) {
          dR[3 * r + c3] = dM[3 * r + c3] * gg.s[c3];
          ds[c3] += dM[3 * r + c3] * gg.R[3 * r + c3];
        }
      if (a.out.log_scales) {
        a.out.log_scales[3 * i] = ds[0] * gg.s[0];
        a.out.log_scales[3 * i + 1] = ds[1] * gg.s[1];
        a.out.log_scales[3 * i + 2] = ds[2] * gg.s[2];
      }
      if (a.out.quats) {
        const float w = gg.qn[0], x = gg.qn[1], y = gg.qn[2], z = gg.qn[3];
        float dq[4];
        dq[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
        dq[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] +
                       w * dR[7] - 2.f * x * dR[8]);
        dq[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] +
                       z * dR[7] - 2.f * y * dR[8]);
        dq[3] = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] +
                       y * dR[5] + x * dR[6] + y * dR[7]);
        const float dot = dq[0] * w + dq[1] * x + dq[2] * y + dq[3] * z;
        const float inv = 1.f / gg.qnorm;
        reinterpret_cast<float4 *>(a.out.quats)[i] =
            make_float4((dq[0] - w * dot) * inv, (dq[1] - x * dot) * inv, (dq[2] - y * dot) * inv,
                        (dq[3] - z * dot) * inv);
      }
    }
  }
  if (!POSE && a.want_basis && GEN) {
    // b_iso gradient: dz_iso f (isotropic); B_dir gradient: dh f^T (directional)
    if (live) {
      for (int k = 0; k < Kr; ++k) {
        const float fk = load_feat1(a.feat_iso, a.feat_dir, a.feat_dir_bf16, rq, br.l, Kr, k);
        if (has_iso && dz_iso != 0.f) atomicAdd(&s_basis[k], dz_iso * fk);
        if (has_dir) {
#pragma unroll
          for (int m = 0; m < KLS; ++m)
            if (m < kL && dh[m] != 0.f) atomicAdd(&s_basis[Kr + m * Kr + k], dh[m] * fk);
        }
      }
    }
    __syncthreads();
    for (int e = tid; e < (1 + kL) * Kr; e += PRE_THREADS) {
      const float x = s_basis[e];
      if (x == 0.f) continue;
      if (e < Kr) {
        if (a.out.b_iso) atomicAdd(a.out.b_iso + (int64_t)br.r * Kr + e, x);
      } else if (a.out.B_dir) {
        atomicAdd(a.out.B_dir + (int64_t)br.r * kL * Kr + (e - Kr), x);
      }
    }
  }
  if (!POSE && a.want_basis && !GEN) {
    // b_iso gradient: dz_iso f (isotropic); B_dir gradient: dh f^T (directional)
    float v32[4 * K];
#pragma unroll
    for (int k = 0; k < K; ++k) v32[k] = (live && !is_dir) ? dz_iso * f[k] : 0.f;
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int k = 0; k < K; ++k) v32[K + m * K + k] = (live && is_dir) ? dh[m] * f[k] : 0.f;
    float lo[16], hi2[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) { lo[k] = v32[k]; hi2[k] = v32[16 + k]; }
    const int c_lo = warp_reduce16(lo);
    warp_reduce16(hi2);
    if ((lane & 1) == 0) {
      atomicAdd(&s_basis[c_lo], lo[0]);
      atomicAdd(&s_basis[16 + c_lo], hi2[0]);
    }
    __syncthreads();
    if (tid < K && a.out.b_iso) atomicAdd(a.out.b_iso + br.r * K + tid, s_basis[tid]);
    if (tid >= K && tid < 4 * K && a.out.B_dir)
      atomicAdd(a.out.B_dir + br.r * 3 * K + (tid - K), s_basis[tid]);
  }
}

}  // namespace

void launch_preprocess_fwd(const ddgs_gaussians &g, const ddgs_views &v, const ddgs_config &c,
                           const RenderShape &s, ddgs_workspace &ws, cudaStream_t st) {
  PreArgs a;
  a.means = g.means; a.log_scales = g.log_scales; a.quats = g.quats; a.logits = g.opacity_logits;
  a.feat_iso = g.feat_iso; a.feat_dir = g.feat_dir; a.feat_dir_bf16 = g.feat_dir_bf16;
  a.b_iso = g.b_iso; a.B_dir = g.B_dir; a.world_to_cam = v.world_to_cam; a.detector = v.detector;
  a.dilation = c.dilation; a.near_plane = c.near_plane; a.q_max = c.q_max;
  a.K = g.feat_dim ? g.feat_dim : K;
  a.L = g.sh_degree ? g.sh_degree : 1;
  a.entangled = g.entangled ? 1 : 0;
  a.per_pixel = g.per_pixel ? 1 : 0;
  a.s = s;
  a.rec = ws.rec; a.rec2 = ws.rec2;
  a.bin_info = reinterpret_cast<uint4 *>(ws.rect);
  a.blk_total = ws.blk_total;
  a.t0 = ws.req_time;
  a.status = ws.d_status;
  if (s.n_blocks > 0) {
    LaunchScope ls(KID_PREPROCESS_FWD, st);
    if (a.K == K && a.L == 1 && !a.entangled && !a.per_pixel)
      preprocess_fwd_kernel<false><<<(unsigned)s.n_blocks, PRE_THREADS, 0, st>>>(a);
    else
      preprocess_fwd_kernel<true><<<(unsigned)s.n_blocks, PRE_THREADS, 0, st>>>(a);
  }
}

void launch_preprocess_bwd(const ddgs_gaussians &g, const ddgs_views &v, const ddgs_config &c,
                           const RenderShape &s, ddgs_workspace &ws, const ddgs_grads &out,
                           cudaStream_t st) {
  PreBwdArgs a;
  a.means = g.means; a.log_scales = g.log_scales; a.quats = g.quats; a.logits = g.opacity_logits;
  a.feat_iso = g.feat_iso; a.feat_dir = g.feat_dir; a.feat_dir_bf16 = g.feat_dir_bf16;
  a.b_iso = g.b_iso; a.B_dir = g.B_dir; a.world_to_cam = v.world_to_cam; a.detector = v.detector;
  a.dilation = c.dilation; a.near_plane = c.near_plane;
  a.K = g.feat_dim ? g.feat_dim : K;
  a.L = g.sh_degree ? g.sh_degree : 1;
  a.entangled = g.entangled ? 1 : 0;
  a.per_pixel = g.per_pixel ? 1 : 0;
  a.s = s;
  a.grad2d = ws.grad2d;
  a.grad_h = ws.grad_h;
  a.out = out;
  a.want_param = (out.means || out.log_scales || out.quats || out.opacity_logits || out.feat_iso ||
                  out.feat_dir) ? 1 : 0;
  a.want_basis = (out.b_iso || out.B_dir) ? 1 : 0;
  a.want_pose = out.world_to_cam ? 1 : 0;
  if (s.n_blocks > 0) {
    LaunchScope ls(KID_PREPROCESS_BWD, st);
    const bool fast = a.K == K && a.L == 1 && !a.entangled && !a.per_pixel;
    if (fast && !a.want_param && !a.want_basis)
      preprocess_bwd_kernel<false, true><<<(unsigned)s.n_blocks, PRE_THREADS, 0, st>>>(a);
    else if (fast)
      preprocess_bwd_kernel<false><<<(unsigned)s.n_blocks, PRE_THREADS, 0, st>>>(a);
    else
      preprocess_bwd_kernel<true><<<(unsigned)s.n_blocks, PRE_THREADS, 0, st>>>(a);
  }
}

}  // namespace ddgs
