// raster.cu -- per-tile front-to-back blending (Eq. 1) and its backward pass.
//
// One thread block renders one (view, tile) list; one thread owns one pixel.
// Warps own 8 x 4 pixel blocks, so a Gaussian whose q <= q_max ellipse misses
// a warp's block is skipped by the whole warp with one uniform test. Gaussians
// of the list are staged in shared memory one batch (one per thread) at a
// time: the batch is a gather by Gaussian index from the per-view records,
// which is why it uses plain vector loads rather than a bulk tensor copy.
//
// Forward per pixel p, over the list in ascending depth (Eq. 1):
//   q = (p - mu-hat)^T conic (p - mu-hat); skip if q > q_max;
//   sigma = min(alpha_max, alpha exp(-q/2)); skip if sigma < alpha_min;
//   T' = T (1 - sigma); stop (without adding) if T' < t_min;
//   C += c sigma T; T = T'.
// Backward per pixel, over the same list from the last added Gaussian to the
// first, recovering T before each Gaussian as T' / (1 - sigma) and carrying
// the suffix sum S = sum over later Gaussians of c sigma T:
//   dC/dc = sigma T,  dC/dsigma = c T - S / (1 - sigma),
//   dsigma/dalpha = G and dsigma/dq = -alpha G / 2 unless sigma was clamped.
// The per-pixel 2D gradients of one Gaussian are summed over the warp with
// shuffles, over the block in shared memory, and reach global memory with one
// vector atomic per (tile, Gaussian).
//
// PIX = true renders the Eq. 3 variant whose ray angles are each pixel's own:
// a record then carries (a, h) instead of a colour, and the pair's colour is
// c = sigmoid(a + Y_1(d_p) . h) with d_p the pixel ray's unit direction. The
// backward pass sums dL/dz (z the logit) and dL/dh per (tile, Gaussian) and
// adds the pose gradient through each pixel's ray.
#include <map>
#include <mutex>
#include <utility>

#include "ddgs_internal.cuh"

namespace ddgs {
namespace {

struct RasterArgs {
  RenderShape s;
  RasterParams P;
  const float4 *rec;  // two float4 per record
  const uint32_t *vals;  // tile lists: Gaussian indices in depth order
  const uint2 *ranges;
  float4 *grad2d;
  float *image, *t_final;
  uint32_t *n_last;
  const float *dL_dimage, *t_final_in;
  const uint32_t *n_last_in;
  const uint32_t *order;     // global tiles, longest list first
  uint32_t *counter;         // work-queue head (zero at launch)
  unsigned long long *req_end;  // [R]: latest %globaltimer of a finished tile, or null
  // per-pixel ray angles only
  const float4 *rec2;        // (a, h_0, h_1, h_2) per record
  float4 *grad_h;            // dL/dh per record
  const float *world_to_cam, *detector;
  float *pose_grad;          // [V][12] or null
};

__device__ __forceinline__ float sigmoid_r(float x) { return rcp_approx(1.f + __expf(-x)); }

// The ray through pixel centre (px, py) of a view: rc = ((px - c_u) pitch_u,
// (py - c_v) pitch_v, sdd) in camera coordinates, world direction d = W^T rc,
// and Y_1 of d / |d| (real harmonics of degree 1: sqrt(3/(4 pi)) (-y, z, -x)).
struct PixRay {
  float rc[3], dh[3], inv, Y[3];
};

__device__ __forceinline__ void pixel_ray(const float *pose, const float *det, int H, int W,
                                          float px, float py, PixRay &r) {
  const float cu = 0.5f * (float)W + det[3], cv = 0.5f * (float)H + det[4];
  r.rc[0] = (px - cu) * det[1];
  r.rc[1] = (py - cv) * det[2];
  r.rc[2] = det[0];
  float d[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) d[c] = pose[c] * r.rc[0] + pose[4 + c] * r.rc[1] + pose[8 + c] * r.rc[2];
  r.inv = 1.f / sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
  for (int c = 0; c < 3; ++c) r.dh[c] = d[c] * r.inv;
  r.Y[0] = -SH_C1 * r.dh[1];
  r.Y[1] = SH_C1 * r.dh[2];
  r.Y[2] = -SH_C1 * r.dh[0];
}

__device__ __forceinline__ float pixel_colour(const PixRay &r, float4 z) {
  return sigmoid_r(fmaf(r.Y[2], z.w, fmaf(r.Y[1], z.z, fmaf(r.Y[0], z.y, z.x))));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Pixel-space box of the q <= q_max ellipse: the record's packed
// half-extents (computed from the 2D covariance by the preprocess).
__device__ __forceinline__ float4 ellipse_box(float4 r0, float4 r1, float q_max) {
  (void)q_max;
  const float2 e = unpack_halfwidths(r1.w);
  return make_float4(r0.x - e.x, r0.x + e.x, r0.y - e.y, r0.y + e.y);
}

__device__ __forceinline__ float4 empty_box() {
  return make_float4(__int_as_float(0x7f800000), -__int_as_float(0x7f800000),
                     __int_as_float(0x7f800000), -__int_as_float(0x7f800000));
}

// A warp's 8 x 4 pixels are split into groups of GW x 2 pixels, one lane per
// pixel: four 4 x 2 quarters of 8 lanes (GW = 4) or eight 2 x 2 groups of 4
// lanes (GW = 2, the warp-streamed forward). Each group walks only the list
// entries whose box meets it. Smaller groups skip more entries but take more
// ballots per batch; the backward keeps quarters, whose 8-lane gradient
// reduction leaves one shared-memory accumulator update per lane (2 x 2 groups
// measured slower there: 4.71 -> 4.95 ms at 64 poses, forward 1.99 -> 1.89).
template <int T, int GW = 4>
struct TileGeom {
  static_assert(GW == 2 || GW == 4, "groups are 4 x 2 or 2 x 2 pixels");
  static constexpr int LG = 2 * GW;  // lanes per group
  static constexpr int NG = 32 / LG; // groups per warp
  static constexpr int GX = 8 / GW;  // groups per pixel row of the warp
  int v, txi, tyi, px, py, wx0, wy0, H, W;
  bool inside;
  int64_t gtile, rec_base, img_off, n_req;
  // region: which 8 x 4 pixel block of the tile this warp owns
  __device__ __forceinline__ TileGeom(const RenderShape &s, int64_t gt, int region) {
    gtile = gt;
    v = find_view(s.view, s.V, gt);
    const ViewTab vt = s.view[v];
    H = vt.H;
    W = vt.W;
    rec_base = vt.rec_off;
    img_off = vt.img_off;
    n_req = s.req[vt.req].n;
    const int64_t local = gt - vt.tile_base;
    tyi = (int)(local / vt.tiles_x);
    txi = (int)(local - (int64_t)tyi * vt.tiles_x);
    constexpr int WX = T / 8;
    const int lane = threadIdx.x & 31;
    const int wx = region % WX, wy = region / WX;
    wx0 = txi * T + wx * 8;
    wy0 = tyi * T + wy * 4;
    const int g = lane / LG;
    px = wx0 + (g % GX) * GW + lane % GW;
    py = wy0 + (g / GX) * 2 + (lane / GW) % 2;
    inside = px < W && py < H;
  }
  __device__ __forceinline__ int64_t pixel() const { return img_off + (int64_t)py * W + px; }
  // does the box miss the GW x 2 pixel centres of group q of this warp?
  __device__ __forceinline__ bool misses_q(float4 b, int q) const {
    const float x0 = (float)(wx0 + (q % GX) * GW), y0 = (float)(wy0 + (q / GX) * 2);
    return b.x > x0 + (GW - 0.5f) || b.y < x0 + 0.5f || b.z > y0 + 1.5f || b.w < y0 + 0.5f;
  }
};

// Each lane tests list entry c0 + lane of the staged batch against the four
// quarters of its warp (ok: the entry exists and passes the caller's test);
// returns the entries this lane's quarter must evaluate, in list order.
template <int T>
__device__ __forceinline__ uint32_t quarter_todo(const TileGeom<T> &tg, float4 box, bool ok) {
  static_assert(TileGeom<T>::NG == 4, "four quarters of 8 lanes");
  const int q = (threadIdx.x & 31) >> 3;
  const uint32_t m0 = __ballot_sync(0xffffffffu, ok && !tg.misses_q(box, 0));
  const uint32_t m1 = __ballot_sync(0xffffffffu, ok && !tg.misses_q(box, 1));
  const uint32_t m2 = __ballot_sync(0xffffffffu, ok && !tg.misses_q(box, 2));
  const uint32_t m3 = __ballot_sync(0xffffffffu, ok && !tg.misses_q(box, 3));
  return q == 0 ? m0 : (q == 1 ? m1 : (q == 2 ? m2 : m3));
}

// One (view, tile) work item of the forward pass; BATCH list entries are
// staged in shared memory per round.
template <int T, int BATCH, bool PIX>
__device__ __forceinline__ void fwd_tile(const RasterArgs &a, int64_t gt, float4 *s_a, float4 *s_b,
                                         float4 *s_box, float4 *s_c) {
  constexpr int NT = T * T;
  const int tid = threadIdx.x;
  const TileGeom<T> tg(a.s, gt, threadIdx.x >> 5);
  const uint2 range = a.ranges[tg.gtile];
  const uint32_t *vals = a.vals;
  const int64_t rec_base = tg.rec_base;
  const float px = tg.px + 0.5f, py = tg.py + 0.5f;
  PixRay ray;
  if (PIX) pixel_ray(a.world_to_cam + 12 * tg.v, a.detector + 5 * tg.v, tg.H, tg.W, px, py, ray);
  float Tr = 1.f, C = 0.f;
  uint32_t last = 0;
  bool done = !tg.inside;
  for (uint32_t b0 = range.x; b0 < range.y; b0 += BATCH) {
    if (__syncthreads_count(done) == NT) break;
    for (int e = tid; e < BATCH; e += NT) {
      const uint32_t j = b0 + e;
      if (j < range.y) {
        const uint32_t id = vals[j];
        if (id < tg.n_req) {
          const int64_t r = rec_base + id;
          const float4 r0 = a.rec[2 * r], r1 = a.rec[2 * r + 1];
          s_a[e] = r0;
          s_b[e] = r1;
          s_box[e] = ellipse_box(r0, r1, a.P.q_max);
          if (PIX) s_c[e] = a.rec2[r];
        } else {
          s_box[e] = empty_box();  // only after a capacity overflow
        }
      }
    }
    __syncthreads();
    const int cnt = (int)min((uint32_t)BATCH, range.y - b0);
    // 32 entries at a time: each lane tests one entry's box against the four
    // quarters of its warp; each quarter then walks its own entries, so one
    // instruction serves up to four (quarter, entry) pairs.
    const int lane = threadIdx.x & 31;
    for (int c0 = 0; c0 < cnt; c0 += 32) {
      const uint32_t dmask = __ballot_sync(0xffffffffu, done);
      if (dmask == 0xffffffffu) break;
      const int ec = c0 + lane;
      const float4 box = ec < cnt ? s_box[ec] : empty_box();
      uint32_t mine = quarter_todo<T>(tg, box, ec < cnt);
      if (((dmask >> (lane & 24)) & 0xffu) == 0xffu) mine = 0;  // quarter finished
      while (__any_sync(0xffffffffu, mine != 0)) {
        if (mine == 0) continue;
        const int k = c0 + __ffs(mine) - 1;
        mine &= mine - 1;
        if (done) continue;
        const float4 A = s_a[k], B = s_b[k];
        PairEval e;
        if (!eval_pair(A.x, A.y, A.z, A.w, B.x, B.y, px, py, a.P, e)) continue;
        const float Tn = __fmaf_rn(-Tr, e.sigma, Tr);  // T (1 - sigma)
        if (Tn < a.P.t_min) {
          done = true;
          continue;
        }
        const float col = PIX ? pixel_colour(ray, s_c[k]) : B.z;
        C = fmaf(col * e.sigma, Tr, C);
        Tr = Tn;
        last = b0 + (uint32_t)k - range.x + 1u;
      }
    }
  }
  if (tg.inside) {
    const int64_t pix = tg.pixel();
    a.image[pix] = C;
    a.t_final[pix] = Tr;
    a.n_last[pix] = last;
  }
}

// Persistent forward rasteriser: each block takes work items from the queue
// (longest tile lists first) until it is empty.
// Minimum resident blocks per SM requested from the register allocator: six
// 256-thread blocks (40 registers) for the forward, five (48) for the backward.
template <int T>
constexpr int fwd_min_blocks() { return T == 16 ? 6 : (T == 8 ? 16 : 1); }
template <int T>
constexpr int bwd_min_blocks() { return T == 16 ? 5 : (T == 8 ? 12 : 1); }

template <int T, int BATCH, bool PIX>
__global__ void __launch_bounds__(T *T, fwd_min_blocks<T>()) raster_fwd_kernel(RasterArgs a) {
  __shared__ float4 s_a[BATCH], s_b[BATCH], s_box[BATCH], s_c[PIX ? BATCH : 1];
  __shared__ uint32_t s_item;
  for (;;) {
    __syncthreads();  // the previous item is finished by every thread
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= (uint32_t)a.s.total_tiles) break;
    const int64_t gt = a.order[item];
    fwd_tile<T, BATCH, PIX>(a, gt, s_a, s_b, s_box, s_c);
    if (a.req_end && threadIdx.x == 0)
      atomicMax(a.req_end + a.s.view[find_view(a.s.view, a.s.V, gt)].req, global_ns());
  }
}

// Sum 8 per-lane values over each group of 8 lanes (a quarter) with 7
// shuffles. Afterwards lane l of the quarter holds in v[0] the quarter's total
// of component ((l >> 2) & 1) * 4 + ((l >> 1) & 1) * 2 + (l & 1), returned.
__device__ __forceinline__ int quarter_reduce8(float v[8]) {
  const int lane = threadIdx.x & 31;
  bool hi = lane & 4;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float send = hi ? v[k] : v[k + 4];
    float keep = hi ? v[k + 4] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  hi = lane & 2;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    float send = hi ? v[k] : v[k + 2];
    float keep = hi ? v[k + 2] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  hi = lane & 1;
  {
    float send = hi ? v[0] : v[1];
    float keep = hi ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
  }
  return ((lane >> 2) & 1) * 4 + ((lane >> 1) & 1) * 2 + (lane & 1);
}

// Sum 10 per-lane values over each quarter (8 lanes) with 10 shuffles: v[8]
// and v[9] first (lanes with l % 4 == 0 end with component 8, if bit 2 of the
// lane is clear, or 9 in v[8]), then v[0..7] as quarter_reduce8 (lane l ends
// with the component it returns in v[0]).
__device__ __forceinline__ int quarter_reduce10(float v[10]) {
  const int lane = threadIdx.x & 31;
  const bool hi = lane & 4;
  const float send = hi ? v[8] : v[9], keep = hi ? v[9] : v[8];
  float w = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  w += __shfl_xor_sync(0xffffffffu, w, 2);
  w += __shfl_xor_sync(0xffffffffu, w, 1);
  v[8] = w;
  return quarter_reduce8(v);
}

// Accumulated components per (tile, Gaussian): u, v, conic a, b, c, alpha and
// the colour (or, with PIX, the logit z and h_0..h_2).
template <bool PIX>
constexpr int n_acc() { return PIX ? 12 : 8; }

template <int BATCH, bool PIX>
struct BwdSmem {
  float4 a[BATCH], b[BATCH], box[BATCH], c[PIX ? BATCH : 1];
  uint32_t id[BATCH];
  float acc[BATCH][n_acc<PIX>()];
  float pose[PIX ? 12 : 1];  // per-tile pose gradient through the pixel rays
  uint32_t max_last;
};

// One (view, tile) work item of the backward pass.
template <int T, int BATCH, bool PIX>
__device__ __forceinline__ void bwd_tile(const RasterArgs &a, int64_t gt, BwdSmem<BATCH, PIX> &sm) {
  float4 *s_a = sm.a, *s_b = sm.b, *s_box = sm.box, *s_c = sm.c;
  uint32_t *s_id = sm.id;
  float (*s_acc)[n_acc<PIX>()] = sm.acc;
  uint32_t &s_max = sm.max_last;
  constexpr int NT = T * T;
  const int tid = threadIdx.x;
  const TileGeom<T> tg(a.s, gt, threadIdx.x >> 5);
  const uint2 range = a.ranges[tg.gtile];
  const uint32_t *vals = a.vals;
  const int64_t rec_base = tg.rec_base;
  const float px = tg.px + 0.5f, py = tg.py + 0.5f;
  PixRay ray;
  float gY[3] = {0.f, 0.f, 0.f};  // dL/dY_1 of this pixel's ray
  if (PIX) pixel_ray(a.world_to_cam + 12 * tg.v, a.detector + 5 * tg.v, tg.H, tg.W, px, py, ray);
  float Tr = 1.f, g = 0.f;
  uint32_t last = 0;
  if (tg.inside) {
    const int64_t pix = tg.pixel();
    Tr = a.t_final_in[pix];
    last = a.n_last_in[pix];
    g = a.dL_dimage[pix];
  }
  if (g == 0.f) last = 0;  // nothing to propagate from this pixel
  if (last > range.y - range.x) last = range.y - range.x;  // never read past the list
  if (tid == 0) s_max = 0;
  __syncthreads();
  if (last) atomicMax(&s_max, last);
  __syncthreads();
  const uint32_t max_last = s_max;
  // last list position any pixel of each quarter added (every lane learns all four)
  uint32_t qlast = last;
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) qlast = max(qlast, __shfl_xor_sync(0xffffffffu, qlast, o));
  const uint32_t ql0 = __shfl_sync(0xffffffffu, qlast, 0), ql1 = __shfl_sync(0xffffffffu, qlast, 8);
  const uint32_t ql2 = __shfl_sync(0xffffffffu, qlast, 16), ql3 = __shfl_sync(0xffffffffu, qlast, 24);
  float S = 0.f;
  for (int64_t hi = max_last; hi > 0; hi -= BATCH) {
    const int64_t lo = hi > BATCH ? hi - BATCH : 0;
    for (int e = tid; e < BATCH; e += NT) {
      const int64_t pos_t = hi - 1 - e;  // batches run back to front
      if (pos_t >= lo) {
        const uint32_t id = vals[range.x + (uint32_t)pos_t];
        if (id < tg.n_req) {
          const int64_t r = rec_base + id;
          const float4 r0 = a.rec[2 * r], r1 = a.rec[2 * r + 1];
          s_a[e] = r0;
          s_b[e] = r1;
          s_box[e] = ellipse_box(r0, r1, a.P.q_max);
          if (PIX) s_c[e] = a.rec2[r];
        } else {
          s_box[e] = empty_box();  // only after a capacity overflow
        }
        s_id[e] = id;
      }
#pragma unroll
      for (int c = 0; c < n_acc<PIX>(); ++c) s_acc[e][c] = 0.f;
    }
    __syncthreads();
    const int cnt = (int)(hi - lo);
    const int lane = threadIdx.x & 31;
    for (int c0 = 0; c0 < cnt; c0 += 32) {
      // each lane tests one entry against the four quarters: inside the
      // quarter's box and before the last Gaussian the quarter added
      const int ec = c0 + lane;
      const bool ok = ec < cnt;
      const float4 box = ok ? s_box[ec] : empty_box();
      const uint32_t pe = (uint32_t)(hi - 1 - ec);
      const uint32_t m0 = __ballot_sync(0xffffffffu, ok && pe < ql0 && !tg.misses_q(box, 0));
      const uint32_t m1 = __ballot_sync(0xffffffffu, ok && pe < ql1 && !tg.misses_q(box, 1));
      const uint32_t m2 = __ballot_sync(0xffffffffu, ok && pe < ql2 && !tg.misses_q(box, 2));
      const uint32_t m3 = __ballot_sync(0xffffffffu, ok && pe < ql3 && !tg.misses_q(box, 3));
      const int qi = lane >> 3;
      uint32_t mine = qi == 0 ? m0 : (qi == 1 ? m1 : (qi == 2 ? m2 : m3));
      while (__any_sync(0xffffffffu, mine != 0)) {
        const bool has = mine != 0;
        const int k = has ? c0 + __ffs(mine) - 1 : c0;
        if (has) mine &= mine - 1;
        const uint32_t pos = (uint32_t)(hi - 1 - k);
        float gv[PIX ? 10 : 8];
#pragma unroll
        for (int c = 0; c < (PIX ? 10 : 8); ++c) gv[c] = 0.f;
        bool act = has && pos < last;
        if (act) {
          const float4 A = s_a[k], B = s_b[k];
          PairEval e;
          act = eval_pair(A.x, A.y, A.z, A.w, B.x, B.y, px, py, a.P, e);
          if (act) {
            // 1 / (1 - sigma) with sigma <= alpha_max < 1: the fast reciprocal's
            // relative error (~1 ulp) is far inside the gradient tolerance
            const float inv_om = rcp_approx(__fsub_rn(1.f, e.sigma));
            Tr = Tr * inv_om;  // transmittance before this Gaussian
            float4 cz;
            if (PIX) cz = s_c[k];
            const float c = PIX ? pixel_colour(ray, cz) : B.z;
            const float dC_dsigma = fmaf(c, Tr, -S * inv_om);
            S = fmaf(c * e.sigma, Tr, S);
            const float gs = g * dC_dsigma;
            float gq = 0.f;
            if (!(e.aG > a.P.alpha_max)) {
              gv[5] = gs * e.G;
              gq = -0.5f * gs * B.y * e.G;
            }
            // sums of gq dx, gq dy, gq dx^2, gq dx dy and gq dy^2; the mean and
            // conic gradients are formed from them once per entry (below)
            const float gdx = gq * e.dx, gdy = gq * e.dy;
            gv[0] = gdx;
            gv[1] = gdy;
            gv[2] = gdx * e.dx;
            gv[3] = gdx * e.dy;
            gv[4] = gdy * e.dy;
            const float dcol = g * e.sigma * Tr;  // dL/dc
            if (PIX) {
              const float dz = dcol * c * (1.f - c);
              gv[6] = dz;
              gv[7] = dz * ray.Y[0];
              gv[8] = dz * ray.Y[1];
              gv[9] = dz * ray.Y[2];
              gY[0] = fmaf(dz, cz.y, gY[0]);
              gY[1] = fmaf(dz, cz.z, gY[1]);
              gY[2] = fmaf(dz, cz.w, gY[2]);
            } else {
              gv[6] = dcol;
            }
          }
        }
        // sum the quarter's 8 lanes (each quarter has its own entry k)
        if (__any_sync(0xffffffffu, act)) {
          if (PIX) {
            const int comp = quarter_reduce10(gv);
            if (has) {
              if (gv[0] != 0.f) atomicAdd(&s_acc[k][comp], gv[0]);
              if ((lane & 3) == 0 && gv[8] != 0.f) atomicAdd(&s_acc[k][(lane & 4) ? 9 : 8], gv[8]);
            }
          } else {
            const int comp = quarter_reduce8(gv);
            if (has && gv[0] != 0.f) atomicAdd(&s_acc[k][comp], gv[0]);
          }
        }
      }
    }
    __syncthreads();
    for (int e = tid; e < cnt; e += NT) {
      const float *acc = s_acc[e];
      bool nz = (acc[0] != 0.f) | (acc[1] != 0.f) | (acc[2] != 0.f) | (acc[3] != 0.f) |
                (acc[4] != 0.f) | (acc[5] != 0.f) | (acc[6] != 0.f);
      if (PIX) nz |= (acc[7] != 0.f) | (acc[8] != 0.f) | (acc[9] != 0.f);
      if (nz) {
        float4 *dst = a.grad2d + 2 * (rec_base + s_id[e]);
        // dq/du = 2 (a dx + b dy), dq/dv = 2 (b dx + c dy), dq/db = 2 dx dy
        // the record holds CONIC_SCALE (a, 2b, c)
        const float ca = s_a[e].z * INV_CONIC_SCALE, cb = (0.5f * INV_CONIC_SCALE) * s_a[e].w,
                    cc = s_b[e].x * INV_CONIC_SCALE;
        const float du = 2.f * fmaf(ca, acc[0], cb * acc[1]);
        const float dv = 2.f * fmaf(cb, acc[0], cc * acc[1]);
        atomicAdd(dst, make_float4(du, dv, acc[2], 2.f * acc[3]));
        atomicAdd(dst + 1, make_float4(acc[4], acc[5], acc[6], 0.f));
        if (PIX) atomicAdd(a.grad_h + rec_base + s_id[e], make_float4(acc[7], acc[8], acc[9], 0.f));
      }
    }
    __syncthreads();
  }
  if (PIX && a.pose_grad) {
    // Y_1(d / |d|), d = W^T rc: dL/dW[r][c] = rc[r] dL/dd[c]
    float w9[9];
    const bool mine = tg.inside && ((gY[0] != 0.f) | (gY[1] != 0.f) | (gY[2] != 0.f));
    const float ddh[3] = {-SH_C1 * gY[2], -SH_C1 * gY[0], SH_C1 * gY[1]};
    const float dot = ddh[0] * ray.dh[0] + ddh[1] * ray.dh[1] + ddh[2] * ray.dh[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float dd = mine ? (ddh[c] - ray.dh[c] * dot) * ray.inv : 0.f;
#pragma unroll
      for (int r = 0; r < 3; ++r) w9[3 * r + c] = ray.rc[r] * dd;
    }
    if (__any_sync(0xffffffffu, mine)) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w9[i] += __shfl_xor_sync(0xffffffffu, w9[i], o);
      }
      if ((tid & 31) == 0)
#pragma unroll
        for (int i = 0; i < 9; ++i) atomicAdd(&sm.pose[i], w9[i]);
    }
    __syncthreads();
    if (tid < 9) {
      const float x = sm.pose[tid];
      if (x != 0.f) atomicAdd(a.pose_grad + 12 * (int64_t)tg.v + 4 * (tid / 3) + tid % 3, x);
      sm.pose[tid] = 0.f;
    }
  }
}

template <int T, int BATCH, bool PIX>
__global__ void __launch_bounds__(T *T, bwd_min_blocks<T>()) raster_bwd_kernel(RasterArgs a) {
  __shared__ BwdSmem<BATCH, PIX> sm;
  __shared__ uint32_t s_item;
  if (PIX && threadIdx.x < 12) sm.pose[threadIdx.x] = 0.f;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= (uint32_t)a.s.total_tiles) break;
    const int64_t gt = a.order[item];
    bwd_tile<T, BATCH, PIX>(a, gt, sm);
    if (a.req_end && threadIdx.x == 0)
      atomicMax(a.req_end + a.s.view[find_view(a.s.view, a.s.V, gt)].req, global_ns());
  }
}

// ---- warp-streamed rasterisers (staging depth 32) ----
// Every warp takes its own (tile, 8 x 4 region) item from the queue, stages 32
// list entries at a time in its own slice of shared memory and never waits
// for the other warps of its block. Item i is region i % NW of tile
// order[i / NW] (NW = regions per tile), so the regions of one tile are taken
// together and share its list in L1/L2. The backward sums a batch's 2D
// gradients per entry in the warp's slice and sends the non-zero sums to
// global memory with vector atomics.

constexpr int WARPS = 8;  // warps per block of the warp-streamed kernels

__device__ __forceinline__ uint32_t warp_next_item(uint32_t *counter) {
  uint32_t it = 0;
  if ((threadIdx.x & 31) == 0) it = atomicAdd(counter, 1u);
  return __shfl_sync(0xffffffffu, it, 0);
}

// ---- per-lane walks ----
// Lane l owns pixel (l & 7, l >> 3) of the warp's 8 x 4 region. Every staged
// entry turns its ellipse box into a 32-bit mask of the region's pixels whose
// centres it covers; a bit-matrix transpose across the warp then gives each
// lane the staged entries covering its own pixel, and each lane walks only
// those (in list order). A lane evaluates far fewer entries than a group of
// lanes sharing one walk would, and no lane waits for a group.

// Warp-wide transpose of a 32 x 32 bit matrix: lane r holds row r on entry;
// on return lane c holds column c (bit r = bit c of row r). Five rounds of
// block swaps (16, 8, 4, 2, 1).
__device__ __forceinline__ uint32_t transpose32(uint32_t x) {
  const int lane = threadIdx.x & 31;
  constexpr uint32_t LO[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const int d = 16 >> r;
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, d);
    x = (lane & d) ? ((x & ~LO[r]) | ((y >> d) & LO[r])) : ((x & LO[r]) | ((y << d) & ~LO[r]));
  }
  return x;
}

// Pixels of an 8 x 4 region whose centres lie in the box (x0, x1, y0, y1):
// bit y * 8 + x for pixel centre (cx + x, cy + y).
__device__ __forceinline__ uint32_t region_cover(float4 b, float cx, float cy) {
  const int x0 = max(0, __float2int_ru(b.x - cx)), x1 = min(7, __float2int_rd(b.y - cx));
  const int y0 = max(0, __float2int_ru(b.z - cy)), y1 = min(3, __float2int_rd(b.w - cy));
  if (x0 > x1 || y0 > y1) return 0u;
  const uint32_t row = (0xffu >> (7 - x1)) & (0xffu << x0);
  const uint32_t rows = (0xffffffffu >> (8 * (3 - y1))) & (0xffffffffu << (8 * y0));
  return (row * 0x01010101u) & rows;
}

// The 8 x 4 pixel region of a work item, lane l at pixel (l & 7, l >> 3).
struct Region {
  int v, H, W, wx0, wy0, px, py;
  bool inside;
  int64_t rec_base, img_off, n_req;
  // tile edge T (8, 16 or 32): T / 8 regions per tile row
  __device__ __forceinline__ Region(const RenderShape &s, int64_t gt, int region, int T) {
    v = find_view(s.view, s.V, gt);
    const ViewTab vt = s.view[v];
    H = vt.H;
    W = vt.W;
    rec_base = vt.rec_off;
    img_off = vt.img_off;
    n_req = s.req[vt.req].n;
    const int64_t local = gt - vt.tile_base;
    const int tyi = (int)(local / vt.tiles_x), txi = (int)(local - (int64_t)tyi * vt.tiles_x);
    const int WX = T / 8;
    wx0 = txi * T + (region % WX) * 8;
    wy0 = tyi * T + (region / WX) * 4;
    const int lane = threadIdx.x & 31;
    px = wx0 + (lane & 7);
    py = wy0 + (lane >> 3);
    inside = px < W && py < H;
  }
  __device__ __forceinline__ int64_t pixel() const { return img_off + (int64_t)py * W + px; }
};

template <int T, bool PIX>
__device__ __forceinline__ void fwd_lane_item(const RasterArgs &a, int64_t gt, int region, float4 *sA,
                                              float4 *sB, float4 *sC) {
  const int lane = threadIdx.x & 31;
  const Region rg(a.s, gt, region, T);
  const uint2 range = a.ranges[gt];
  const uint32_t *vals = a.vals;
  const float px = rg.px + 0.5f, py = rg.py + 0.5f;
  const float cx = rg.wx0 + 0.5f, cy = rg.wy0 + 0.5f;
  PixRay ray;
  if (PIX) pixel_ray(a.world_to_cam + 12 * rg.v, a.detector + 5 * rg.v, rg.H, rg.W, px, py, ray);
  float Tr = 1.f, C = 0.f;
  uint32_t last = 0;
  bool done = !rg.inside;
  // software pipeline: the list ids two batches ahead and the records one
  // batch ahead are in flight while a batch is walked
  uint32_t id1 = 0xffffffffu, id2 = 0xffffffffu;
  float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0;
  if (range.x + lane < range.y) id1 = vals[range.x + lane];
  if (range.x + 32 + lane < range.y) id2 = vals[range.x + 32 + lane];
  if (id1 < rg.n_req) { const int64_t r = rg.rec_base + id1; n0 = a.rec[2 * r]; n1 = a.rec[2 * r + 1]; }
  for (uint32_t b0 = range.x; b0 < range.y; b0 += 32) {
    if (__all_sync(0xffffffffu, done)) break;
    const uint32_t j = b0 + lane;
    uint32_t cover = 0;
    const uint32_t id = id1;
    const float4 r0 = n0, r1 = n1;
    id1 = id2;
    id2 = 0xffffffffu;
    if (b0 + 64 + lane < range.y) id2 = vals[b0 + 64 + lane];
    if (id1 < rg.n_req) { const int64_t r = rg.rec_base + id1; n0 = a.rec[2 * r]; n1 = a.rec[2 * r + 1]; }
    if (j < range.y) {
      if (id < rg.n_req) {
        const int64_t r = rg.rec_base + id;
        sA[lane] = r0;
        sB[lane] = r1;
        if (PIX) sC[lane] = a.rec2[r];
        cover = region_cover(ellipse_box(r0, r1, a.P.q_max), cx, cy);
      }
    }
    __syncwarp();
    uint32_t mine = transpose32(cover);  // staged entries covering this lane's pixel
    if (done) mine = 0;
    const uint32_t pos1 = b0 - range.x + 1u;  // 1 + list position of staged entry 0
    const int trips = (int)__reduce_max_sync(0xffffffffu, (uint32_t)__popc(mine));
    for (int t = 0; t < trips; ++t) {
      if (mine == 0) continue;
      const int k = __ffs(mine) - 1;
      mine &= mine - 1;
      const float4 A = sA[k], B = sB[k];
      PairEval e;
      if (!eval_pair(A.x, A.y, A.z, A.w, B.x, B.y, px, py, a.P, e)) continue;
      const float Tn = __fmaf_rn(-Tr, e.sigma, Tr);  // T (1 - sigma)
      if (Tn < a.P.t_min) {
        done = true;
        mine = 0;
        continue;
      }
      const float col = PIX ? pixel_colour(ray, sC[k]) : B.z;
      C = fmaf(col * e.sigma, Tr, C);
      Tr = Tn;
      last = pos1 + (uint32_t)k;
    }
    __syncwarp();  // the slice is rewritten by the next batch
  }
  if (rg.inside) {
    const int64_t pix = rg.pixel();
    a.image[pix] = C;
    a.t_final[pix] = Tr;
    a.n_last[pix] = last;
  }
}

// Resident blocks per SM asked of the register allocator. WIDE: eight (32
// registers, a few bytes spilled; 64 warps per SM: 1.48 -> 1.42 ms at 64
// poses, where six blocks at 40 registers measured 1.69 and five at 48 1.48),
// for renders with several work items per warp slot. Otherwise five (48
// registers), whose warps finish an item sooner: one 512^2 view, 0.078 ->
// 0.069 ms. Per-pixel directions always take five (their walk would spill).
template <int T, bool PIX, bool WIDE>
__global__ void __launch_bounds__(WARPS * 32, WIDE ? 8 : 5) raster_fwd_warp_kernel(RasterArgs a) {
  constexpr int NW = T * T / 32;
  __shared__ float4 s_a[WARPS][32], s_b[WARPS][32], s_c[WARPS][PIX ? 32 : 1];
  const int w = threadIdx.x >> 5;
  const uint64_t n_items = (uint64_t)a.s.total_tiles * NW;
  for (;;) {
    const uint32_t item = warp_next_item(a.counter);
    if (item >= n_items) break;
    const int64_t gt = a.order[item / NW];
    fwd_lane_item<T, PIX>(a, gt, (int)(item % NW), s_a[w], s_b[w], s_c[w]);
    if (a.req_end && (threadIdx.x & 31) == 0)
      atomicMax(a.req_end + a.s.view[find_view(a.s.view, a.s.V, gt)].req, global_ns());
  }
}

template <int T, bool PIX>
__device__ __forceinline__ void bwd_warp_item(const RasterArgs &a, int64_t gt, int region, float4 *sA,
                                              float4 *sB, float4 *sC, uint32_t *sId,
                                              float (*sAcc)[n_acc<PIX>()]) {
  const int lane = threadIdx.x & 31;
  const TileGeom<T> tg(a.s, gt, region);
  const uint2 range = a.ranges[tg.gtile];
  const uint32_t *vals = a.vals;
  const float px = tg.px + 0.5f, py = tg.py + 0.5f;
  PixRay ray;
  float gY[3] = {0.f, 0.f, 0.f};
  if (PIX) pixel_ray(a.world_to_cam + 12 * tg.v, a.detector + 5 * tg.v, tg.H, tg.W, px, py, ray);
  float Tr = 1.f, g = 0.f;
  uint32_t last = 0;
  if (tg.inside) {
    const int64_t pix = tg.pixel();
    Tr = a.t_final_in[pix];
    last = a.n_last_in[pix];
    g = a.dL_dimage[pix];
  }
  if (g == 0.f) last = 0;  // nothing to propagate from this pixel
  if (last > range.y - range.x) last = range.y - range.x;  // never read past the list
  uint32_t max_last = last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) max_last = max(max_last, __shfl_xor_sync(0xffffffffu, max_last, o));
  uint32_t qlast = last;
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) qlast = max(qlast, __shfl_xor_sync(0xffffffffu, qlast, o));
  const uint32_t ql0 = __shfl_sync(0xffffffffu, qlast, 0), ql1 = __shfl_sync(0xffffffffu, qlast, 8);
  const uint32_t ql2 = __shfl_sync(0xffffffffu, qlast, 16), ql3 = __shfl_sync(0xffffffffu, qlast, 24);
  float S = 0.f;
  for (int64_t hi = max_last; hi > 0; hi -= 32) {
    const int64_t lo = hi > 32 ? hi - 32 : 0;
    const int cnt = (int)(hi - lo);
    // lane e stages list position hi - 1 - e (batches run back to front)
    const bool ok = lane < cnt;
    float4 box = empty_box();
    if (ok) {
      const uint32_t id = vals[range.x + (uint32_t)(hi - 1 - lane)];
      if (id < tg.n_req) {  // else only after a capacity overflow
        const int64_t r = tg.rec_base + id;
        const float4 r0 = a.rec[2 * r], r1 = a.rec[2 * r + 1];
        sA[lane] = r0;
        sB[lane] = r1;
        if (PIX) sC[lane] = a.rec2[r];
        box = ellipse_box(r0, r1, a.P.q_max);
      }
      sId[lane] = id;
    }
#pragma unroll
    for (int c = 0; c < n_acc<PIX>(); ++c) sAcc[lane][c] = 0.f;
    __syncwarp();
    const uint32_t pe = (uint32_t)(hi - 1 - lane);
    const uint32_t m0 = __ballot_sync(0xffffffffu, ok && pe < ql0 && !tg.misses_q(box, 0));
    const uint32_t m1 = __ballot_sync(0xffffffffu, ok && pe < ql1 && !tg.misses_q(box, 1));
    const uint32_t m2 = __ballot_sync(0xffffffffu, ok && pe < ql2 && !tg.misses_q(box, 2));
    const uint32_t m3 = __ballot_sync(0xffffffffu, ok && pe < ql3 && !tg.misses_q(box, 3));
    const int qi = lane >> 3;
    uint32_t mine = qi == 0 ? m0 : (qi == 1 ? m1 : (qi == 2 ? m2 : m3));
    while (__any_sync(0xffffffffu, mine != 0)) {
      const bool has = mine != 0;
      const int k = has ? __ffs(mine) - 1 : 0;
      if (has) mine &= mine - 1;
      const uint32_t pos = (uint32_t)(hi - 1 - k);
      float gv[PIX ? 10 : 8];
#pragma unroll
      for (int c = 0; c < (PIX ? 10 : 8); ++c) gv[c] = 0.f;
      bool act = has && pos < last;
      if (act) {
        const float4 A = sA[k], B = sB[k];
        PairEval e;
        act = eval_pair(A.x, A.y, A.z, A.w, B.x, B.y, px, py, a.P, e);
        if (act) {
          // 1 / (1 - sigma) with sigma <= alpha_max < 1
          const float inv_om = rcp_approx(__fsub_rn(1.f, e.sigma));
          Tr = Tr * inv_om;  // transmittance before this Gaussian
          float4 cz;
          if (PIX) cz = sC[k];
          const float c = PIX ? pixel_colour(ray, cz) : B.z;
          const float dC_dsigma = fmaf(c, Tr, -S * inv_om);
          S = fmaf(c * e.sigma, Tr, S);
          const float gs = g * dC_dsigma;
          float gq = 0.f;
          if (!(e.aG > a.P.alpha_max)) {
            gv[5] = gs * e.G;
            gq = -0.5f * gs * B.y * e.G;
          }
          // sums of gq dx, gq dy, gq dx^2, gq dx dy and gq dy^2; the mean and
          // conic gradients are formed from them once per entry (below)
          const float gdx = gq * e.dx, gdy = gq * e.dy;
          gv[0] = gdx;
          gv[1] = gdy;
          gv[2] = gdx * e.dx;
          gv[3] = gdx * e.dy;
          gv[4] = gdy * e.dy;
          const float dcol = g * e.sigma * Tr;  // dL/dc
          if (PIX) {
            const float dz = dcol * c * (1.f - c);
            gv[6] = dz;
            gv[7] = dz * ray.Y[0];
            gv[8] = dz * ray.Y[1];
            gv[9] = dz * ray.Y[2];
            gY[0] = fmaf(dz, cz.y, gY[0]);
            gY[1] = fmaf(dz, cz.z, gY[1]);
            gY[2] = fmaf(dz, cz.w, gY[2]);
          } else {
            gv[6] = dcol;
          }
        }
      }
      if (__any_sync(0xffffffffu, act)) {
        if (PIX) {
          const int comp = quarter_reduce10(gv);
          if (has) {
            if (gv[0] != 0.f) atomicAdd(&sAcc[k][comp], gv[0]);
            if ((lane & 3) == 0 && gv[8] != 0.f) atomicAdd(&sAcc[k][(lane & 4) ? 9 : 8], gv[8]);
          }
        } else {
          const int comp = quarter_reduce8(gv);
          if (has && gv[0] != 0.f) atomicAdd(&sAcc[k][comp], gv[0]);
        }
      }
    }
    __syncwarp();
    if (ok) {  // lane e sends entry e's sums
      const float *acc = sAcc[lane];
      bool nz = (acc[0] != 0.f) | (acc[1] != 0.f) | (acc[2] != 0.f) | (acc[3] != 0.f) |
                (acc[4] != 0.f) | (acc[5] != 0.f) | (acc[6] != 0.f);
      if (PIX) nz |= (acc[7] != 0.f) | (acc[8] != 0.f) | (acc[9] != 0.f);
      if (nz) {
        const int64_t r = tg.rec_base + sId[lane];
        float4 *dst = a.grad2d + 2 * r;
        // dq/du = 2 (a dx + b dy), dq/dv = 2 (b dx + c dy), dq/db = 2 dx dy
        // the record holds CONIC_SCALE (a, 2b, c)
        const float ca = sA[lane].z * INV_CONIC_SCALE, cb = (0.5f * INV_CONIC_SCALE) * sA[lane].w,
                    cc = sB[lane].x * INV_CONIC_SCALE;
        const float du = 2.f * fmaf(ca, acc[0], cb * acc[1]);
        const float dv = 2.f * fmaf(cb, acc[0], cc * acc[1]);
        atomicAdd(dst, make_float4(du, dv, acc[2], 2.f * acc[3]));
        atomicAdd(dst + 1, make_float4(acc[4], acc[5], acc[6], 0.f));
        if (PIX) atomicAdd(a.grad_h + r, make_float4(acc[7], acc[8], acc[9], 0.f));
      }
    }
    __syncwarp();
  }
  if (PIX && a.pose_grad) {
    // Y_1(d / |d|), d = W^T rc: dL/dW[r][c] = rc[r] dL/dd[c], summed over the warp
    const bool mine = tg.inside && ((gY[0] != 0.f) | (gY[1] != 0.f) | (gY[2] != 0.f));
    if (__any_sync(0xffffffffu, mine)) {
      float w9[9];
      const float ddh[3] = {-SH_C1 * gY[2], -SH_C1 * gY[0], SH_C1 * gY[1]};
      const float dot = ddh[0] * ray.dh[0] + ddh[1] * ray.dh[1] + ddh[2] * ray.dh[2];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float dd = mine ? (ddh[c] - ray.dh[c] * dot) * ray.inv : 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r) w9[3 * r + c] = ray.rc[r] * dd;
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w9[i] += __shfl_xor_sync(0xffffffffu, w9[i], o);
      }
      if (lane < 9) {
        float x = w9[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) if (lane == i) x = w9[i];
        if (x != 0.f) atomicAdd(a.pose_grad + 12 * (int64_t)tg.v + 4 * (lane / 3) + lane % 3, x);
      }
    }
  }
}

template <int T, bool PIX>
__global__ void __launch_bounds__(WARPS * 32, 4) raster_bwd_warp_kernel(RasterArgs a) {
  constexpr int NW = T * T / 32;
  __shared__ float4 s_a[WARPS][32], s_b[WARPS][32], s_c[WARPS][PIX ? 32 : 1];
  __shared__ uint32_t s_id[WARPS][32];
  __shared__ float s_acc[WARPS][32][n_acc<PIX>()];
  const int w = threadIdx.x >> 5;
  const uint64_t n_items = (uint64_t)a.s.total_tiles * NW;
  for (;;) {
    const uint32_t item = warp_next_item(a.counter);
    if (item >= n_items) break;
    const int64_t gt = a.order[item / NW];
    bwd_warp_item<T, PIX>(a, gt, (int)(item % NW), s_a[w], s_b[w], s_c[w], s_id[w], s_acc[w]);
    if (a.req_end && (threadIdx.x & 31) == 0)
      atomicMax(a.req_end + a.s.view[find_view(a.s.view, a.s.V, gt)].req, global_ns());
  }
}

// Backward of one (tile, region) item in two phases per staged batch of 32
// entries (back to front):
//  1. every lane walks the entries covering its pixel, from the last one the
//     forward pass added, recovering T and the suffix sum S, and stores two
//     numbers per (pixel, entry) it adds: A = dL/dsigma * G (0 where sigma
//     was clamped) and Bc = dL/dc = g sigma T;
//  2. after a transpose of the (pixel, entry) bits, lane e sums entry e's
//     numbers over its pixels in registers: sum A, sum Bc and the moments
//     sum A x, A y, A x^2, A x y, A y^2 of the pixel offsets (x, y) in the
//     region. With u' = u - (region origin), dx = u' - x, dy = v' - y and
//     dL/dq = -alpha A / 2, the sums of dL/dq dx, dL/dq dy, dL/dq dx^2, ...
//     that the mean and conic gradients need follow from those moments.
// No lane reduces another lane's values and no shared-memory atomic is used.
constexpr int AB_STRIDE = 32;  // float2 per pixel row of the (pixel, entry) table
constexpr int LANE_WARPS = 8;  // warps per block of the per-lane backward (3 blocks per SM)

struct LaneBwdSmem {
  float4 a[33], b[33];  // entry 32: a sentinel that no pixel adds
  uint32_t id[32];
  float2 ab[32 * AB_STRIDE];  // [pixel][entry ^ pixel]: (A, Bc)
};

template <int T>
__device__ __forceinline__ void bwd_lane_item(const RasterArgs &a, int64_t gt, int region, LaneBwdSmem &sm) {
  const int lane = threadIdx.x & 31;
  const Region rg(a.s, gt, region, T);
  const uint2 range = a.ranges[gt];
  const uint32_t *vals = a.vals;
  const float px = rg.px + 0.5f, py = rg.py + 0.5f;
  const float cx = rg.wx0 + 0.5f, cy = rg.wy0 + 0.5f;
  float Tr = 1.f, g = 0.f;
  uint32_t last = 0;
  if (rg.inside) {
    const int64_t pix = rg.pixel();
    Tr = a.t_final_in[pix];
    last = a.n_last_in[pix];
    g = a.dL_dimage[pix];
  }
  if (g == 0.f) last = 0;  // nothing to propagate from this pixel
  if (last > range.y - range.x) last = range.y - range.x;  // never read past the list
  if (lane == 0) {  // q' = -inf at every pixel
    sm.a[32] = make_float4(3.0e38f, 3.0e38f, -1.f, 0.f);
    sm.b[32] = make_float4(-1.f, 0.f, 0.f, 0.f);
  }
  // the walk carries g T and g S (Tr, S), so that g drops out of the per-pair
  // products: g dC/dsigma = c gT - gS / (1 - sigma), g dC/dc = sigma gT
  Tr *= g;
  uint32_t max_last = last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) max_last = max(max_last, __shfl_xor_sync(0xffffffffu, max_last, o));
  float S = 0.f;
  // software pipeline: the list ids two batches ahead and the records one
  // batch ahead are in flight while a batch is walked
  uint32_t id1 = 0xffffffffu, id2 = 0xffffffffu;
  float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0;
  if ((int64_t)lane < (int64_t)max_last) id1 = vals[range.x + (uint32_t)(max_last - 1 - lane)];
  if ((int64_t)max_last > 32 && (int64_t)lane < (int64_t)max_last - 32)
    id2 = vals[range.x + (uint32_t)(max_last - 33 - lane)];
  if (id1 < rg.n_req) { const int64_t r = rg.rec_base + id1; n0 = a.rec[2 * r]; n1 = a.rec[2 * r + 1]; }
  for (int64_t hi = max_last; hi > 0; hi -= 32) {
    const int cnt = (int)(hi > 32 ? 32 : hi);
    uint32_t cover = 0;
    const uint32_t id = id1;
    const float4 r0 = n0, r1 = n1;
    id1 = id2;
    id2 = 0xffffffffu;
    if (hi - 64 > 0 && (int64_t)lane < hi - 64) id2 = vals[range.x + (uint32_t)(hi - 65 - lane)];
    if (id1 < rg.n_req) { const int64_t r = rg.rec_base + id1; n0 = a.rec[2 * r]; n1 = a.rec[2 * r + 1]; }
    if (lane < cnt) {
      if (id < rg.n_req) {
        sm.a[lane] = r0;
        sm.b[lane] = r1;
        cover = region_cover(ellipse_box(r0, r1, a.P.q_max), cx, cy);
      }
      sm.id[lane] = id;
    }
    __syncwarp();
    uint32_t mine = transpose32(cover);
    // staged entries e >= hi - last lie before this pixel's last added Gaussian
    const int64_t skip = hi - (int64_t)last;
    mine &= skip <= 0 ? 0xffffffffu : (skip >= 32 ? 0u : (0xffffffffu << skip));
    uint32_t used = 0;
    const int trips = (int)__reduce_max_sync(0xffffffffu, (uint32_t)__popc(mine));
    // one entry per trip, written without branches (a lane past its last
    // entry evaluates the sentinel entry 32, whose q' is -inf, so that no
    // flag of its own is needed: 2.87 -> 2.84 ms): eval_pair's decisions, in
    // the same arithmetic. (Two entries per trip paid while the walk branched;
    // without branches the odd trip's padding costs more than the overlap
    // gives: 2.95 -> 2.93 ms.)
    // the next entry's record is read from shared memory while this one is
    // evaluated (2.92 -> 2.91 ms); the entry's own bit (the lowest of mine)
    // marks it walked and added (2.84 -> 2.83 ms)
    uint32_t bn = mine & (0u - mine);  // the next entry's bit (0 past the last)
    int kn = __popc(bn - 1u);          // its index: 32, the sentinel, past the last
    float4 An = sm.a[kn], Bn = sm.b[kn];
    for (int t = 0; t < trips; ++t) {
      const int k = kn;
      const uint32_t bit = bn;
      const float4 A = An, B = Bn;
      mine ^= bit;
      bn = mine & (0u - mine);
      kn = __popc(bn - 1u);
      An = sm.a[kn];
      Bn = sm.b[kn];
      const float dx = __fsub_rn(A.x, px), dy = __fsub_rn(A.y, py);
      const float tq = __fmaf_rn(A.w, dy, __fmul_rn(A.z, dx));
      const float q = __fmaf_rn(__fmul_rn(B.x, dy), dy, __fmul_rn(dx, tq));
      const float G = exp2_approx(q), aG = __fmul_rn(B.y, G), sigma = fminf(a.P.alpha_max, aG);
      const bool ok = !(q < a.P.q_lim || q > 0.f) && sigma >= a.P.alpha_min;
      // 1 / (1 - sigma) with sigma <= alpha_max < 1: the fast reciprocal's
      // relative error (~1 ulp) is far inside the gradient tolerance
      const float inv_om = rcp_approx(__fsub_rn(1.f, sigma));
      const float Tn = Tr * inv_om;
      const float g_dC = fmaf(B.z, Tn, -S * inv_om);  // g dC/dsigma
      const float sT = sigma * Tn;  // g dC/dc, shared with S's update (2.83 -> 2.81 ms)
      const float Sn = fmaf(B.z, sT, S);
      const float gA = (aG > a.P.alpha_max) ? 0.f : g_dC * G;
      if (ok) sm.ab[lane * AB_STRIDE + (k ^ lane)] = make_float2(gA, sT);
      Tr = ok ? Tn : Tr;
      S = ok ? Sn : S;
      used |= ok ? bit : 0u;
    }
    __syncwarp();
    uint32_t pm = transpose32(used);  // lane e: the pixels that added entry e
    if (pm) {
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f, s5 = 0.f, s6 = 0.f;
      do {  // two pixels per trip: half the loop overhead, two loads in flight
        const int p = __ffs(pm) - 1;
        pm &= pm - 1;
        const bool two = pm != 0;
        const int q = two ? __ffs(pm) - 1 : p;
        pm &= pm - 1;
        const float2 ab = sm.ab[p * AB_STRIDE + (lane ^ p)];
        float2 cd = sm.ab[q * AB_STRIDE + (lane ^ q)];
        if (!two) cd = make_float2(0.f, 0.f);
        // pixel offsets in the region by conversion (a table in shared memory
        // cost bank conflicts: 2.91 -> 2.89 ms without it)
        const float x = (float)(p & 7), y = (float)(p >> 3);
        const float x2 = (float)(q & 7), y2 = (float)(q >> 3);
        const float ax = ab.x * x, ay = ab.x * y, cx2 = cd.x * x2, cy2 = cd.x * y2;
        s0 += ab.x + cd.x;
        s1 += ax + cx2;
        s2 += ay + cy2;
        s3 = fmaf(ax, x, fmaf(cx2, x2, s3));
        s4 = fmaf(ax, y, fmaf(cx2, y2, s4));
        s5 = fmaf(ay, y, fmaf(cy2, y2, s5));
        s6 += ab.y + cd.y;
      } while (pm);
      const float4 A = sm.a[lane], B = sm.b[lane];
      const float u = A.x - cx, v = A.y - cy;  // mean relative to pixel (0, 0)
      // sums over the entry's pixels of A dx, A dy, A dx^2, A dx dy, A dy^2
      const float sdx = fmaf(u, s0, -s1), sdy = fmaf(v, s0, -s2);
      const float sxx = fmaf(u, fmaf(u, s0, -2.f * s1), s3);
      const float sxy = fmaf(u, fmaf(v, s0, -s2), fmaf(-v, s1, s4));
      const float syy = fmaf(v, fmaf(v, s0, -2.f * s2), s5);
      const float hq = -0.5f * B.y;  // dL/dq = -alpha A / 2
      // dq/du = 2 (a dx + b dy), dq/dv = 2 (b dx + c dy), dq/db = 2 dx dy;
      // the record holds (a', 2b', c') = CONIC_SCALE (a, 2b, c) in A.z, A.w, B.x
      const float hk = hq * INV_CONIC_SCALE;
      const float gx = hk * sdx, gy = hk * sdy;
      const float du = fmaf(2.f * A.z, gx, A.w * gy);
      const float dv = fmaf(A.w, gx, 2.f * B.x * gy);
      float4 *dst = a.grad2d + 2 * (rg.rec_base + sm.id[lane]);
      atomicAdd(dst, make_float4(du, dv, hq * sxx, 2.f * hq * sxy));
      atomicAdd(dst + 1, make_float4(hq * syy, s0, s6, 0.f));
    }
    __syncwarp();  // the slice is rewritten by the next batch
  }
}

template <int T>
__global__ void __launch_bounds__(LANE_WARPS * 32, 3) raster_bwd_lane_kernel(RasterArgs a) {
  constexpr int NW = T * T / 32;
  extern __shared__ __align__(16) unsigned char lane_smem[];
  LaneBwdSmem &sm = reinterpret_cast<LaneBwdSmem *>(lane_smem)[threadIdx.x >> 5];
  const uint64_t n_items = (uint64_t)a.s.total_tiles * NW;
  for (;;) {
    const uint32_t item = warp_next_item(a.counter);
    if (item >= n_items) break;
    const int64_t gt = a.order[item / NW];
    bwd_lane_item<T>(a, gt, (int)(item % NW), sm);
    if (a.req_end && (threadIdx.x & 31) == 0)
      atomicMax(a.req_end + a.s.view[find_view(a.s.view, a.s.V, gt)].req, global_ns());
  }
}

constexpr size_t LANE_BWD_SMEM = LANE_WARPS * sizeof(LaneBwdSmem);

// ---- work order: view by view, and within a view the tiles by descending
// list length (bucketed by log2). At any time the persistent blocks then work
// on a few views, whose records and gradient accumulators stay in L2 while
// the longest lists of each view still start first. ----

constexpr int LPT_BUCKETS = 34;  // 0 = empty list, b = 1 + floor(log2(len))

__device__ __forceinline__ int lpt_bucket(uint2 r) {
  const uint32_t len = r.y - r.x;
  return len ? 33 - __clz(len) : 0;  // 1..33
}

// One block per view: a counting sort of the view's tiles by bucket, longest
// bucket first, written to order[tile_base .. tile_base + tiles).
__global__ void __launch_bounds__(256) tile_order_view_kernel(const ViewTab *view, const uint2 *ranges,
                                                              uint32_t *order) {
  __shared__ uint32_t h[LPT_BUCKETS], start[LPT_BUCKETS];
  const int v = blockIdx.x;
  const int64_t t0 = view[v].tile_base, nt = view[v + 1].tile_base - t0;
  for (int b = threadIdx.x; b < LPT_BUCKETS; b += blockDim.x) h[b] = 0;
  __syncthreads();
  for (int64_t t = threadIdx.x; t < nt; t += blockDim.x) atomicAdd(&h[lpt_bucket(ranges[t0 + t])], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int b = LPT_BUCKETS - 1; b >= 0; --b) {
      start[b] = run;
      run += h[b];
      h[b] = 0;  // reused as the bucket's cursor
    }
  }
  __syncthreads();
  for (int64_t t = threadIdx.x; t < nt; t += blockDim.x) {
    const int b = lpt_bucket(ranges[t0 + t]);
    order[t0 + start[b] + atomicAdd(&h[b], 1u)] = (uint32_t)(t0 + t);
  }
}


// Resident blocks per SM of a kernel, cached per (device, kernel); the query
// is not a stream operation, so it is also legal while a stream is captured.
int blocks_per_sm(void (*k)(RasterArgs), int threads, size_t dyn_smem = 0) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(dev, reinterpret_cast<const void *>(k));
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, dyn_smem) != cudaSuccess || n < 1) n = 1;
  cache[key] = n;
  return n;
}

template <int T, int BATCH, bool PIX>
void launch_fwd_t(const RasterArgs &a, cudaStream_t st) {
  if (a.s.total_tiles <= 0) return;
  auto k = raster_fwd_kernel<T, BATCH, PIX>;
  int64_t grid = (int64_t)blocks_per_sm(k, T * T) * device_sms();
  if (grid > a.s.total_tiles) grid = a.s.total_tiles;
  LaunchScope ls(KID_RASTER_FWD, st);
  k<<<(unsigned)grid, T * T, 0, st>>>(a);
}

template <int T, int BATCH, bool PIX>
void launch_bwd_t(const RasterArgs &a, cudaStream_t st) {
  if (a.s.total_tiles <= 0) return;
  auto k = raster_bwd_kernel<T, BATCH, PIX>;
  int64_t grid = (int64_t)blocks_per_sm(k, T * T) * device_sms();
  if (grid > a.s.total_tiles) grid = a.s.total_tiles;
  LaunchScope ls(KID_RASTER_BWD, st);
  k<<<(unsigned)grid, T * T, 0, st>>>(a);
}

template <int T, bool PIX>
void launch_fwd_warp_t(const RasterArgs &a, cudaStream_t st) {
  const int64_t need = (a.s.total_tiles * (T * T / 32) + WARPS - 1) / WARPS;
  auto k = raster_fwd_warp_kernel<T, PIX, false>;
  if constexpr (!PIX) {
    // at least two items for each warp of eight resident blocks per SM
    if (need >= 2 * 8 * (int64_t)device_sms()) k = raster_fwd_warp_kernel<T, PIX, true>;
  }
  int64_t grid = (int64_t)blocks_per_sm(k, WARPS * 32) * device_sms();
  if (grid > need) grid = need;
  LaunchScope ls(KID_RASTER_FWD, st);
  k<<<(unsigned)grid, WARPS * 32, 0, st>>>(a);
}

template <int T>
void launch_bwd_lane_t(const RasterArgs &a, cudaStream_t st) {
  if (prepare_raster_kernels() != cudaSuccess) return;  // surfaces via cudaGetLastError
  auto k = raster_bwd_lane_kernel<T>;
  const int64_t need = (a.s.total_tiles * (T * T / 32) + LANE_WARPS - 1) / LANE_WARPS;
  int64_t grid = (int64_t)blocks_per_sm(k, LANE_WARPS * 32, LANE_BWD_SMEM) * device_sms();
  if (grid > need) grid = need;
  LaunchScope ls(KID_RASTER_BWD, st);
  k<<<(unsigned)grid, LANE_WARPS * 32, LANE_BWD_SMEM, st>>>(a);
}

template <int T, bool PIX>
void launch_bwd_warp_t(const RasterArgs &a, cudaStream_t st) {
  if (!PIX) {
    launch_bwd_lane_t<T>(a, st);
    return;
  }
  auto k = raster_bwd_warp_kernel<T, PIX>;
  const int64_t need = (a.s.total_tiles * (T * T / 32) + WARPS - 1) / WARPS;
  int64_t grid = (int64_t)blocks_per_sm(k, WARPS * 32) * device_sms();
  if (grid > need) grid = need;
  LaunchScope ls(KID_RASTER_BWD, st);
  k<<<(unsigned)grid, WARPS * 32, 0, st>>>(a);
}

// The warp-streamed kernels count items in 32 bits.
bool warp_mode(const RenderShape &s, const ddgs_workspace &ws) {
  return ws.batch_depth == 32 && s.total_tiles * (int64_t)(s.tile * s.tile / 32) < (int64_t(1) << 32);
}

template <bool PIX>
void fwd_warp_dispatch(const RasterArgs &a, int tile, cudaStream_t st) {
  if (a.s.total_tiles <= 0) return;
  switch (tile) {
    case 8: launch_fwd_warp_t<8, PIX>(a, st); break;
    case 16: launch_fwd_warp_t<16, PIX>(a, st); break;
    default: launch_fwd_warp_t<32, PIX>(a, st); break;
  }
}

template <bool PIX>
void bwd_warp_dispatch(const RasterArgs &a, int tile, cudaStream_t st) {
  if (a.s.total_tiles <= 0) return;
  switch (tile) {
    case 8: launch_bwd_warp_t<8, PIX>(a, st); break;
    case 16: launch_bwd_warp_t<16, PIX>(a, st); break;
    default: launch_bwd_warp_t<32, PIX>(a, st); break;
  }
}

template <int BATCH, bool PIX>
void fwd_dispatch(const RasterArgs &a, int tile, cudaStream_t st) {
  switch (tile) {
    case 8: launch_fwd_t<8, BATCH, PIX>(a, st); break;
    case 16: launch_fwd_t<16, BATCH, PIX>(a, st); break;
    default: launch_fwd_t<32, BATCH, PIX>(a, st); break;
  }
}

template <int BATCH, bool PIX>
void bwd_dispatch(const RasterArgs &a, int tile, cudaStream_t st) {
  switch (tile) {
    case 8: launch_bwd_t<8, BATCH, PIX>(a, st); break;
    case 16: launch_bwd_t<16, BATCH, PIX>(a, st); break;
    default: launch_bwd_t<32, BATCH, PIX>(a, st); break;
  }
}

}  // namespace

void launch_tile_order(const RenderShape &s, ddgs_workspace &ws, cudaStream_t st) {
  if (s.total_tiles <= 0 || s.V <= 0) return;
  LaunchScope ls(KID_TILE_ORDER, st);
  tile_order_view_kernel<<<(unsigned)s.V, 256, 0, st>>>(s.view, ws.ranges, ws.order);
}

void launch_raster_fwd(const RenderShape &s, const RasterParams &p, ddgs_workspace &ws,
                       float *image, float *t_final, uint32_t *n_last, const PixelRays *pr,
                       cudaStream_t st) {
  RasterArgs a{};
  a.s = s;
  a.P = p;
  a.rec = ws.rec;
  a.vals = ws.vals;
  a.ranges = ws.ranges;
  a.image = image;
  a.t_final = t_final;
  a.n_last = n_last;
  a.order = ws.order;
  a.counter = ws.queue;
  a.req_end = ws.req_time ? ws.req_time + 1 : nullptr;
  cudaMemsetAsync(ws.queue, 0, sizeof(uint32_t), st);
  if (pr) {  // per-pixel ray angles: one staging depth
    a.rec2 = ws.rec2;
    a.world_to_cam = pr->world_to_cam;
    a.detector = pr->detector;
    if (warp_mode(s, ws)) fwd_warp_dispatch<true>(a, s.tile, st);
    else fwd_dispatch<256, true>(a, s.tile, st);
  } else if (warp_mode(s, ws)) {
    fwd_warp_dispatch<false>(a, s.tile, st);
  } else if (ws.batch_depth == 128) {
    fwd_dispatch<128, false>(a, s.tile, st);
  } else if (ws.batch_depth == 512) {
    fwd_dispatch<512, false>(a, s.tile, st);
  } else {
    fwd_dispatch<256, false>(a, s.tile, st);
  }
}

void launch_raster_bwd(const RenderShape &s, const RasterParams &p, ddgs_workspace &ws,
                       const float *dL_dimage, const float *t_final, const uint32_t *n_last,
                       const PixelRays *pr, cudaStream_t st) {
  RasterArgs a{};
  a.s = s;
  a.P = p;
  a.rec = ws.rec;
  a.vals = ws.vals;
  a.ranges = ws.ranges;
  a.grad2d = ws.grad2d;
  a.dL_dimage = dL_dimage;
  a.t_final_in = t_final;
  a.n_last_in = n_last;
  a.order = ws.order;
  a.counter = ws.queue + 1;
  a.req_end = ws.req_time ? ws.req_time + 1 + s.R : nullptr;
  cudaMemsetAsync(ws.queue + 1, 0, sizeof(uint32_t), st);
  if (pr) {  // per-pixel ray angles: one staging depth
    a.rec2 = ws.rec2;
    a.grad_h = ws.grad_h;
    a.world_to_cam = pr->world_to_cam;
    a.detector = pr->detector;
    a.pose_grad = pr->pose_grad;
    if (warp_mode(s, ws)) bwd_warp_dispatch<true>(a, s.tile, st);
    else bwd_dispatch<256, true>(a, s.tile, st);
  } else if (warp_mode(s, ws)) {
    bwd_warp_dispatch<false>(a, s.tile, st);
  } else if (ws.batch_depth == 128) {
    bwd_dispatch<128, false>(a, s.tile, st);
  } else if (ws.batch_depth == 512) {
    bwd_dispatch<512, false>(a, s.tile, st);
  } else {
    bwd_dispatch<256, false>(a, s.tile, st);
  }
}

cudaError_t prepare_raster_kernels() {
  // the per-lane backward keeps its (pixel, entry) tables in dynamic shared
  // memory beyond the default 48 KiB; set once per device, outside any capture
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  for (auto k : {raster_bwd_lane_kernel<8>, raster_bwd_lane_kernel<16>, raster_bwd_lane_kernel<32>}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LANE_BWD_SMEM);
    if (e != cudaSuccess) return e;
  }
  if (dev >= 0 && dev < 64) done[dev] = true;
  return cudaSuccess;
}

// Streaming multiprocessors of the current device (cached per device).
int device_sms() {
  static int sms[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 152;
  if (!sms[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = n > 0 ? n : 152;
  }
  return sms[dev];
}

}  // namespace ddgs
