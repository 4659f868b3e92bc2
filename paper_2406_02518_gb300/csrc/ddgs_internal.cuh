// ddgs_internal.cuh -- shared declarations of the sm_103a DRR splatting kernels.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/ddgs.h"

namespace ddgs {

constexpr int K = DDGS_FEAT_DIM;          // features per Gaussian
constexpr int PRE_THREADS = 256;          // Gaussians per preprocess block
constexpr int VIEW_CHUNK = 64;            // views staged in shared memory at once
// Binning (bin.cu): blocks of Gaussians of one view count and place their
// pairs with per-tile counters in shared memory, over bands of at most
// BIN_HIST_MAX tiles; every tile list is then ordered in shared memory.
constexpr int BIN_HIST_MAX = 8192;           // tiles of one band
constexpr int64_t BIN_CHUNK = 2048;          // Gaussians per binning block (their pairs,
                                             // about two per Gaussian, are staged at once)
constexpr int64_t BIN_SLOT_BUDGET = int64_t(1) << 24;  // per-block tile counters of a render
constexpr int BIN_LIST_LONG = 8192;          // longest list ordered by one block at once
constexpr int64_t BIN_MAX_PAIRS = (int64_t(1) << 31) - 1;  // offsets leave bit 31 free
constexpr float SH_C1 = 0.48860251190291992f;  // sqrt(3 / (4 pi))

// Device status bits (latched in the workspace): a tile list did not fit the
// reserved pair capacity; an input parameter was NaN or infinite.
enum : int32_t { ST_CAPACITY = 1, ST_NONFINITE = 2 };

// A batch is R requests; request r owns a contiguous range of Gaussians (its
// own cloud and bases) and a contiguous range of views; every view has its
// own detector size. The single-cloud calls are the case R = 1. The tables
// live in device memory (entry R / V is a sentinel holding the totals).
struct ReqTab {
  int64_t g_off;     // first Gaussian of the request in the parameter arrays
  int64_t n;         // Gaussians of the request
  int64_t n_iso;     // its first n_iso Gaussians are isotropic
  int64_t iso_row;   // first row of the request in feat_iso
  int64_t dir_row;   // first row of the request in feat_dir
  int64_t blk_base;  // first preprocess block of the request
  int32_t v_off;     // first view of the request
  int32_t n_views;
};

struct ViewTab {
  int64_t tile_base;  // first global tile of the view
  int64_t rec_off;    // first (view, Gaussian) record of the view
  int64_t img_off;    // first pixel of the view in the concatenated images
  int32_t req, H, W, tiles_x;
  // binning: (band, chunk) blocks of the view, and their tile counters
  int64_t item_base;  // first binning block of the view
  int64_t hist_base;  // first tile counter of the view
  int32_t chunks;     // Gaussian chunks (0 for an empty request)
  int32_t band_w, band_h, bands_x;  // bands of band_w x band_h tiles, row-major
};

// Per-view constants staged in shared memory by the preprocess kernels
// (IEEE-exact where the binning depends on them).
struct ViewConst {
  float W[9];   // rotation rows
  float t[3];
  float wt[3];  // W^T t: the source sits at -wt in world coordinates
  float fu, fv, cu, cv, sdd;
  int32_t H, Wd, tiles_x;
  int64_t tile_base, rec_off;
};

// Tile lists sorted by the binning, by length class: 2 to 32 entries (one
// warp), up to 1024, up to 2048, up to BIN_LIST_LONG (one block each; longer
// lists are cut into BIN_LIST_LONG-entry chunks here) and longer (chunks
// merged).
enum : int { LIST_WARP = 0, LIST_SHORT, LIST_MID, LIST_BLOCK, LIST_LONG, LIST_CLASSES };
struct BinLists {
  uint64_t *item[LIST_CLASSES];  // entries: global tile << 24 | chunk
  uint32_t *count;               // device [LIST_CLASSES]
};

// Parameters shared by the rasterisers. q_lim = CONIC_SCALE q_max: the q cutoff
// in the units of the records' scaled conic (see eval_pair).
struct RasterParams {
  float alpha_min, alpha_max, t_min, q_max, q_lim;
};

// The records hold the conic multiplied by -log2(e) / 2, so that the
// rasterisers' q' = CONIC_SCALE q is already the exponent of
// G = exp(-q / 2) = 2^q'. INV_CONIC_SCALE = 1 / CONIC_SCALE = -2 ln 2.
constexpr float CONIC_SCALE = -0.72134752044448170368f;
constexpr float INV_CONIC_SCALE = -1.38629436111989061883f;

// Everything the kernels need about one render (passed by value).
struct RenderShape {
  int32_t R, V, tile, hist_area;  // hist_area: largest band (tiles) of any view
  int64_t n_total, total_tiles, records, pixels, n_blocks;
  int64_t n_items, hist_slots;    // binning blocks and their tile counters
  const ReqTab *req;    // device [R + 1]
  const ViewTab *view;  // device [V + 1]
};

// Largest r with tab[r].blk_base <= b (the sentinel tab[R] holds the total).
__device__ __forceinline__ int find_request(const ReqTab *tab, int R, int64_t b) {
  int lo = 0, hi = R;  // invariant: tab[lo].blk_base <= b < tab[hi].blk_base
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (tab[mid].blk_base <= b) lo = mid; else hi = mid;
  }
  return lo;
}

// Largest v with tab[v].item_base <= i: the view of binning block i (views
// without blocks share their successor's item_base and are skipped).
__device__ __forceinline__ int find_item_view(const ViewTab *tab, int V, int64_t i) {
  int lo = 0, hi = V;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (tab[mid].item_base <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// Binning blocks of a layout (host): every view's Gaussians are cut into
// chunks of about BIN_CHUNK (fewer and larger where the tile counters would
// exceed `budget` beyond one per tile) and its tiles into bands of at most
// BIN_HIST_MAX tiles (whole rows where a row fits). view[V] is the sentinel;
// req[r].n gives each request's size.
inline void plan_binning(ViewTab *view, int32_t V, const ReqTab *req, int64_t total_tiles,
                         int32_t tile, RenderShape &s, int64_t budget = BIN_SLOT_BUDGET) {
  int64_t items = 0, slots = 0;
  int32_t area = 0;
  const int64_t by_slots = total_tiles > 0 ? budget / total_tiles : 1;
  for (int32_t v = 0; v < V; ++v) {
    ViewTab &t = view[v];
    const int64_t n = req[t.req].n;
    const int64_t tx = t.tiles_x, ty = (t.H + tile - 1) / tile;
    int64_t chunks = (n + BIN_CHUNK - 1) / BIN_CHUNK;
    if (chunks > by_slots) chunks = by_slots;
    if (chunks < 1) chunks = 1;
    if (n == 0) chunks = 0;
    int64_t bw = tx, bh = ty;
    if (tx * ty > BIN_HIST_MAX) {
      if (tx <= BIN_HIST_MAX) bh = BIN_HIST_MAX / tx;
      else { bw = BIN_HIST_MAX; bh = 1; }
    }
    const int64_t bands = ((tx + bw - 1) / bw) * ((ty + bh - 1) / bh);
    t.item_base = items;
    t.hist_base = slots;
    t.chunks = (int32_t)chunks;
    t.band_w = (int32_t)bw;
    t.band_h = (int32_t)bh;
    t.bands_x = (int32_t)((tx + bw - 1) / bw);
    items += chunks * bands;
    slots += chunks * bands * bw * bh;
    if (chunks > 0 && bw * bh > area) area = (int32_t)(bw * bh);
  }
  view[V].item_base = items;
  view[V].hist_base = slots;
  view[V].chunks = 0;
  s.n_items = items;
  s.hist_slots = slots;
  s.hist_area = area;
}

// Tile counters any layout with this many tiles can need: bands cover less
// than twice a view's tiles, and chunks x tiles stays within the budget.
inline int64_t hist_slot_bound(int64_t tiles, int64_t budget = BIN_SLOT_BUDGET) {
  return 2 * (tiles > budget ? tiles : budget);
}

// Largest v with tab[v].tile_base <= t.
__device__ __forceinline__ int find_view(const ViewTab *tab, int V, int64_t t) {
  int lo = 0, hi = V;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (tab[mid].tile_base <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// IEEE-exact binary32 helpers: one correctly rounded operation each, never
// contracted into an FMA, so that the binning matches its written definition.
__device__ __forceinline__ float mulr(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float addr(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float subr(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float divr(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sqrtr(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ float dot3r(float a0, float a1, float a2, float b0, float b1, float b2) {
  return addr(addr(mulr(a0, b0), mulr(a1, b1)), mulr(a2, b2));
}

// 1 / x by the hardware's approximate reciprocal (about 1 ulp). Used only where
// the result feeds the image or the gradients through tolerances far above
// that error (never in the binning): the transmittance recovered in the
// backward as T' / (1 - sigma) (1 - sigma >= 0.01), the per-pixel radiosity
// sigmoid, and the backward preprocess's conic and perspective factors.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 2^x by the hardware's approximate base-2 exponential (ex2.approx).
__device__ __forceinline__ float exp2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Per-pair evaluation shared by the forward and backward rasterisers, written
// with explicit rounding so both kernels take bit-identical decisions.
struct PairEval {
  float dx, dy, G, aG, sigma;
};

// Half-extents of the q <= q_max ellipse of a 2D covariance, sqrt(q_max
// Sigma_xx) and sqrt(q_max Sigma_yy), widened by 1e-3 relative + 1e-3 px and
// rounded up to binary16, packed into the record's fourth float (x in the low
// half). The rasterisers cull with this box; rounding up keeps it conservative.
__device__ __forceinline__ float box_halfwidths(const float cov[3], float q_max) {
  // approximate square roots (a few ulp): far inside the 1e-3 widening
  float ex, ey;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(ex) : "f"(q_max * cov[0]));
  asm("sqrt.approx.f32 %0, %1;" : "=f"(ey) : "f"(q_max * cov[2]));
  ex = ex * 1.001f + 1e-3f;
  ey = ey * 1.001f + 1e-3f;
  const uint32_t hx = __half_as_ushort(__float2half_ru(ex));
  const uint32_t hy = __half_as_ushort(__float2half_ru(ey));
  return __uint_as_float(hx | (hy << 16));
}

__device__ __forceinline__ float2 unpack_halfwidths(float w) {
  const uint32_t b = __float_as_uint(w);
  return make_float2(__half2float(__ushort_as_half((unsigned short)(b & 0xffffu))),
                     __half2float(__ushort_as_half((unsigned short)(b >> 16))));
}

// q = d^T K d for the conic K = [[a, b], [b, c]], evaluated in the records'
// scaled units as q' = dx (a' dx + 2b' dy) + c' dy^2 from the record's
// (a', 2b', c') = CONIC_SCALE (a, 2b, c); q <= q_max is q' >= q_lim (both
// sides negative), and G = exp(-q / 2) = 2^q'.
__device__ __forceinline__ bool eval_pair(float u, float v, float ca, float cb2, float cc,
                                          float alpha, float px, float py,
                                          const RasterParams &P, PairEval &e) {
  e.dx = __fsub_rn(u, px);
  e.dy = __fsub_rn(v, py);
  const float t = __fmaf_rn(cb2, e.dy, __fmul_rn(ca, e.dx));
  const float q = __fmaf_rn(__fmul_rn(cc, e.dy), e.dy, __fmul_rn(e.dx, t));
  if (q < P.q_lim || q > 0.f) return false;
  e.G = exp2_approx(q);
  e.aG = __fmul_rn(alpha, e.G);
  e.sigma = fminf(P.alpha_max, e.aG);
  return e.sigma >= P.alpha_min;
}

}  // namespace ddgs

// Workspace (device memory owned by the library).
struct ddgs_workspace {
  int device = -1;
  int64_t rec_cap = 0, pair_cap = 0, tile_cap = 0, blk_cap = 0, hist_cap = 0, list_cap = 0;
  // per (view, Gaussian) records
  float4 *rec = nullptr;         // [records][2]: (u, v, a', 2b'), (c', alpha, colour, packed
                                 // box half-extents), (a', b', c') = CONIC_SCALE x conic:
                                 // one 32-byte sector per gather
  uint2 *rect = nullptr;         // (tx0 | ty0 << 16, tx1 | ty1 << 16)
  uint32_t *tiles_touched = nullptr;
  float4 *grad2d = nullptr;      // [records][2]: (u, v, ca, cb), (cc, alpha, colour, 0);
                                 // with per-pixel directions the colour slot holds dL/dz
  bool grad_zero = false;        // grad2d (and grad_h) hold zeros over their whole capacity:
                                 // the backward preprocess clears what it consumed
  // per-pixel directions only (allocated by the first such render)
  float4 *rec2 = nullptr;        // (a, h_0, h_1, h_2): colour logit z = a + Y(ray) . h
  float4 *grad_h = nullptr;      // (dL/dh_0, dL/dh_1, dL/dh_2, 0)
  int64_t pix_cap = 0;
  bool last_per_pixel = false;   // mode of the last forward render
  // scan
  uint32_t *blk_total = nullptr;
  // pairs: (depth bits << 32 | Gaussian) placed by tile, then each tile's
  // Gaussians in depth order
  uint64_t *keys[2] = {nullptr, nullptr};  // [pairs]; keys[1] only for merging long lists
  uint32_t *vals = nullptr;      // [pairs] the tile lists the rasterisers read
  uint32_t *hist = nullptr;      // [hist_cap] per (binning block, tile) counts, then offsets
  uint64_t *part = nullptr;      // [2 x tile blocks + 2] partial sums of the tile counts
  uint64_t *lists = nullptr;     // [list_cap] tile lists to sort, by length class
  uint32_t *list_count = nullptr;  // [LIST_CLASSES]
  uint2 *ranges = nullptr;       // [tiles]
  uint32_t *order = nullptr;     // [tiles] work order of the persistent rasterisers
  uint32_t *queue = nullptr;     // work-queue heads of the forward / backward rasterisers
  unsigned long long *req_time = nullptr;  // [1 + 2 R]: batch start, per-request fwd / bwd ends
  int batch_depth = 256;         // list entries staged per round in the rasterisers
  // scalars
  uint64_t *d_pairs = nullptr;   // device pair count M
  uint64_t *h_pairs = nullptr;   // pinned host mirror
  int32_t *d_status = nullptr;
  // request / view tables: device copies and a pinned host staging area
  ddgs::ReqTab *d_req = nullptr;
  ddgs::ViewTab *d_view = nullptr;
  unsigned char *h_tab = nullptr;
  int64_t req_cap = 0, view_cap = 0;
  // the last render
  ddgs::RenderShape shape{};
  bool have_render = false;
  uint64_t pair_bound = 0;       // grid bound used for the pair kernels
  int64_t last_hash = 0;         // identifies the batch layout of the last render
  // initialisation (rads.cu): crossing keys and per-chunk scratch
  uint64_t *rads_keys = nullptr;
  int64_t rads_key_cap = 0;
  unsigned char *rads_buf = nullptr;
  int64_t rads_buf_cap = 0;
};

namespace ddgs {

// Kernel ids of the launch counter and profiler (api.cu).
enum KernelId : int {
  KID_PREPROCESS_FWD = 0, KID_SCAN_BLOCKS, KID_BIN_COUNT, KID_BIN_OFFSETS, KID_BIN_SCATTER,
  KID_BIN_SORT, KID_BIN_MERGE, KID_RASTER_FWD, KID_L1_LOSS, KID_RASTER_BWD,
  KID_PREPROCESS_BWD, KID_DEBUG, KID_TILE_ORDER, KID_RADS_MINMAX, KID_RADS_COUNT, KID_RADS_SCAN,
  KID_RADS_EMIT, KID_RADS_SELECT, KID_RADS_DRAW, KID_RADS_KNN, KID_COUNT
};

// Records a failed CUDA call for ddgs_last_cuda_error and maps it to a status.
ddgs_status cuda_status(cudaError_t e, const char *what);

// Brackets one kernel launch: counts it and, when profiling, records events.
struct LaunchScope {
  int id;
  cudaStream_t st;
  cudaEvent_t ev0 = nullptr;
  LaunchScope(int kid, cudaStream_t s);
  ~LaunchScope();
};

// preprocess.cu
void launch_preprocess_fwd(const ddgs_gaussians &g, const ddgs_views &v, const ddgs_config &c,
                           const RenderShape &s, ddgs_workspace &ws, cudaStream_t st);
void launch_preprocess_bwd(const ddgs_gaussians &g, const ddgs_views &v, const ddgs_config &c,
                           const RenderShape &s, ddgs_workspace &ws, const ddgs_grads &out,
                           cudaStream_t st);

// bin.cu
void launch_scan_blocks(int64_t nblk, ddgs_workspace &ws, cudaStream_t st);
// Tile lists of the render: ranges[tile] and vals, from the records' tile
// rectangles and depths (ws.rect); pair_bound > 0 once pairs exist.
void launch_binning(const RenderShape &s, uint64_t pair_bound, ddgs_workspace &ws,
                    cudaStream_t st);
int64_t list_capacity(int64_t tiles, int64_t pairs);  // entries of ws.lists
int64_t part_capacity(int64_t tiles);                 // entries of ws.part
cudaError_t prepare_bin_kernels();  // once per device, before any capture

// raster.cu
// Per-pixel ray angles (Eq. 3 variant): the views' poses and detectors, and
// the backward pass's pose-gradient output (may be null). A null PixelRays
// selects the per-Gaussian colours of the records.
struct PixelRays {
  const float *world_to_cam = nullptr, *detector = nullptr;
  float *pose_grad = nullptr;
};
void launch_tile_order(const RenderShape &s, ddgs_workspace &ws, cudaStream_t st);
void launch_raster_fwd(const RenderShape &s, const RasterParams &p, ddgs_workspace &ws,
                       float *image, float *t_final, uint32_t *n_last, const PixelRays *pr,
                       cudaStream_t st);
void launch_raster_bwd(const RenderShape &s, const RasterParams &p, ddgs_workspace &ws,
                       const float *dL_dimage, const float *t_final, const uint32_t *n_last,
                       const PixelRays *pr, cudaStream_t st);

int device_sms();  // streaming multiprocessors of the current device (raster.cu)
cudaError_t prepare_raster_kernels();  // once per device, before any capture (raster.cu)

// api.cu
void launch_l1_loss(const float *image, const float *target, int per_view, int V, int64_t hw,
                    float *loss, float *grad, cudaStream_t st);

}  // namespace ddgs
