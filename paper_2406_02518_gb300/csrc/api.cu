// api.cu -- the C ABI: argument checks, workspace management and the order of
// the kernels of a render and of its backward pass.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ddgs_internal.cuh"

namespace {

thread_local char g_cuda_err[256] = "";

ddgs_status cuda_fail(cudaError_t e, const char *what) {
  std::snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? DDGS_ERR_OUT_OF_MEMORY : DDGS_ERR_CUDA;
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

}  // namespace

namespace ddgs {
ddgs_status cuda_status(cudaError_t e, const char *what) { return cuda_fail(e, what); }
}  // namespace ddgs

namespace {

// Reallocate p for `need` elements. The capacity field of p's group is zeroed
// first and set by the caller once every buffer of the group has grown, so a
// failed allocation leaves the group marked empty and the next call retries
// it instead of running on a null or short buffer.
template <class Tp>
ddgs_status grow(Tp *&p, int64_t &cap_field, int64_t need, size_t elem) {
  cap_field = 0;
  if (p) CK(cudaFree(p));
  p = nullptr;
  CK(cudaMalloc(reinterpret_cast<void **>(&p), (size_t)(need > 0 ? need : 1) * elem));
  return DDGS_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// The workspace's buffers live on the device that was current at its
// creation; kernels launched on another device must not receive them.
bool on_workspace_device(const ddgs_workspace *ws) {
  int dev = -1;
  return cudaGetDevice(&dev) == cudaSuccess && dev == ws->device;
}

ddgs_status check_inputs(const ddgs_gaussians *g, const ddgs_views *v, const ddgs_config *c) {
  if (!g || !v || !c) return DDGS_ERR_INVALID_ARG;
  if (g->n < 0 || g->n_iso < 0 || g->n_iso > g->n || g->n >= (int64_t(1) << 31))
    return DDGS_ERR_INVALID_ARG;
  if (v->n_views < 0 || v->height <= 0 || v->width <= 0 || v->height > 65535 * 8 ||
      v->width > 65535 * 8)
    return DDGS_ERR_INVALID_ARG;
  if (c->tile != 8 && c->tile != 16 && c->tile != 32) return DDGS_ERR_INVALID_ARG;
  if (!(c->q_max > 0) || !(c->alpha_max > 0) || !(c->t_min >= 0) || !(c->dilation >= 0))
    return DDGS_ERR_INVALID_ARG;
  if (g->feat_dim < 0 || g->feat_dim > DDGS_MAX_FEAT_DIM || g->sh_degree < 0 ||
      g->sh_degree > DDGS_MAX_SH_DEGREE)
    return DDGS_ERR_INVALID_ARG;
  if ((g->entangled != 0 && g->entangled != 1) || (g->per_pixel != 0 && g->per_pixel != 1) ||
      (g->per_pixel && g->sh_degree > 1))
    return DDGS_ERR_INVALID_ARG;
  if (g->n > 0) {
    if (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->b_iso || !g->B_dir)
      return DDGS_ERR_INVALID_ARG;
    if (!aligned16(g->quats)) return DDGS_ERR_INVALID_ARG;
    const bool vec = g->feat_dim == 0 || g->feat_dim == ddgs::K;  // 16-byte rows read as vectors
    if (g->n_iso > 0 && (!g->feat_iso || (vec && !aligned16(g->feat_iso)))) return DDGS_ERR_INVALID_ARG;
    if (g->n > g->n_iso && (!g->feat_dir || (vec && !aligned16(g->feat_dir)))) return DDGS_ERR_INVALID_ARG;
  }
  if (v->n_views > 0 && (!v->world_to_cam || !v->detector)) return DDGS_ERR_INVALID_ARG;
  return DDGS_OK;
}

// Host description of one render: the request and view tables plus totals.
struct Layout {
  int32_t R = 0, V = 0, tile = 16;
  std::vector<ddgs::ReqTab> req;   // R + 1 (sentinel)
  std::vector<ddgs::ViewTab> view; // V + 1 (sentinel)
  ddgs::RenderShape shape{};       // totals; device pointers filled by upload
  uint64_t hash = 0;
};

uint64_t mix(uint64_t h, uint64_t x) {
  h ^= x + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  return h;
}

// counts per request, views per request, sizes per view
ddgs_status make_layout(int32_t R, const int64_t *n, const int64_t *n_iso, const int32_t *nv,
                        const int32_t *H, const int32_t *W, int32_t heights_uniform,
                        int32_t tile, Layout &L) {
  if (R < 0 || (R > 0 && (!n || !n_iso || !nv))) return DDGS_ERR_INVALID_ARG;
  L.R = R;
  L.tile = tile;
  L.req.assign((size_t)R + 1, ddgs::ReqTab{});
  int64_t g = 0, iso = 0, dir = 0, blk = 0;
  int32_t v = 0;
  uint64_t h = mix(0, (uint64_t)R);
  h = mix(h, (uint64_t)tile);
  for (int32_t r = 0; r < R; ++r) {
    if (n[r] < 0 || n_iso[r] < 0 || n_iso[r] > n[r] || nv[r] < 0) return DDGS_ERR_INVALID_ARG;
    ddgs::ReqTab &q = L.req[r];
    q.g_off = g; q.n = n[r]; q.n_iso = n_iso[r]; q.iso_row = iso; q.dir_row = dir;
    q.blk_base = blk; q.v_off = v; q.n_views = nv[r];
    g += n[r]; iso += n_iso[r]; dir += n[r] - n_iso[r];
    blk += (n[r] + ddgs::PRE_THREADS - 1) / ddgs::PRE_THREADS;
    v += nv[r];
    h = mix(mix(mix(h, (uint64_t)n[r]), (uint64_t)n_iso[r]), (uint64_t)nv[r]);
  }
  if (g >= (int64_t(1) << 31)) return DDGS_ERR_INVALID_ARG;
  L.req[R].g_off = g; L.req[R].iso_row = iso; L.req[R].dir_row = dir; L.req[R].blk_base = blk;
  L.req[R].v_off = v;
  L.V = v;
  L.view.assign((size_t)v + 1, ddgs::ViewTab{});
  int64_t tiles = 0, recs = 0, pix = 0;
  for (int32_t r = 0, vi = 0; r < R; ++r)
    for (int32_t k = 0; k < nv[r]; ++k, ++vi) {
      const int32_t hv = heights_uniform ? H[0] : H[vi], wv = heights_uniform ? W[0] : W[vi];
      if (hv <= 0 || wv <= 0 || hv > 65535 * 8 || wv > 65535 * 8) return DDGS_ERR_INVALID_ARG;
      ddgs::ViewTab &t = L.view[vi];
      t.req = r; t.H = hv; t.W = wv; t.tiles_x = (wv + tile - 1) / tile;
      t.tile_base = tiles; t.rec_off = recs; t.img_off = pix;
      tiles += (int64_t)t.tiles_x * ((hv + tile - 1) / tile);
      recs += n[r];
      pix += (int64_t)hv * wv;
      h = mix(mix(h, (uint64_t)hv), (uint64_t)wv);
    }
  L.view[v].tile_base = tiles; L.view[v].rec_off = recs; L.view[v].img_off = pix;
  L.view[v].req = R;
  ddgs::RenderShape &s = L.shape;
  s.R = R; s.V = v; s.tile = tile;
  s.n_total = g; s.total_tiles = tiles; s.records = recs; s.pixels = pix; s.n_blocks = blk;
  ddgs::plan_binning(L.view.data(), v, L.req.data(), tiles, tile, s);
  L.hash = h ? h : 1;
  return DDGS_OK;
}

constexpr int64_t kTabReq0 = 4096, kTabView0 = 16384;  // initial table capacity

ddgs_status ensure_tables(ddgs_workspace *ws, int64_t R, int64_t V) {
  if (R + 1 <= ws->req_cap && V + 1 <= ws->view_cap && ws->h_tab) return DDGS_OK;
  const int64_t rc = std::max<int64_t>(R + 1, std::max<int64_t>(ws->req_cap, kTabReq0));
  const int64_t vc = std::max<int64_t>(V + 1, std::max<int64_t>(ws->view_cap, kTabView0));
  if (ws->h_tab) {
    CK(cudaDeviceSynchronize());  // the staging area may still feed a copy
    CK(cudaFreeHost(ws->h_tab));
    ws->h_tab = nullptr;
  }
  if (ws->d_req) CK(cudaFree(ws->d_req));
  if (ws->d_view) CK(cudaFree(ws->d_view));
  if (ws->req_time) CK(cudaFree(ws->req_time));
  ws->d_req = nullptr;
  ws->d_view = nullptr;
  ws->req_time = nullptr;
  ws->req_cap = ws->view_cap = 0;
  CK(cudaHostAlloc(&ws->h_tab, rc * sizeof(ddgs::ReqTab) + vc * sizeof(ddgs::ViewTab),
                   cudaHostAllocDefault));
  CK(cudaMalloc(&ws->d_req, rc * sizeof(ddgs::ReqTab)));
  CK(cudaMalloc(&ws->d_view, vc * sizeof(ddgs::ViewTab)));
  CK(cudaMalloc(&ws->req_time, (1 + 2 * rc) * sizeof(unsigned long long)));
  ws->req_cap = rc;
  ws->view_cap = vc;
  ws->last_hash = 0;
  return DDGS_OK;
}

// Copy the tables to the device when the layout differs from the last one;
// repeated renders of one layout (and CUDA-graph replays) reuse them.
ddgs_status upload_layout(ddgs_workspace *ws, Layout &L, bool no_sync, cudaStream_t st) {
  if (L.R + 1 > ws->req_cap || L.V + 1 > ws->view_cap) {
    if (no_sync) return DDGS_ERR_CAPACITY;
    ddgs_status e = ensure_tables(ws, L.R, L.V);
    if (e) return e;
  }
  if (ws->last_hash != L.hash) {
    // the previous upload must have left the staging area before it is reused
    if (ws->last_hash != 0) CK(cudaStreamSynchronize(st));
    ddgs::ReqTab *hr = reinterpret_cast<ddgs::ReqTab *>(ws->h_tab);
    ddgs::ViewTab *hv = reinterpret_cast<ddgs::ViewTab *>(ws->h_tab + ws->req_cap * sizeof(ddgs::ReqTab));
    std::memcpy(hr, L.req.data(), L.req.size() * sizeof(ddgs::ReqTab));
    std::memcpy(hv, L.view.data(), L.view.size() * sizeof(ddgs::ViewTab));
    CK(cudaMemcpyAsync(ws->d_req, hr, L.req.size() * sizeof(ddgs::ReqTab), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ws->d_view, hv, L.view.size() * sizeof(ddgs::ViewTab), cudaMemcpyHostToDevice, st));
    ws->last_hash = L.hash;
  }
  L.shape.req = ws->d_req;
  L.shape.view = ws->d_view;
  return DDGS_OK;
}

// Sort queues of the binning: sized by the tile and pair capacities.
ddgs_status ensure_lists(ddgs_workspace *ws) {
  const int64_t need = ddgs::list_capacity(ws->tile_cap, ws->pair_cap);
  if (need <= ws->list_cap && ws->lists) return DDGS_OK;
  const int64_t cap = need + need / 4;
  ddgs_status st = grow(ws->lists, ws->list_cap, cap, sizeof(uint64_t));
  if (st) return st;
  ws->list_cap = cap;
  return DDGS_OK;
}

ddgs_status ensure_records(ddgs_workspace *ws, const ddgs::RenderShape &s) {
  const int64_t blk = s.n_blocks;
  if (s.records > ws->rec_cap || !ws->rec) {
    int64_t cap = s.records + s.records / 4 + 1024;
    ddgs_status st;
    if ((st = grow(ws->rec, ws->rec_cap, 2 * cap, sizeof(float4)))) return st;
    if ((st = grow(ws->rect, ws->rec_cap, cap, sizeof(uint4)))) return st;
    ws->grad_zero = false;
    if ((st = grow(ws->grad2d, ws->rec_cap, 2 * cap, sizeof(float4)))) return st;
    ws->rec_cap = cap;
  }
  if (ws->rec2 && ws->pix_cap < ws->rec_cap) {  // per-pixel storage follows the records
    ddgs_status st;
    ws->grad_zero = false;
    if ((st = grow(ws->rec2, ws->pix_cap, ws->rec_cap, sizeof(float4)))) return st;
    if ((st = grow(ws->grad_h, ws->pix_cap, ws->rec_cap, sizeof(float4)))) return st;
    ws->pix_cap = ws->rec_cap;
  }
  if (blk > ws->blk_cap || !ws->blk_total) {
    int64_t cap = blk + blk / 4 + 64;
    ddgs_status st;
    if ((st = grow(ws->blk_total, ws->blk_cap, cap, sizeof(uint32_t)))) return st;
    ws->blk_cap = cap;
  }
  if (s.total_tiles > ws->tile_cap || !ws->ranges) {
    int64_t cap = s.total_tiles + s.total_tiles / 4 + 64;
    ddgs_status st;
    if ((st = grow(ws->ranges, ws->tile_cap, cap, sizeof(uint2)))) return st;
    if ((st = grow(ws->order, ws->tile_cap, cap, sizeof(uint32_t)))) return st;
    int64_t pc = 0;  // the part sums follow the tiles
    if ((st = grow(ws->part, pc, ddgs::part_capacity(cap), sizeof(uint64_t)))) return st;
    ws->tile_cap = cap;
  }
  if (s.hist_slots > ws->hist_cap || !ws->hist) {
    int64_t cap = std::max<int64_t>(s.hist_slots + s.hist_slots / 4, 1024);
    ddgs_status st;
    if ((st = grow(ws->hist, ws->hist_cap, cap, sizeof(uint32_t)))) return st;
    ws->hist_cap = cap;
  }
  return ensure_lists(ws);
}

ddgs_status ensure_pairs(ddgs_workspace *ws, int64_t pairs) {
  if (pairs > ddgs::BIN_MAX_PAIRS) return DDGS_ERR_CAPACITY;
  if (pairs <= ws->pair_cap && ws->keys[0]) return DDGS_OK;
  const int64_t cap = std::min<int64_t>(pairs + pairs / 4 + 4096, ddgs::BIN_MAX_PAIRS);
  ddgs_status st;
  for (int b = 0; b < 2; ++b)
    if ((st = grow(ws->keys[b], ws->pair_cap, cap, sizeof(uint64_t)))) return st;
  if ((st = grow(ws->vals, ws->pair_cap, cap, sizeof(uint32_t)))) return st;
  ws->pair_cap = cap;
  return ensure_lists(ws);
}

// ---- launch counter and event profiler ----
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_prof_on{0};
std::mutex g_prof_mu;
struct ProfRec {
  int id;
  cudaEvent_t a, b;
};
std::vector<ProfRec> g_pending;
std::vector<cudaEvent_t> g_pool;
const char *const KERNEL_NAMES[ddgs::KID_COUNT] = {
    "preprocess_fwd", "scan_blocks", "bin_count", "bin_offsets", "bin_scatter",
    "bin_sort", "bin_merge", "raster_fwd", "l1_loss", "raster_bwd",
    "preprocess_bwd", "debug_copy", "tile_order", "rads_minmax", "rads_count", "rads_scan",
    "rads_emit", "rads_select", "rads_draw", "rads_knn"};

cudaEvent_t pool_event() {  // caller holds g_prof_mu
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return true;
  return cs != cudaStreamCaptureStatusNone;
}

}  // namespace

ddgs::LaunchScope::LaunchScope(int kid, cudaStream_t s) : id(kid), st(s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_prof_on.load(std::memory_order_relaxed) || capturing(s)) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ev0 = pool_event();
  if (ev0 && cudaEventRecord(ev0, s) != cudaSuccess) {
    g_pool.push_back(ev0);
    ev0 = nullptr;
  }
}

ddgs::LaunchScope::~LaunchScope() {
  if (!ev0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEvent_t e1 = pool_event();
  if (e1 && cudaEventRecord(e1, st) == cudaSuccess) {
    g_pending.push_back({id, ev0, e1});
  } else {
    g_pool.push_back(ev0);
    if (e1) g_pool.push_back(e1);
  }
}

extern "C" {

int64_t ddgs_kernel_launches(void) { return g_launches.load(); }

ddgs_status ddgs_profiler_enable(int32_t on) {
  g_prof_on.store(on ? 1 : 0);
  return DDGS_OK;
}

ddgs_status ddgs_profiler_collect(int32_t max_kernels, double *total_ms, int64_t *launches,
                                  int32_t *n_kernels) {
  if (max_kernels < 0 || (max_kernels > 0 && (!total_ms || !launches))) return DDGS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (int k = 0; k < max_kernels; ++k) {
    total_ms[k] = 0.0;
    launches[k] = 0;
  }
  ddgs_status st = DDGS_OK;
  for (const ProfRec &r : g_pending) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "profiler event");
    } else if (r.id < max_kernels) {
      total_ms[r.id] += ms;
      launches[r.id] += 1;
    }
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_pending.clear();
  if (n_kernels) *n_kernels = ddgs::KID_COUNT;
  return st;
}

const char *ddgs_profiler_kernel_name(int32_t id) {
  return (id >= 0 && id < ddgs::KID_COUNT) ? KERNEL_NAMES[id] : "";
}

const char *ddgs_status_string(ddgs_status s) {
  switch (s) {
    case DDGS_OK: return "ok";
    case DDGS_ERR_INVALID_ARG: return "invalid argument";
    case DDGS_ERR_CAPACITY: return "pair capacity exceeded";
    case DDGS_ERR_NONFINITE: return "non-finite value";
    case DDGS_ERR_TIMEOUT: return "device wait timed out";
    case DDGS_ERR_CUDA: return "CUDA error";
    case DDGS_ERR_UNSUPPORTED: return "unsupported device";
    case DDGS_ERR_OUT_OF_MEMORY: return "out of device memory";
  }
  return "unknown status";
}

const char *ddgs_last_cuda_error(void) { return g_cuda_err; }

int64_t ddgs_parameter_count(int64_t n, int32_t k, int32_t L) {
  if (n < 0 || k < 0 || L < 0) return -1;
  const int64_t kl = (int64_t)L * (L + 2);
  return n * (3 + 4 + 3 + 1 + (int64_t)k) + k + kl * k;
}

int32_t ddgs_device_supported(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return 0;
  return (p.major == 10 && p.minor == 3) ? 1 : 0;
}

ddgs_status ddgs_workspace_create(ddgs_workspace **out) {
  if (!out) return DDGS_ERR_INVALID_ARG;
  *out = nullptr;
  ddgs_workspace *ws = new (std::nothrow) ddgs_workspace();
  if (!ws) return DDGS_ERR_OUT_OF_MEMORY;
  cudaError_t e;
  if ((e = cudaGetDevice(&ws->device)) != cudaSuccess ||
      (e = cudaMalloc(&ws->d_pairs, sizeof(uint64_t))) != cudaSuccess ||
      (e = cudaMalloc(&ws->d_status, sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMalloc(&ws->queue, 2 * sizeof(uint32_t))) != cudaSuccess ||
      (e = cudaMalloc(&ws->list_count, ddgs::LIST_CLASSES * sizeof(uint32_t))) != cudaSuccess ||
      (e = cudaHostAlloc(&ws->h_pairs, 2 * sizeof(uint64_t), cudaHostAllocDefault)) != cudaSuccess ||
      (e = cudaMemset(ws->d_status, 0, sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMemset(ws->d_pairs, 0, sizeof(uint64_t))) != cudaSuccess) {
    ddgs_status st = cuda_fail(e, "workspace create");
    ddgs_workspace_destroy(ws);
    return st;
  }
  ws->h_pairs[0] = ws->h_pairs[1] = 0;
  if (ensure_tables(ws, 0, 0) != DDGS_OK) {
    ddgs_workspace_destroy(ws);
    return DDGS_ERR_OUT_OF_MEMORY;
  }
  if ((e = ddgs::prepare_bin_kernels()) != cudaSuccess ||
      (e = ddgs::prepare_raster_kernels()) != cudaSuccess) {
    ddgs_status st = cuda_fail(e, "binning kernel set-up");
    ddgs_workspace_destroy(ws);
    return st;
  }
  *out = ws;
  return DDGS_OK;
}

ddgs_status ddgs_workspace_destroy(ddgs_workspace *ws) {
  if (!ws) return DDGS_OK;
  void *dev[] = {ws->rec, ws->rect, ws->tiles_touched, ws->grad2d, ws->blk_total,
                 ws->keys[0], ws->keys[1], ws->vals, ws->hist, ws->part, ws->lists,
                 ws->list_count, ws->ranges, ws->d_pairs, ws->d_status, ws->d_req, ws->d_view,
                 ws->order, ws->queue, ws->req_time, ws->rec2, ws->grad_h,
                 ws->rads_keys, ws->rads_buf};
  for (void *p : dev)
    if (p) cudaFree(p);
  if (ws->h_pairs) cudaFreeHost(ws->h_pairs);
  if (ws->h_tab) cudaFreeHost(ws->h_tab);
  delete ws;
  return DDGS_OK;
}

ddgs_status ddgs_workspace_reserve(ddgs_workspace *ws, int64_t records, int64_t pairs,
                                   int64_t tiles) {
  if (!ws || records < 0 || pairs < 0 || tiles < 0 || !on_workspace_device(ws))
    return DDGS_ERR_INVALID_ARG;
  CK(cudaDeviceSynchronize());
  ddgs::RenderShape s{};
  s.records = records;
  // any split of the records into requests and views needs at most this many
  // preprocess blocks (one partial block per request, up to 4096 requests)
  s.n_blocks = records / ddgs::PRE_THREADS + 4096;
  s.total_tiles = tiles;
  s.hist_slots = ddgs::hist_slot_bound(tiles);
  ddgs_status st = ensure_records(ws, s);
  if (st) return st;
  st = ensure_pairs(ws, pairs);
  if (st) return st;
  st = ensure_tables(ws, 0, 0);
  if (st) return st;
  CK(cudaDeviceSynchronize());
  return DDGS_OK;
}

}  // extern "C"

namespace {

// The kernels read the parameter arrays through ddgs_gaussians / ddgs_views
// (pointers only); sizes come from the layout.
ddgs_status render_common(const ddgs_gaussians &g, const ddgs_views &v, const ddgs_config *c,
                          Layout &L, ddgs_workspace *ws, float *image, float *t_final,
                          uint32_t *n_last, cudaStream_t s_) {
  if (!on_workspace_device(ws)) return DDGS_ERR_INVALID_ARG;
  ddgs_status st;
  ddgs::RenderShape &s = L.shape;
  if (c->no_sync) {
    if (s.records > ws->rec_cap || s.n_blocks > ws->blk_cap || s.total_tiles > ws->tile_cap ||
        s.hist_slots > ws->hist_cap || !ws->keys[0] ||
        ddgs::list_capacity(s.total_tiles, ws->pair_cap) > ws->list_cap)
      return DDGS_ERR_CAPACITY;
    if (g.per_pixel && (!ws->rec2 || ws->pix_cap < s.records)) return DDGS_ERR_CAPACITY;
  } else {
    if ((st = ensure_records(ws, s))) return st;
    if (g.per_pixel && !ws->rec2) {
      ws->grad_zero = false;
      if ((st = grow(ws->rec2, ws->pix_cap, ws->rec_cap, sizeof(float4)))) return st;
      if ((st = grow(ws->grad_h, ws->pix_cap, ws->rec_cap, sizeof(float4)))) return st;
      ws->pix_cap = ws->rec_cap;
    }
  }
  if ((st = upload_layout(ws, L, c->no_sync != 0, s_))) return st;
  ws->have_render = false;
  ws->batch_depth = (c->batch_depth == 32 || c->batch_depth == 128 || c->batch_depth == 512)
                        ? c->batch_depth : 256;
  // timing slots: batch start (min) and per-request ends (max)
  CK(cudaMemsetAsync(ws->req_time, 0xff, sizeof(unsigned long long), s_));
  CK(cudaMemsetAsync(ws->req_time + 1, 0, 2 * (size_t)s.R * sizeof(unsigned long long), s_));
  uint64_t bound = 0;
  bool nonfinite = false;
  if (s.records > 0) {
    ddgs::launch_preprocess_fwd(g, v, *c, s, *ws, s_);
    CK(cudaGetLastError());
    ddgs::launch_scan_blocks(s.n_blocks, *ws, s_);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ws->h_pairs, ws->d_pairs, sizeof(uint64_t), cudaMemcpyDeviceToHost, s_));
    if (!c->no_sync) {
      // the status word rides along with the pair count: a non-finite input
      // is reported by this call (and cleared), other bits stay latched
      int32_t *h_st = reinterpret_cast<int32_t *>(ws->h_pairs + 1);
      CK(cudaMemcpyAsync(h_st, ws->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s_));
      CK(cudaStreamSynchronize(s_));
      if (h_st[0] & ddgs::ST_NONFINITE) {
        nonfinite = true;
        h_st[1] = h_st[0] & ~ddgs::ST_NONFINITE;
        CK(cudaMemcpyAsync(ws->d_status, h_st + 1, sizeof(int32_t), cudaMemcpyHostToDevice, s_));
      }
      bound = *ws->h_pairs;
      if (bound > (uint64_t)ddgs::BIN_MAX_PAIRS) return DDGS_ERR_CAPACITY;
      if ((st = ensure_pairs(ws, (int64_t)bound))) return st;
    } else {
      bound = (uint64_t)ws->pair_cap;
    }
  } else {
    *ws->h_pairs = 0;
    CK(cudaMemsetAsync(ws->d_pairs, 0, sizeof(uint64_t), s_));
  }
  if (s.total_tiles > 0) {
    ddgs::launch_binning(s, bound, *ws, s_);
    CK(cudaGetLastError());
    ddgs::launch_tile_order(s, *ws, s_);
    CK(cudaGetLastError());
    ddgs::RasterParams P{c->alpha_min, c->alpha_max, c->t_min, c->q_max,
                          c->q_max * ddgs::CONIC_SCALE};
    ddgs::PixelRays pr;
    pr.world_to_cam = v.world_to_cam;
    pr.detector = v.detector;
    ddgs::launch_raster_fwd(s, P, *ws, image, t_final, n_last, g.per_pixel ? &pr : nullptr, s_);
    CK(cudaGetLastError());
  }
  ws->last_per_pixel = g.per_pixel != 0;
  ws->shape = s;
  ws->pair_bound = bound;
  ws->have_render = true;
  return nonfinite ? DDGS_ERR_NONFINITE : DDGS_OK;
}

ddgs_status backward_common(const ddgs_gaussians &g, const ddgs_views &v, const ddgs_config *c,
                            Layout &L, ddgs_workspace *ws, const float *dL_dimage,
                            const float *t_final, const uint32_t *n_last, const ddgs_grads *out,
                            cudaStream_t s_) {
  if (!ws || !out || !ws->have_render || L.hash != ws->last_hash ||
      (g.per_pixel != 0) != ws->last_per_pixel || !on_workspace_device(ws))
    return DDGS_ERR_INVALID_ARG;
  ddgs::RenderShape &s = L.shape;
  s.req = ws->d_req;
  s.view = ws->d_view;
  if (s.total_tiles > 0 && (!dL_dimage || !t_final || !n_last)) return DDGS_ERR_INVALID_ARG;
  if ((out->quats && !aligned16(out->quats)) || (out->feat_iso && !aligned16(out->feat_iso)) ||
      (out->feat_dir && !aligned16(out->feat_dir)))
    return DDGS_ERR_INVALID_ARG;
  const int kf = g.feat_dim ? g.feat_dim : ddgs::K, lsh = g.sh_degree ? g.sh_degree : 1;
  if (out->b_iso) CK(cudaMemsetAsync(out->b_iso, 0, (size_t)s.R * kf * sizeof(float), s_));
  if (out->B_dir)
    CK(cudaMemsetAsync(out->B_dir, 0, (size_t)s.R * lsh * (lsh + 2) * kf * sizeof(float), s_));
  if (out->world_to_cam)
    CK(cudaMemsetAsync(out->world_to_cam, 0, (size_t)s.V * 12 * sizeof(float), s_));
  if (s.n_total == 0) return DDGS_OK;  // parameter gradients empty, pose/basis zero
  // The rasteriser accumulates 2D gradients into zeros, and the backward
  // preprocess clears every record it consumes, so the buffers are cleared
  // here only after an allocation or a failed call.
  if (!ws->grad_zero) {
    if (ws->rec_cap > 0) CK(cudaMemsetAsync(ws->grad2d, 0, (size_t)ws->rec_cap * 2 * sizeof(float4), s_));
    if (ws->grad_h && ws->pix_cap > 0)
      CK(cudaMemsetAsync(ws->grad_h, 0, (size_t)ws->pix_cap * sizeof(float4), s_));
  }
  ws->grad_zero = false;  // until both kernels are queued
  ddgs::RasterParams P{c->alpha_min, c->alpha_max, c->t_min, c->q_max,
                          c->q_max * ddgs::CONIC_SCALE};
  if (s.records > 0 && s.total_tiles > 0 && ws->pair_bound > 0) {
    ddgs::PixelRays pr;
    pr.world_to_cam = v.world_to_cam;
    pr.detector = v.detector;
    pr.pose_grad = out->world_to_cam;
    ddgs::launch_raster_bwd(s, P, *ws, dL_dimage, t_final, n_last, g.per_pixel ? &pr : nullptr, s_);
    CK(cudaGetLastError());
  }
  ddgs::launch_preprocess_bwd(g, v, *c, s, *ws, *out, s_);
  CK(cudaGetLastError());
  ws->grad_zero = true;
  return DDGS_OK;
}

ddgs_status single_layout(const ddgs_gaussians *g, const ddgs_views *v, const ddgs_config *c,
                          Layout &L) {
  ddgs_status st = check_inputs(g, v, c);
  if (st) return st;
  const int64_t n = g->n, ni = g->n_iso;
  const int32_t nv = v->n_views;
  return make_layout(1, &n, &ni, &nv, &v->height, &v->width, 1, c->tile, L);
}

ddgs_status check_batch(const ddgs_batch *b, const ddgs_config *c) {
  if (!b || !c || b->n_requests < 0) return DDGS_ERR_INVALID_ARG;
  if (b->feat_dim < 0 || b->feat_dim > DDGS_MAX_FEAT_DIM || b->sh_degree < 0 ||
      b->sh_degree > DDGS_MAX_SH_DEGREE)
    return DDGS_ERR_INVALID_ARG;
  if ((b->entangled != 0 && b->entangled != 1) || (b->per_pixel != 0 && b->per_pixel != 1) ||
      (b->per_pixel && b->sh_degree > 1))
    return DDGS_ERR_INVALID_ARG;
  const bool vec = b->feat_dim == 0 || b->feat_dim == ddgs::K;
  if (c->tile != 8 && c->tile != 16 && c->tile != 32) return DDGS_ERR_INVALID_ARG;
  if (!(c->q_max > 0) || !(c->alpha_max > 0) || !(c->t_min >= 0) || !(c->dilation >= 0))
    return DDGS_ERR_INVALID_ARG;
  if (b->n_requests > 0 && (!b->gaussian_counts || !b->iso_counts || !b->view_counts))
    return DDGS_ERR_INVALID_ARG;
  int64_t n = 0, ni = 0, nv = 0;
  for (int32_t r = 0; r < b->n_requests; ++r) {
    // per-request bounds first, so that the sums below cannot overflow
    const int64_t nr = b->gaussian_counts[r], nir = b->iso_counts[r];
    if (nr < 0 || nr >= (int64_t(1) << 31) || nir < 0 || nir > nr || b->view_counts[r] < 0)
      return DDGS_ERR_INVALID_ARG;
    n += b->gaussian_counts[r];
    ni += b->iso_counts[r];
    nv += b->view_counts[r];
  }
  if (nv > 0 && (!b->heights || !b->widths || !b->world_to_cam || !b->detector))
    return DDGS_ERR_INVALID_ARG;
  if (n > 0) {
    if (!b->means || !b->log_scales || !b->quats || !b->opacity_logits || !b->b_iso || !b->B_dir ||
        !aligned16(b->quats))
      return DDGS_ERR_INVALID_ARG;
    if (ni > 0 && (!b->feat_iso || (vec && !aligned16(b->feat_iso)))) return DDGS_ERR_INVALID_ARG;
    if (n > ni && (!b->feat_dir || (vec && !aligned16(b->feat_dir)))) return DDGS_ERR_INVALID_ARG;
  }
  return DDGS_OK;
}

void batch_structs(const ddgs_batch *b, ddgs_gaussians &g, ddgs_views &v) {
  g = ddgs_gaussians{};
  g.means = b->means; g.log_scales = b->log_scales; g.quats = b->quats;
  g.opacity_logits = b->opacity_logits; g.feat_iso = b->feat_iso; g.feat_dir = b->feat_dir;
  g.feat_dir_bf16 = b->feat_dir_bf16; g.b_iso = b->b_iso; g.B_dir = b->B_dir;
  g.feat_dim = b->feat_dim; g.sh_degree = b->sh_degree;
  g.entangled = b->entangled; g.per_pixel = b->per_pixel;
  v = ddgs_views{};
  v.world_to_cam = b->world_to_cam;
  v.detector = b->detector;
}

}  // namespace

extern "C" {

ddgs_status ddgs_render(const ddgs_gaussians *g, const ddgs_views *v, const ddgs_config *c,
                        ddgs_workspace *ws, float *image, float *t_final, uint32_t *n_last,
                        void *stream) {
  Layout L;
  ddgs_status st = single_layout(g, v, c, L);
  if (st) return st;
  if (!ws) return DDGS_ERR_INVALID_ARG;
  if (v->n_views > 0 && (!image || !t_final || !n_last)) return DDGS_ERR_INVALID_ARG;
  return render_common(*g, *v, c, L, ws, image, t_final, n_last, static_cast<cudaStream_t>(stream));
}

ddgs_status ddgs_render_backward(const ddgs_gaussians *g, const ddgs_views *v,
                                 const ddgs_config *c, ddgs_workspace *ws,
                                 const float *dL_dimage, const float *t_final,
                                 const uint32_t *n_last, const ddgs_grads *out, void *stream) {
  Layout L;
  ddgs_status st = single_layout(g, v, c, L);
  if (st) return st;
  return backward_common(*g, *v, c, L, ws, dL_dimage, t_final, n_last, out,
                         static_cast<cudaStream_t>(stream));
}

ddgs_status ddgs_render_batched(const ddgs_batch *b, const ddgs_config *c, ddgs_workspace *ws,
                                float *image, float *t_final, uint32_t *n_last, void *stream) {
  ddgs_status st = check_batch(b, c);
  if (st) return st;
  if (!ws) return DDGS_ERR_INVALID_ARG;
  Layout L;
  if ((st = make_layout(b->n_requests, b->gaussian_counts, b->iso_counts, b->view_counts,
                        b->heights, b->widths, 0, c->tile, L)))
    return st;
  if (L.shape.pixels > 0 && (!image || !t_final || !n_last)) return DDGS_ERR_INVALID_ARG;
  ddgs_gaussians g;
  ddgs_views v;
  batch_structs(b, g, v);
  return render_common(g, v, c, L, ws, image, t_final, n_last, static_cast<cudaStream_t>(stream));
}

ddgs_status ddgs_render_batched_backward(const ddgs_batch *b, const ddgs_config *c,
                                         ddgs_workspace *ws, const float *dL_dimage,
                                         const float *t_final, const uint32_t *n_last,
                                         const ddgs_grads *out, void *stream) {
  ddgs_status st = check_batch(b, c);
  if (st) return st;
  Layout L;
  if ((st = make_layout(b->n_requests, b->gaussian_counts, b->iso_counts, b->view_counts,
                        b->heights, b->widths, 0, c->tile, L)))
    return st;
  ddgs_gaussians g;
  ddgs_views v;
  batch_structs(b, g, v);
  return backward_common(g, v, c, L, ws, dL_dimage, t_final, n_last, out,
                         static_cast<cudaStream_t>(stream));
}

ddgs_status ddgs_request_times(const ddgs_workspace *ws, uint64_t *fwd_ns, uint64_t *bwd_ns,
                               void *stream) {
  if (!ws || !ws->have_render) return DDGS_ERR_INVALID_ARG;
  const int R = ws->shape.R;
  std::vector<unsigned long long> t((size_t)(1 + 2 * R));
  CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  CK(cudaMemcpy(t.data(), ws->req_time, t.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  const unsigned long long t0 = t[0];
  for (int r = 0; r < R; ++r) {
    if (fwd_ns) fwd_ns[r] = (t[1 + r] && t[1 + r] >= t0) ? t[1 + r] - t0 : 0;
    if (bwd_ns) bwd_ns[r] = (t[1 + R + r] && t[1 + R + r] >= t0) ? t[1 + R + r] - t0 : 0;
  }
  return DDGS_OK;
}

ddgs_status ddgs_workspace_pairs(const ddgs_workspace *ws, int64_t *pairs) {
  if (!ws || !pairs) return DDGS_ERR_INVALID_ARG;
  *pairs = (int64_t)*ws->h_pairs;
  return DDGS_OK;
}

}  // extern "C"

namespace {
__global__ void tiles_touched_kernel(const uint4 *info, int64_t n, uint32_t *out) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    out[j] = info[j].w;
}

// The sort key (global tile << 32 | depth bits) of every list entry, one
// thread per tile writing its list's keys.
__global__ void list_keys_kernel(ddgs::RenderShape s, const uint2 *ranges, const uint32_t *vals,
                                 const uint4 *info, uint64_t *keys) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < s.total_tiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint2 r = ranges[t];
    const ddgs::ViewTab vt = s.view[ddgs::find_view(s.view, s.V, t)];
    for (uint32_t j = r.x; j < r.y; ++j) keys[j] = ((uint64_t)t << 32) | info[vt.rec_off + vals[j]].z;
  }
}

__global__ void l1_loss_kernel(const float *image, const float *target, int per_view, int64_t hw,
                               float *loss, float *grad) {
  // one block row per view: blockIdx.y = view
  const int v = blockIdx.y;
  const float *img = image + (int64_t)v * hw;
  const float *tgt = target + (per_view ? (int64_t)v * hw : 0);
  float *gr = grad + (int64_t)v * hw;
  const float inv = 1.0f / (float)hw;
  float acc = 0.f;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < hw;
       j += (int64_t)gridDim.x * blockDim.x) {
    const float d = img[j] - tgt[j];
    acc += fabsf(d);
    gr[j] = d > 0.f ? inv : (d < 0.f ? -inv : 0.f);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ float s_w[32];
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w];
    atomicAdd(loss + v, t * inv);
  }
}
}  // namespace

namespace ddgs {
void launch_l1_loss(const float *image, const float *target, int per_view, int V, int64_t hw,
                    float *loss, float *grad, cudaStream_t st) {
  int64_t bx = (hw + 255) / 256;
  if (bx > 64) bx = 64;
  dim3 grid((unsigned)bx, (unsigned)V);
  LaunchScope ls(KID_L1_LOSS, st);
  l1_loss_kernel<<<grid, 256, 0, st>>>(image, target, per_view, hw, loss, grad);
}
}  // namespace ddgs

extern "C" {

ddgs_status ddgs_debug_binning(const ddgs_workspace *ws, uint32_t *tiles_touched, uint64_t *keys,
                               uint32_t *vals, uint32_t *ranges, void *stream) {
  if (!ws || !ws->have_render || !on_workspace_device(ws)) return DDGS_ERR_INVALID_ARG;
  cudaStream_t s_ = static_cast<cudaStream_t>(stream);
  const ddgs::RenderShape &s = ws->shape;
  if (tiles_touched && s.records > 0) {
    int64_t b = (s.records + 255) / 256;
    if (b > 4096) b = 4096;
    ddgs::LaunchScope ls(ddgs::KID_DEBUG, s_);
    tiles_touched_kernel<<<(unsigned)b, 256, 0, s_>>>(reinterpret_cast<const uint4 *>(ws->rect),
                                                      s.records, tiles_touched);
    CK(cudaGetLastError());
  }
  uint64_t m = *ws->h_pairs;
  if (m > (uint64_t)ws->pair_cap) m = (uint64_t)ws->pair_cap;  // after an overflow
  if (keys && m && s.total_tiles > 0) {
    int64_t b = (s.total_tiles + 255) / 256;
    if (b > 4096) b = 4096;
    ddgs::LaunchScope ls(ddgs::KID_DEBUG, s_);
    list_keys_kernel<<<(unsigned)b, 256, 0, s_>>>(s, ws->ranges, ws->vals,
                                                  reinterpret_cast<const uint4 *>(ws->rect), keys);
    CK(cudaGetLastError());
  }
  if (vals && m) CK(cudaMemcpyAsync(vals, ws->vals, m * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s_));
  if (ranges && s.total_tiles)
    CK(cudaMemcpyAsync(ranges, ws->ranges, (size_t)s.total_tiles * sizeof(uint2), cudaMemcpyDeviceToDevice, s_));
  return DDGS_OK;
}

ddgs_status ddgs_l1_loss(const float *image, const float *target, int32_t target_per_view,
                         int32_t n_views, int64_t hw, float *loss, float *dL_dimage, void *stream) {
  if (n_views < 0 || hw < 0) return DDGS_ERR_INVALID_ARG;
  if (n_views == 0 || hw == 0) return DDGS_OK;
  if (!image || !target || !loss || !dL_dimage || n_views > 65535) return DDGS_ERR_INVALID_ARG;
  cudaStream_t s_ = static_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(loss, 0, (size_t)n_views * sizeof(float), s_));
  ddgs::launch_l1_loss(image, target, target_per_view, n_views, hw, loss, dL_dimage, s_);
  CK(cudaGetLastError());
  return DDGS_OK;
}

ddgs_status ddgs_sync_status(ddgs_workspace *ws, void *stream) {
  if (!ws) return DDGS_ERR_INVALID_ARG;
  cudaStream_t s_ = static_cast<cudaStream_t>(stream);
  int32_t h = 0;
  CK(cudaStreamSynchronize(s_));
  CK(cudaMemcpy(&h, ws->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost));
  CK(cudaMemset(ws->d_status, 0, sizeof(int32_t)));
  if (h & ddgs::ST_CAPACITY) return DDGS_ERR_CAPACITY;
  if (h & ddgs::ST_NONFINITE) return DDGS_ERR_NONFINITE;
  return DDGS_OK;
}

}  // extern "C"
