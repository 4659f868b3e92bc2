// render_static.cu -- ddgs_render_static: the forward render with its scratch
// memory in a fixed, file-scope device array instead of a workspace.
//
// Who needs it: code that must not allocate device memory once it runs. For
// example an intra-operative registration loop whose memory budget is fixed
// at start-up, code that runs inside another framework's allocator callback,
// or a process whose device memory is entirely owned by a caching allocator
// that the library cannot see. For those callers every cudaMalloc is either
// forbidden or a source of stalls and fragmentation, so this entry point
// allocates nothing: the caller passes inputs and outputs, and all scratch
// (per-(view, Gaussian) records, tile lists, tile counters and ranges) lives in
// one static array that every GPU loading the library holds until exit.
//
// The array is shared by every call on a device and keeps the last call's
// contents; whatever must start at zero is cleared by each call. Calls whose
// work overlaps on the GPU (two streams, or two host threads) race on it.
#include <mutex>

#include "ddgs_internal.cuh"

namespace {

// Limits of one call (see include/ddgs.h).
constexpr int64_t kMaxRecords = int64_t(1) << 18;  // views x Gaussians
constexpr int64_t kMaxPairs = int64_t(1) << 20;    // (Gaussian, tile) pairs
constexpr int64_t kMaxTiles = int64_t(1) << 16;    // views x tiles per view
constexpr int64_t kMaxViews = 1024;                // views per call
constexpr int64_t kMaxBlocks = kMaxRecords / ddgs::PRE_THREADS + 1;
constexpr int64_t kSlotBudget = int64_t(1) << 18;  // tile counters of the binning blocks
constexpr int64_t kMaxSlots = 2 * (kMaxTiles > kSlotBudget ? kMaxTiles : kSlotBudget);
constexpr int64_t kMaxParts = 2 * ((kMaxTiles + 1023) / 1024) + 2;
constexpr int64_t kMaxListItems = ddgs::LIST_CLASSES * kMaxTiles + kMaxPairs / ddgs::BIN_LIST_LONG + 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
// Byte offsets of each buffer inside the scratch array.
constexpr size_t kOffRec0 = 0;
constexpr size_t kOffRec1 = align256(kOffRec0 + kMaxRecords * sizeof(float4));
constexpr size_t kOffInfo = align256(kOffRec1 + kMaxRecords * sizeof(float4));
static_assert(kOffRec1 == kOffRec0 + kMaxRecords * sizeof(float4),
              "the records are one interleaved array over both regions");
constexpr size_t kOffBlkTotal = align256(kOffInfo + kMaxRecords * sizeof(uint4));
constexpr size_t kOffKeys0 = align256(kOffBlkTotal + kMaxBlocks * sizeof(uint32_t));
constexpr size_t kOffKeys1 = align256(kOffKeys0 + kMaxPairs * sizeof(uint64_t));
constexpr size_t kOffVals = align256(kOffKeys1 + kMaxPairs * sizeof(uint64_t));
constexpr size_t kOffHist = align256(kOffVals + kMaxPairs * sizeof(uint32_t));
constexpr size_t kOffPart = align256(kOffHist + kMaxSlots * sizeof(uint32_t));
constexpr size_t kOffLists = align256(kOffPart + kMaxParts * sizeof(uint64_t));
constexpr size_t kOffListCount = align256(kOffLists + kMaxListItems * sizeof(uint64_t));
constexpr size_t kOffRanges = align256(kOffListCount + ddgs::LIST_CLASSES * sizeof(uint32_t));
constexpr size_t kOffPairs = align256(kOffRanges + kMaxTiles * sizeof(uint2));
constexpr size_t kOffStatus = align256(kOffPairs + sizeof(uint64_t));
constexpr size_t kOffOrder = align256(kOffStatus + sizeof(int32_t));
constexpr size_t kOffQueue = align256(kOffOrder + kMaxTiles * sizeof(uint32_t));
constexpr size_t kOffReq = align256(kOffQueue + 2 * sizeof(uint32_t));
constexpr size_t kOffView = align256(kOffReq + 2 * sizeof(ddgs::ReqTab));
constexpr size_t kScratchBytes = align256(kOffView + (kMaxViews + 1) * sizeof(ddgs::ViewTab));

// Host-side tables of one call (thread-local storage, not heap).
thread_local ddgs::ReqTab t_req[2];
thread_local ddgs::ViewTab t_view[kMaxViews + 1];

// The scratch itself (about 37 MiB per device).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, looked up once per device.
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_setup_mu;

// A failed CUDA call: its message goes where ddgs_last_cuda_error reads it.
#define CK_STATIC(call)                                             \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return ddgs::cuda_status(e_, #call);     \
  } while (0)

ddgs_status scratch_for_current_device(unsigned char **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DDGS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    CK_STATIC(cudaGetSymbolAddress(&p, g_scratch));
    if (!p) return DDGS_ERR_CUDA;
    g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_ptr[dev];
  return DDGS_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" ddgs_status ddgs_render_static(const ddgs_gaussians *g, const ddgs_views *v,
                                          const ddgs_config *c, float *image, float *t_final,
                                          uint32_t *n_last, void *stream) {
  // argument checks (as ddgs_render)
  if (!g || !v || !c) return DDGS_ERR_INVALID_ARG;
  if (g->feat_dim < 0 || g->feat_dim > DDGS_MAX_FEAT_DIM || g->sh_degree < 0 ||
      g->sh_degree > DDGS_MAX_SH_DEGREE)
    return DDGS_ERR_INVALID_ARG;
  // per-pixel ray angles need per-record storage the static scratch does not hold
  if ((g->entangled != 0 && g->entangled != 1) || g->per_pixel != 0) return DDGS_ERR_INVALID_ARG;
  if (g->n < 0 || g->n_iso < 0 || g->n_iso > g->n || v->n_views < 0 || v->height <= 0 ||
      v->width <= 0 || v->height > 65535 * 8 || v->width > 65535 * 8)
    return DDGS_ERR_INVALID_ARG;
  if (c->tile != 8 && c->tile != 16 && c->tile != 32) return DDGS_ERR_INVALID_ARG;
  if (!(c->q_max > 0) || !(c->alpha_max > 0) || !(c->t_min >= 0) || !(c->dilation >= 0))
    return DDGS_ERR_INVALID_ARG;
  if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->b_iso ||
                   !g->B_dir || !aligned16(g->quats) ||
                   (g->n_iso > 0 && !g->feat_iso) || (g->n > g->n_iso && !g->feat_dir) ||
                   ((g->feat_dim == 0 || g->feat_dim == 8) &&
                    ((g->n_iso > 0 && !aligned16(g->feat_iso)) ||
                     (g->n > g->n_iso && !aligned16(g->feat_dir))))))
    return DDGS_ERR_INVALID_ARG;
  if (v->n_views > 0 && (!v->world_to_cam || !v->detector || !image || !t_final || !n_last))
    return DDGS_ERR_INVALID_ARG;

  // one request, n_views equal views
  if (v->n_views > kMaxViews) return DDGS_ERR_CAPACITY;
  const int32_t tile = c->tile;
  const int32_t tx = (v->width + tile - 1) / tile, ty = (v->height + tile - 1) / tile;
  ddgs::RenderShape s{};
  s.R = 1;
  s.V = v->n_views;
  s.tile = tile;
  s.n_total = g->n;
  s.total_tiles = (int64_t)tx * ty * v->n_views;
  s.records = (int64_t)v->n_views * g->n;
  s.pixels = (int64_t)v->n_views * v->height * v->width;
  s.n_blocks = (g->n + ddgs::PRE_THREADS - 1) / ddgs::PRE_THREADS;
  // the sizes this fixed scratch can hold
  if (s.records > kMaxRecords || s.total_tiles > kMaxTiles) return DDGS_ERR_CAPACITY;
  t_req[0] = ddgs::ReqTab{0, g->n, g->n_iso, 0, 0, 0, 0, v->n_views};
  t_req[1] = ddgs::ReqTab{g->n, 0, 0, g->n_iso, g->n - g->n_iso, s.n_blocks, v->n_views, 0};
  for (int32_t k = 0; k <= v->n_views; ++k) {
    ddgs::ViewTab &t = t_view[k];
    t.tile_base = (int64_t)k * tx * ty;
    t.rec_off = (int64_t)k * g->n;
    t.img_off = (int64_t)k * v->height * v->width;
    t.req = k < v->n_views ? 0 : 1;
    t.H = v->height;
    t.W = v->width;
    t.tiles_x = tx;
  }
  ddgs::plan_binning(t_view, v->n_views, t_req, s.total_tiles, tile, s, kSlotBudget);
  if (s.hist_slots > kMaxSlots) return DDGS_ERR_CAPACITY;  // not reached: kMaxSlots bounds it

  unsigned char *base = nullptr;
  ddgs_status st = scratch_for_current_device(&base);
  if (st) return st;
  // the long-list sort's shared-memory limit (set once per device; the binning
  // would set it too, but here a failure is reported before any work is queued)
  CK_STATIC(ddgs::prepare_bin_kernels());
  CK_STATIC(ddgs::prepare_raster_kernels());
  cudaStream_t cs = static_cast<cudaStream_t>(stream);

  // A workspace view of the static array (host struct on the stack).
  ddgs_workspace ws;
  ws.rec_cap = kMaxRecords;
  ws.pair_cap = kMaxPairs;
  ws.tile_cap = kMaxTiles;
  ws.blk_cap = kMaxBlocks;
  ws.hist_cap = kMaxSlots;
  ws.list_cap = kMaxListItems;
  ws.rec = reinterpret_cast<float4 *>(base + kOffRec0);  // rec0 and rec1 regions, contiguous
  ws.rect = reinterpret_cast<uint2 *>(base + kOffInfo);
  ws.blk_total = reinterpret_cast<uint32_t *>(base + kOffBlkTotal);
  ws.keys[0] = reinterpret_cast<uint64_t *>(base + kOffKeys0);
  ws.keys[1] = reinterpret_cast<uint64_t *>(base + kOffKeys1);
  ws.vals = reinterpret_cast<uint32_t *>(base + kOffVals);
  ws.hist = reinterpret_cast<uint32_t *>(base + kOffHist);
  ws.part = reinterpret_cast<uint64_t *>(base + kOffPart);
  ws.lists = reinterpret_cast<uint64_t *>(base + kOffLists);
  ws.list_count = reinterpret_cast<uint32_t *>(base + kOffListCount);
  ws.ranges = reinterpret_cast<uint2 *>(base + kOffRanges);
  ws.d_pairs = reinterpret_cast<uint64_t *>(base + kOffPairs);
  ws.d_status = reinterpret_cast<int32_t *>(base + kOffStatus);
  ws.order = reinterpret_cast<uint32_t *>(base + kOffOrder);
  ws.queue = reinterpret_cast<uint32_t *>(base + kOffQueue);
  ws.req_time = nullptr;
  ws.batch_depth = (c->batch_depth == 32 || c->batch_depth == 128 || c->batch_depth == 512)
                       ? c->batch_depth : 256;
  ddgs::ReqTab *d_req = reinterpret_cast<ddgs::ReqTab *>(base + kOffReq);
  ddgs::ViewTab *d_view = reinterpret_cast<ddgs::ViewTab *>(base + kOffView);
  s.req = d_req;
  s.view = d_view;
  // tables from pageable host memory: each copy returns once its source is staged
  CK_STATIC(cudaMemcpyAsync(d_req, t_req, sizeof(t_req), cudaMemcpyHostToDevice, cs));
  CK_STATIC(cudaMemcpyAsync(d_view, t_view, (size_t)(v->n_views + 1) * sizeof(ddgs::ViewTab),
                            cudaMemcpyHostToDevice, cs));

  // counters left by the previous call start again from zero
  CK_STATIC(cudaMemsetAsync(ws.d_status, 0, sizeof(int32_t), cs));
  CK_STATIC(cudaMemsetAsync(ws.d_pairs, 0, sizeof(uint64_t), cs));
  uint64_t pairs = 0;
  if (s.records > 0) {
    ddgs::launch_preprocess_fwd(*g, *v, *c, s, ws, cs);
    ddgs::launch_scan_blocks(s.n_blocks, ws, cs);
    CK_STATIC(cudaGetLastError());
    // the pair count decides the sort's size: read it (no allocation)
    CK_STATIC(cudaMemcpyAsync(&pairs, ws.d_pairs, sizeof(uint64_t), cudaMemcpyDeviceToHost, cs));
    CK_STATIC(cudaStreamSynchronize(cs));
    if (pairs > (uint64_t)kMaxPairs) return DDGS_ERR_CAPACITY;
  }
  if (s.total_tiles > 0) {
    ddgs::launch_binning(s, pairs, ws, cs);
    ddgs::launch_tile_order(s, ws, cs);
    ddgs::RasterParams P{c->alpha_min, c->alpha_max, c->t_min, c->q_max,
                          c->q_max * ddgs::CONIC_SCALE};
    ddgs::launch_raster_fwd(s, P, ws, image, t_final, n_last, nullptr, cs);
  }
  CK_STATIC(cudaGetLastError());
  return DDGS_OK;
}
