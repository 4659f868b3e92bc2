// bin.cu -- tile binning: every (Gaussian, tile) pair goes into its tile's
// list, and each list is put in depth order.
//
// Eq. 1's product runs over the Gaussians on the ray in depth order; the
// tiled renderer orders them once per tile. A pair's tile is known from the
// Gaussian's tile rectangle (preprocess), so the lists are built by counting
// instead of a global sort of (tile, depth) keys:
//   count    blocks of (view, Gaussian chunk, band of tiles) count their pairs
//            per tile in shared memory;
//   offsets  per tile, the chunks' counts are turned into running offsets and
//            the tiles' totals into list ranges (exclusive scans);
//   scatter  the same blocks write (depth bits << 32 | Gaussian) into their
//            slots of each tile's list (shared-memory cursors);
//   sort     every list is ordered by (depth bits, Gaussian) in shared
//            memory: a warp for lists up to 32 entries (bitonic network), a
//            block for longer ones (buckets by the top bits of the depth, each
//            entry placed by counting the smaller keys of its bucket; where
//            depths cluster, stable 8-bit counting passes over the depth bits
//            that vary in the list, then over the Gaussian index where depths
//            tie); lists longer than BIN_LIST_LONG
//            are sorted in chunks that one block then merges (merge path).
// Depth is positive, so its IEEE bits order like the number. The result is the
// unique order of Gaussians by (depth, index), the order of a stable sort of
// the pairs by depth in ascending Gaussian order. No block waits on another.
#include <algorithm>
#include <mutex>

#include "ddgs_internal.cuh"

namespace ddgs {
namespace {

constexpr int BIN_THREADS = 256;   // count blocks
constexpr int SCAT_THREADS = 512;  // scatter blocks
constexpr int SORT_SHORT = 1024;  // lists of one 128-thread block (8 entries a thread)
constexpr int SORT_MID = 2048;    // lists of one 128-thread block (16 entries a thread)
constexpr int MERGE_ITEMS = 8;    // outputs per thread per merge step
constexpr int BIN_LOADS = 4;      // records a thread loads before using them

// ---------------------------------------------------------------------------
// Exclusive scan of block totals -> offsets (optional) and the total (one block)
// ---------------------------------------------------------------------------
template <typename In>
__global__ void __launch_bounds__(1024) scan_blocks_kernel(const In *in, uint64_t *out, int64_t n,
                                                            uint64_t *total) {
  __shared__ uint64_t s_warp[32];
  __shared__ uint64_t s_carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  constexpr int PER = 4;
  for (int64_t base = 0; base < n; base += 1024 * PER) {
    uint64_t x[PER], sum = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      int64_t j = base + (int64_t)tid * PER + k;
      x[k] = j < n ? (uint64_t)in[j] : 0;
      sum += x[k];
    }
    uint64_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      uint64_t w = s_warp[lane];
      uint64_t wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      s_warp[lane] = wi - w;  // exclusive prefix of warp totals
    }
    __syncthreads();
    uint64_t run = s_carry + s_warp[wid] + inc - sum;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      int64_t j = base + (int64_t)tid * PER + k;
      if (j < n && out) out[j] = run;
      run += x[k];
    }
    __syncthreads();
    if (tid == 1023) s_carry = run;
    __syncthreads();
  }
  if (tid == 0 && total) *total = s_carry;
}

// ---------------------------------------------------------------------------
// Binning blocks: (view, chunk of its Gaussians, band of its tiles)
// ---------------------------------------------------------------------------
struct BinItem {
  int64_t rec0, l0, l1;  // records of Gaussians [l0, l1) of the view start at rec0
  int64_t slot;          // first tile counter of the block
  int tx0, ty0, bw, bh;  // the band's first tile and size
};

__device__ __forceinline__ BinItem bin_item(const RenderShape &s, const ViewTab &vt, int64_t item) {
  const int64_t n = s.req[vt.req].n;
  const int64_t j = item - vt.item_base;
  const int64_t band = j / vt.chunks, c = j - band * vt.chunks;
  const int64_t g = (n + vt.chunks - 1) / vt.chunks;
  BinItem it;
  it.rec0 = vt.rec_off;
  it.l0 = c * g;
  it.l1 = min(n, it.l0 + g);
  it.bw = vt.band_w;
  it.bh = vt.band_h;
  it.tx0 = (int)(band % vt.bands_x) * vt.band_w;
  it.ty0 = (int)(band / vt.bands_x) * vt.band_h;
  it.slot = vt.hist_base + j * (int64_t)vt.band_w * vt.band_h;
  return it;
}

// The part of a record's tile rectangle inside the block's band; false when
// the record touches no tile of the band.
__device__ __forceinline__ bool band_rect(const uint4 &b, const BinItem &it, int &x0, int &y0,
                                          int &x1, int &y1) {
  if (b.w == 0) return false;
  x0 = max((int)(b.x & 0xffffu), it.tx0);
  y0 = max((int)(b.x >> 16), it.ty0);
  x1 = min((int)(b.y & 0xffffu), it.tx0 + it.bw - 1);
  y1 = min((int)(b.y >> 16), it.ty0 + it.bh - 1);
  return x0 <= x1 && y0 <= y1;
}

// count: the block's pairs per tile of its band -> hist[slot ...]
// Eight blocks per SM (32 registers, a few bytes spilled): the count waits on
// its record loads, and more warps hide them (0.128 -> 0.122 ms at 64 poses).
__global__ void __launch_bounds__(BIN_THREADS, 8) bin_count_kernel(RenderShape s, const uint4 *info,
                                                                  uint32_t *hist) {
  extern __shared__ uint32_t s_cnt[];
  const ViewTab vt = s.view[find_item_view(s.view, s.V, blockIdx.x)];
  const BinItem it = bin_item(s, vt, blockIdx.x);
  const int area = it.bw * it.bh;
  for (int p = threadIdx.x; p < area; p += BIN_THREADS) s_cnt[p] = 0;
  __syncthreads();
  for (int64_t l0 = it.l0 + threadIdx.x; l0 < it.l1; l0 += BIN_LOADS * BIN_THREADS) {
    uint4 b[BIN_LOADS];
#pragma unroll
    for (int k = 0; k < BIN_LOADS; ++k) {
      const int64_t l = l0 + k * BIN_THREADS;
      b[k] = l < it.l1 ? info[it.rec0 + l] : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int k = 0; k < BIN_LOADS; ++k) {
      int x0, y0, x1, y1;
      if (!band_rect(b[k], it, x0, y0, x1, y1)) continue;
      for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x) atomicAdd(&s_cnt[(y - it.ty0) * it.bw + (x - it.tx0)], 1u);
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < area; p += BIN_THREADS) hist[it.slot + p] = s_cnt[p];
}

// Where a tile's counters are: the band of the tile and its place in it.
__device__ __forceinline__ bool tile_slot(const RenderShape &s, int64_t gt, int64_t &first,
                                          int64_t &stride, int &chunks) {
  const ViewTab vt = s.view[find_view(s.view, s.V, gt)];
  chunks = vt.chunks;
  if (chunks == 0) return false;
  const int64_t t = gt - vt.tile_base;
  const int ty = (int)(t / vt.tiles_x), tx = (int)(t - (int64_t)ty * vt.tiles_x);
  const int bx = tx / vt.band_w, by = ty / vt.band_h;
  const int64_t band = (int64_t)by * vt.bands_x + bx;
  stride = (int64_t)vt.band_w * vt.band_h;
  first = vt.hist_base + band * chunks * stride + (int64_t)(ty - by * vt.band_h) * vt.band_w +
          (tx - bx * vt.band_w);
  return true;
}

// offsets, part 1: per tile, the chunks' counts become running offsets within
// the tile's list; the tile total goes to ranges[gt].y, and each 1024-tile
// group's sum of totals is added to part[group] (zeroed beforehand). A block
// takes 32 tiles (one per lane) and splits their chunks over its 8 warps:
// each warp sums its share of the chunks, the warps' sums are scanned in
// shared memory, and each warp then rewrites its share as running offsets.
// Without pairs (counted = 0) every list is empty.
constexpr int COL_WARPS = 8;
__global__ void __launch_bounds__(COL_WARPS * 32) bin_column_kernel(RenderShape s, int counted,
                                                                     uint32_t *hist, uint2 *ranges,
                                                                     uint64_t *part) {
  __shared__ uint32_t s_sum[COL_WARPS][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t gt = (int64_t)blockIdx.x * 32 + lane;
  int64_t first = 0, stride = 0;
  int chunks = 0;
  const bool has = gt < s.total_tiles && counted && tile_slot(s, gt, first, stride, chunks);
  const int seg = (chunks + COL_WARPS - 1) / COL_WARPS;
  const int c0 = min(chunks, w * seg), c1 = min(chunks, c0 + seg);
  uint32_t *h = hist + first;
  uint32_t sum = 0;
  if (has) {  // eight loads in flight per lane (the kernel waits on DRAM latency:
              // 0.081 -> 0.060 ms for the three offset launches at 64 poses)
    int c = c0;
    for (; c + 8 <= c1; c += 8) {
      uint32_t v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = h[(int64_t)(c + j) * stride];
#pragma unroll
      for (int j = 0; j < 8; ++j) sum += v[j];
    }
    for (; c < c1; ++c) sum += h[(int64_t)c * stride];
  }
  s_sum[w][lane] = sum;
  __syncthreads();
  uint32_t run = 0, total = 0;
#pragma unroll
  for (int x = 0; x < COL_WARPS; ++x) {
    const uint32_t v = s_sum[x][lane];
    if (x < w) run += v;
    total += v;
  }
  if (has) {
    int c = c0;
    for (; c + 8 <= c1; c += 8) {
      uint32_t v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = h[(int64_t)(c + j) * stride];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        h[(int64_t)(c + j) * stride] = run;
        run += v[j];
      }
    }
    for (; c < c1; ++c) {
      const uint32_t x = h[(int64_t)c * stride];
      h[(int64_t)c * stride] = run;
      run += x;
    }
  }
  if (w == 0) {
    if (gt < s.total_tiles) ranges[gt] = make_uint2(0u, total);
    uint64_t t = total;  // the block's 32 tiles lie in one 1024-tile group
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0 && t) atomicAdd(reinterpret_cast<unsigned long long *>(part + (gt >> 10)), t);
  }
}

// Appends the tile's k list entries of one class with one atomic per warp.
__device__ __forceinline__ void list_append(const BinLists &L, int cls, uint64_t gt, uint32_t k) {
  const int lane = threadIdx.x & 31;
  uint32_t inc = k;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  const uint32_t all = __shfl_sync(0xffffffffu, inc, 31);
  if (all == 0) return;  // warp-uniform
  uint32_t base = 0;
  if (lane == 31) base = atomicAdd(&L.count[cls], all);
  base = __shfl_sync(0xffffffffu, base, 31) + inc - k;
  for (uint32_t c = 0; c < k; ++c) L.item[cls][base + c] = (gt << 24) | c;
}

// offsets, part 2: list ranges from the exclusive scan of the tile totals
// ((0, 0) for an empty list), and each list of two or more entries queued for
// its sort. A list that does not fit below the pair capacity is left empty
// (whole lists only) and the capacity status is raised.
__global__ void __launch_bounds__(1024) bin_offsets_kernel(int64_t n_tiles, uint2 *ranges,
                                                             const uint64_t *part_off, uint64_t cap,
                                                             BinLists L, int32_t *status) {
  __shared__ uint64_t s_w[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t gt = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  const uint64_t cnt = gt < n_tiles ? ranges[gt].y : 0;
  uint64_t inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  uint64_t before = part_off[blockIdx.x];
  for (int w = 0; w < wid; ++w) before += s_w[w];
  const uint64_t off = before + inc - cnt;
  uint32_t n = 0;
  if (gt < n_tiles) {
    const bool fits = off + cnt <= cap;
    if (!fits) atomicOr(status, ST_CAPACITY);
    n = fits ? (uint32_t)cnt : 0u;
    ranges[gt] = n ? make_uint2((uint32_t)off, (uint32_t)(off + cnt)) : make_uint2(0u, 0u);
  }
  list_append(L, LIST_WARP, (uint64_t)gt, n >= 2 && n <= 32 ? 1u : 0u);
  list_append(L, LIST_SHORT, (uint64_t)gt, n > 32 && n <= SORT_SHORT ? 1u : 0u);
  list_append(L, LIST_MID, (uint64_t)gt, n > SORT_SHORT && n <= SORT_MID ? 1u : 0u);
  list_append(L, LIST_BLOCK, (uint64_t)gt,
              n > SORT_MID ? (n + BIN_LIST_LONG - 1) / BIN_LIST_LONG : 0u);
  list_append(L, LIST_LONG, (uint64_t)gt, n > BIN_LIST_LONG ? 1u : 0u);
}

// L2 eviction priority of the binning records: they stream through once
// (evict first).
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint4 ld_hint(const uint4 *a, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(a), "l"(pol));
  return v;
}

// scatter: every pair of the block goes to its tile's list, at the tile's
// offset plus the earlier chunks' counts plus its rank within the block. The
// block stages its pairs in shared memory, grouped by tile, and then writes
// them out in that order, so that each tile's run of pairs leaves as one
// stretch of consecutive 8-byte entries instead of single scattered stores.
// A chunk whose pairs exceed the staging area is done in windows of
// consecutive band tiles (its records are read again per window, from L2); a
// single tile with more pairs than the area is written directly. Lists of one
// entry are final here (flag bit 31 of the destination; offsets stay below
// BIN_MAX_PAIRS < 2^31). Pairs of lists left empty by a capacity overflow are
// dropped.
constexpr uint32_t CUR_ONE = 0x80000000u, CUR_DROP = 0xffffffffu;
// pairs staged per window (12 bytes each): with a band of 1,024 tiles a block
// then takes 74 KB and three fit an SM (0.59 -> 0.58 ms at 64 poses; 4,096
// makes more chunks need a second window, 0.76 ms)
constexpr int SCAT_STAGE = 5120;

__host__ __device__ constexpr size_t scatter_smem(int area, bool direct = false) {
  return (direct ? 0 : (size_t)SCAT_STAGE * (sizeof(uint64_t) + sizeof(uint32_t))) +
         (size_t)area * 3 * sizeof(uint32_t);
}

// In-place exclusive scan of a[0, n) by the whole block; returns the total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t *a, int n, uint32_t *s_wsum) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int per = (n + SCAT_THREADS - 1) / SCAT_THREADS, b = tid * per;
  uint32_t loc = 0;
  for (int k = 0; k < per; ++k)
    if (b + k < n) loc += a[b + k];
  uint32_t inc = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_wsum[w] = inc;
  __syncthreads();
  uint32_t ex = inc - loc, total = 0;
  for (int x = 0; x < SCAT_THREADS / 32; ++x) {
    if (x < w) ex += s_wsum[x];
    total += s_wsum[x];
  }
  for (int k = 0; k < per; ++k)
    if (b + k < n) {
      const uint32_t c = a[b + k];
      a[b + k] = ex;
      ex += c;
    }
  __syncthreads();
  return total;
}

// Three blocks per SM (40 registers; the staging area and a 1,024-tile band
// fit three times in shared memory): 0.58 -> 0.54 ms at 64 poses, against two
// at the 60 registers the compiler takes by itself.
// DIRECT: no staging; every pair is written where it goes, in one pass over
// the block's records. Chosen per render when the blocks average more pairs
// than two staging windows (each further window would read the chunk's
// records again): 2M Gaussians on eight 1024^2 views, 2.6 -> 1.1 ms.
template <bool DIRECT>
__global__ void __launch_bounds__(SCAT_THREADS, 3) bin_scatter_kernel(RenderShape s, const uint4 *info,
                                                                    const uint32_t *hist,
                                                                    const uint2 *ranges,
                                                                    uint64_t *keys, uint32_t *vals,
                                                                    uint64_t cap) {
  extern __shared__ __align__(16) unsigned char scat_smem[];
  __shared__ uint32_t s_wsum[SCAT_THREADS / 32];
  const ViewTab vt = s.view[find_item_view(s.view, s.V, blockIdx.x)];
  const BinItem it = bin_item(s, vt, blockIdx.x);
  const int tiles_y = (vt.H + s.tile - 1) / s.tile;
  const int area = it.bw * it.bh;
  constexpr int STAGE = DIRECT ? 0 : SCAT_STAGE;
  uint64_t *s_key = reinterpret_cast<uint64_t *>(scat_smem);  // [STAGE] staged pairs
  uint32_t *s_dst = reinterpret_cast<uint32_t *>(s_key + STAGE);  // [STAGE] their places
  uint32_t *s_base = s_dst + STAGE;  // [area] place of the tile's first pair of this block
  uint32_t *s_beg = s_base + area;        // [area] counts, then their exclusive prefix
  uint32_t *s_cur = s_beg + area;         // [area] staging cursors
  const int64_t j = (int64_t)blockIdx.x - vt.item_base;
  const bool last_chunk = j % vt.chunks == vt.chunks - 1;
  for (int p = threadIdx.x; p < area; p += SCAT_THREADS) {
    const int x = it.tx0 + p % it.bw, y = it.ty0 + p / it.bw;
    uint32_t base = CUR_DROP, cnt = 0;
    if (x < vt.tiles_x && y < tiles_y) {
      const uint2 r = ranges[vt.tile_base + (int64_t)y * vt.tiles_x + x];
      if (r.y > r.x) {
        const uint32_t off = hist[it.slot + p];  // the chunk's offset within the list
        const uint32_t next = last_chunk ? r.y - r.x : hist[it.slot + area + p];
        base = (r.x + off) | (r.y - r.x == 1 ? CUR_ONE : 0u);
        cnt = next - off;
      }
    }
    s_base[p] = base;
    s_beg[p] = cnt;
  }
  __syncthreads();
  const uint32_t all = block_exclusive_scan(s_beg, area, s_wsum);  // the block's pairs
  for (int p = threadIdx.x; p < area; p += SCAT_THREADS) s_cur[p] = s_beg[p];
  __syncthreads();
  const uint64_t pol_in = l2_policy_evict_first();
  if (DIRECT) {
    for (int64_t l0 = it.l0 + threadIdx.x; l0 < it.l1; l0 += SCAT_THREADS) {
      const uint4 b = ld_hint(info + it.rec0 + l0, pol_in);
      int x0, y0, x1, y1;
      if (!band_rect(b, it, x0, y0, x1, y1)) continue;
      const uint32_t l = (uint32_t)l0;
      const uint64_t key = ((uint64_t)b.z << 32) | l;
      for (int y = y0; y <= y1; ++y) {
        const int row = (y - it.ty0) * it.bw;
        for (int x = x0; x <= x1; ++x) {
          const int p = row + (x - it.tx0);
          if (s_base[p] == CUR_DROP) continue;
          const uint32_t c = atomicAdd(&s_cur[p], 1u);
          const uint32_t dst = s_base[p] + (c - s_beg[p]);  // keeps the CUR_ONE flag
          const uint32_t pos = dst & ~CUR_ONE;
          if (pos >= cap) continue;
          if (dst & CUR_ONE) vals[pos] = l;
          else keys[pos] = key;
        }
      }
    }
    return;
  }
  int w0 = 0;
  while (w0 < area) {  // block-uniform windows of tiles [w0, w1)
    const uint32_t b0 = s_beg[w0];
    // the largest w1 whose pairs fit the staging area (binary search on the
    // prefix; prefix(area) = all)
    int lo = w0, hi = area;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if ((mid < area ? s_beg[mid] : all) - b0 <= (uint32_t)SCAT_STAGE) lo = mid; else hi = mid - 1;
    }
    const bool direct = lo == w0;  // tile w0 alone has more pairs than the area
    const int w1 = direct ? w0 + 1 : lo;
    const uint32_t n_win = direct ? 0u : (w1 < area ? s_beg[w1] : all) - b0;
    for (int64_t l0 = it.l0 + threadIdx.x; (direct || n_win > 0) && l0 < it.l1;
         l0 += BIN_LOADS * SCAT_THREADS) {
      uint4 b[BIN_LOADS];
#pragma unroll
      for (int k = 0; k < BIN_LOADS; ++k) {
        const int64_t l = l0 + k * SCAT_THREADS;
        b[k] = l < it.l1 ? ld_hint(info + it.rec0 + l, pol_in) : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int k = 0; k < BIN_LOADS; ++k) {
        int x0, y0, x1, y1;
        if (!band_rect(b[k], it, x0, y0, x1, y1)) continue;
        const uint32_t l = (uint32_t)(l0 + k * SCAT_THREADS);
        const uint64_t key = ((uint64_t)b[k].z << 32) | l;
        for (int y = y0; y <= y1; ++y) {
          const int row = (y - it.ty0) * it.bw;
          for (int x = x0; x <= x1; ++x) {
            const int p = row + (x - it.tx0);
            if (p < w0 || p >= w1 || s_base[p] == CUR_DROP) continue;
            const uint32_t c = atomicAdd(&s_cur[p], 1u);
            const uint32_t dst = s_base[p] + (c - s_beg[p]);  // keeps the CUR_ONE flag
            if (direct) {
              const uint32_t pos = dst & ~CUR_ONE;
              if (pos >= cap) continue;
              if (dst & CUR_ONE) vals[pos] = l;
              else keys[pos] = key;
            } else {
              s_key[c - b0] = key;
              s_dst[c - b0] = dst;
            }
          }
        }
      }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n_win; i += SCAT_THREADS) {
      const uint32_t dst = s_dst[i], pos = dst & ~CUR_ONE;
      if (pos >= cap) continue;
      if (dst & CUR_ONE) vals[pos] = (uint32_t)s_key[i];
      else keys[pos] = s_key[i];
    }
    __syncthreads();
    w0 = w1;
  }
}

// ---------------------------------------------------------------------------
// List sorts
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t x, int m) {
  const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)x, m);
  const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(x >> 32), m);
  return ((uint64_t)hi << 32) | lo;
}

// Lists of 2..32 entries: one warp each, a bitonic network over 64-bit keys.
__global__ void __launch_bounds__(256) bin_sort_warp_kernel(const uint64_t *items,
                                                              const uint32_t *count,
                                                              const uint2 *ranges,
                                                              const uint64_t *keys, uint32_t *vals) {
  const int lane = threadIdx.x & 31;
  const uint32_t n_items = *count;
  const uint32_t nw = gridDim.x * (blockDim.x >> 5);
  for (uint32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n_items; i += nw) {
    const uint2 r = ranges[items[i] >> 24];
    const uint32_t n = r.y - r.x;
    uint64_t k = lane < (int)n ? keys[r.x + lane] : ~0ull;
#pragma unroll
    for (int w = 2; w <= 32; w <<= 1) {
#pragma unroll
      for (int j = w >> 1; j > 0; j >>= 1) {
        const uint64_t o = shfl_xor_u64(k, j);
        const bool up = (lane & w) == 0, lower = (lane & j) == 0;
        k = (lower == up) ? (k < o ? k : o) : (k < o ? o : k);
      }
    }
    if (lane < (int)n) vals[r.x + lane] = (uint32_t)k;
  }
}

// One stable counting pass of a block over the 8-bit digit at `shift` of
// src[0, m) into dst. Warp w owns the entries [w seg, (w + 1) seg) and ranks
// them in order: the lanes holding the same digit are found from eight
// ballots (one per digit bit), and the lowest of them advances a per-warp
// counter. The digit totals of all warps are then scanned digit-major,
// warp-minor.
template <int NT, int E>
__device__ __forceinline__ void block_digit_pass(const uint64_t *src, uint64_t *dst, int m,
                                                 int seg, int rows, int shift,
                                                 uint32_t (*cnt)[256], uint32_t *s_wsum) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  for (int d = lane; d < 256; d += 32) cnt[w][d] = 0;
  __syncwarp();
  uint32_t rank[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    if (r < rows) {  // block-uniform
      const int idx = w * seg + r * 32 + lane;
      const bool ok = idx < m;
      const uint32_t d = ok ? (uint32_t)(src[idx] >> shift) & 255u : 0u;
      uint32_t peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const uint32_t bit = (d >> b) & 1u;
        const uint32_t v = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? v : ~v;
      }
      const int leader = ok ? __ffs(peers) - 1 : lane;
      uint32_t before = 0;
      if (ok && lane == leader) {
        before = cnt[w][d];
        cnt[w][d] = before + __popc(peers);
      }
      rank[r] = __shfl_sync(0xffffffffu, before, leader) + __popc(peers & lt);
      __syncwarp();
    }
  }
  __syncthreads();
  // per digit: the warps' running bases, then an exclusive scan over digits
  // (each thread takes DPT consecutive digits)
  constexpr int DPT = NT < 256 ? 256 / NT : 1;
  const bool dig = tid * DPT < 256;  // warp-uniform
  uint32_t tot[DPT], loc = 0, inc = 0;
  if (dig) {
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int d = tid * DPT + j;
      uint32_t run = 0;
#pragma unroll
      for (int x = 0; x < NW; ++x) {
        const uint32_t c = cnt[x][d];
        cnt[x][d] = run;
        run += c;
      }
      tot[j] = run;
      loc += run;
    }
    inc = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_wsum[w] = inc;
  }
  __syncthreads();
  if (dig) {
    uint32_t ex = inc - loc;
    for (int x = 0; x < w; ++x) ex += s_wsum[x];
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
      const int d = tid * DPT + j;
#pragma unroll
      for (int x = 0; x < NW; ++x) cnt[x][d] += ex;
      ex += tot[j];
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < E; ++r) {
    if (r < rows) {
      const int idx = w * seg + r * 32 + lane;
      if (idx < m) {
        const uint64_t k = src[idx];
        dst[cnt[w][(uint32_t)(k >> shift) & 255u] + rank[r]] = k;
      }
    }
  }
  __syncthreads();
}

// Lists (or BIN_LIST_LONG-entry chunks of longer lists) of up to NT x E
// entries: one block each, in shared memory. First a bucket sort: the top
// bits of (depth - smallest depth) spread the entries over about as many
// buckets as entries (shared-memory counters); then every entry finds its
// place as its bucket's start plus the number of smaller (depth, index) keys
// in its bucket (keys are unique), and goes straight to the output. (An
// insertion sort per bucket, one thread a bucket, cost 25 % more at the
// benchmark: views near an axis of the voxel grid put up to ~20 entries of
// near-equal depth in one bucket.) Where a bucket would hold more than
// BUCKET_MAX entries (clustered or equal depths), the list is sorted instead
// by stable 8-bit passes over the depth bits that differ in it, redone with
// the index digits first if two depths are equal. Whole lists write their
// values; chunks write their sorted keys back for the merge.
constexpr uint32_t BUCKET_MAX = 24;
template <int NT, int E, int MINB>
__global__ void __launch_bounds__(NT, MINB) bin_sort_block_kernel(const uint64_t *items,
                                                                    const uint32_t *count,
                                                                    const uint2 *ranges,
                                                                    uint64_t *keys, uint32_t *vals) {
  constexpr int NW = NT / 32, CAP = NT * E;
  extern __shared__ __align__(16) uint64_t s_buf[];  // [2][CAP]
  // digit counters, or up to NW x 256 bucket counters stored with one pad word
  // after every eight (bkp), so that the bucket scan's per-thread runs of
  // eight counters fall in distinct banks (0.70 -> 0.64 ms for the sorts at 64
  // poses; unpadded, the runs of a warp's lanes met 8-way bank conflicts)
  __shared__ __align__(16) uint32_t s_bk[NW * 256 + NW * 32];
  uint32_t(*cnt)[256] = reinterpret_cast<uint32_t(*)[256]>(s_bk);
  auto bkp = [](uint32_t b) { return b + (b >> 3); };
  __shared__ uint32_t s_wsum[NW > 8 ? NW : 8];
  __shared__ uint32_t s_red[4][NW];
  uint32_t *bc = s_bk;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t n_items = *count;
  // the next item's keys are copied to s_buf asynchronously while the
  // current one is placed (once its keys have left s_buf)
  auto prefetch = [&](uint32_t in) {
    if (in >= n_items) return false;
    const uint64_t it2 = items[in];
    const uint2 r2 = ranges[it2 >> 24];
    const uint32_t c2 = (uint32_t)(it2 & 0xffffffu);
    const uint32_t b2 = r2.x + c2 * (uint32_t)CAP;
    const int m2 = (int)min((uint32_t)CAP, (r2.y - r2.x) - c2 * (uint32_t)CAP);
    for (int j = tid; j < m2; j += NT) {
      const unsigned sa = (unsigned)__cvta_generic_to_shared(s_buf + j);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(keys + b2 + j) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    return true;
  };
  bool have = false;
  for (uint32_t i = blockIdx.x; i < n_items; i += gridDim.x) {
    const uint64_t item = items[i];
    const uint2 r = ranges[item >> 24];
    const uint32_t chunk = (uint32_t)(item & 0xffffffu);
    const uint32_t n_all = r.y - r.x;
    const uint32_t base = r.x + chunk * (uint32_t)CAP;
    const int m = (int)min((uint32_t)CAP, n_all - chunk * (uint32_t)CAP);
    uint64_t *cur = s_buf, *oth = s_buf + CAP;
    uint32_t dmin = ~0u, dmax = 0u, lmin = ~0u, lmax = 0u;
    if (have) {
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();
    }
    for (int j = tid; j < m; j += NT) {
      uint64_t k;
      if (have) {
        k = cur[j];
      } else {
        k = keys[base + j];
        cur[j] = k;
      }
      const uint32_t d = (uint32_t)(k >> 32), l = (uint32_t)k;
      dmin = min(dmin, d); dmax = max(dmax, d);
      lmin = min(lmin, l); lmax = max(lmax, l);
    }
    have = false;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dmin = min(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
      dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
      lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    }
    if (lane == 0) {
      s_red[0][w] = dmin; s_red[1][w] = dmax; s_red[2][w] = lmin; s_red[3][w] = lmax;
    }
    __syncthreads();
    dmin = s_red[0][0]; dmax = s_red[1][0]; lmin = s_red[2][0]; lmax = s_red[3][0];
#pragma unroll
    for (int x = 1; x < NW; ++x) {
      dmin = min(dmin, s_red[0][x]); dmax = max(dmax, s_red[1][x]);
      lmin = min(lmin, s_red[2][x]); lmax = max(lmax, s_red[3][x]);
    }
    bool sorted = false;
    if (dmin != dmax && m > 1) {
      // buckets: 2^lg >= m of them (at least 32, at most NW x 256)
      int lg = 32 - __clz((uint32_t)m - 1u);
      lg = max(5, min(lg, 31 - __clz((uint32_t)(NW * 256))));
      const int nbk = 1 << lg;
      const int sh = max(0, (32 - __clz(dmax - dmin)) - lg);
      for (int b = tid; b < nbk; b += NT) bc[bkp(b)] = 0;
      __syncthreads();
      uint32_t rk[E];
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int j = tid + r * NT;
        if (j < m) rk[r] = atomicAdd(&bc[bkp(((uint32_t)(cur[j] >> 32) - dmin) >> sh)], 1u);
      }
      __syncthreads();
      // exclusive scan of the bucket counts (contiguous runs per thread) and
      // the largest bucket
      const int q = (nbk + NT - 1) / NT;
      uint32_t loc = 0, big = 0;
      for (int k = 0; k < q; ++k) {
        const int b = tid * q + k;
        if (b < nbk) {
          const uint32_t c = bc[bkp(b)];
          loc += c;
          big = max(big, c);
        }
      }
      uint32_t inc = loc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
        big = max(big, __shfl_xor_sync(0xffffffffu, big, o));
      }
      if (lane == 31) s_wsum[w] = inc;
      if (lane == 0) s_red[0][w] = big;
      __syncthreads();
      uint32_t ex = inc - loc;
      big = 0;
      for (int x = 0; x < NW; ++x) {
        if (x < w) ex += s_wsum[x];
        big = max(big, s_red[0][x]);
      }
      for (int k = 0; k < q; ++k) {
        const int b = tid * q + k;
        if (b < nbk) {
          const uint32_t c = bc[bkp(b)];
          bc[bkp(b)] = ex;
          ex += c;
        }
      }
      __syncthreads();
      if (big <= BUCKET_MAX) {  // block-uniform
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const int j = tid + r * NT;
          if (j < m) {
            const uint64_t k = cur[j];
            oth[bc[bkp(((uint32_t)(k >> 32) - dmin) >> sh)] + rk[r]] = k;
          }
        }
        __syncthreads();
        have = prefetch(i + gridDim.x);  // s_buf (cur) is free from here
        // every entry's place: its bucket's start plus the number of smaller
        // keys in its bucket (keys are unique), written straight to the output
        const bool whole = n_all <= (uint32_t)CAP;
        for (int j = tid; j < m; j += NT) {
          const uint64_t k = oth[j];
          const uint32_t b = ((uint32_t)(k >> 32) - dmin) >> sh;
          const uint32_t b0 = bc[bkp(b)], b1 = b + 1 < (uint32_t)nbk ? bc[bkp(b + 1)] : (uint32_t)m;
          uint32_t pos = b0;
          for (uint32_t x = b0; x < b1; ++x) pos += oth[x] < k;
          if (whole) vals[base + pos] = (uint32_t)k;
          else keys[base + pos] = k;
        }
        __syncthreads();
        continue;
      }
    }
    const int rows_all = (m + 31) / 32;
    const int rows = (rows_all + NW - 1) / NW, seg = rows * 32;
    // depth digits first; only if two depths tie, redo with the index digits
    // below them (least significant first)
    const int nd = sorted || dmin == dmax ? 0 : (39 - __clz(dmin ^ dmax)) / 8;
    int nl = 0;
    for (int round = 0; round < 2 && !sorted; ++round) {
      for (int p = 0; p < nl + nd; ++p) {
        const int shift = p < nl ? 8 * p : 32 + 8 * (p - nl);
        block_digit_pass<NT, E>(cur, oth, m, seg, rows, shift, cnt, s_wsum);
        uint64_t *t = cur; cur = oth; oth = t;
      }
      if (round == 1) break;
      int tie = 0;
      for (int j = tid + 1; j < m; j += NT) tie |= (cur[j] >> 32) == (cur[j - 1] >> 32);
      if (!__syncthreads_or(tie)) break;
      nl = lmin == lmax ? 0 : (39 - __clz(lmin ^ lmax)) / 8;
    }
    if (n_all <= (uint32_t)CAP) {
      for (int j = tid; j < m; j += NT) vals[base + j] = (uint32_t)cur[j];
    } else {
      for (int j = tid; j < m; j += NT) keys[base + j] = cur[j];
    }
    __syncthreads();
    have = prefetch(i + gridDim.x);
  }
}

// Lists longer than BIN_LIST_LONG: their sorted chunks are merged pairwise,
// one block per list, run length doubling until one run is left (the last
// merge writes the values). Each thread finds where its MERGE_ITEMS outputs
// start on the merge path by binary search, then merges them.
__global__ void __launch_bounds__(256) bin_merge_kernel(const uint64_t *items, const uint32_t *count,
                                                         const uint2 *ranges, uint64_t *keys0,
                                                         uint64_t *keys1, uint32_t *vals) {
  const uint32_t n_items = *count;
  for (uint32_t i = blockIdx.x; i < n_items; i += gridDim.x) {
    const uint2 r = ranges[items[i] >> 24];
    const uint64_t n = r.y - r.x;
    uint64_t *src = keys0 + r.x, *dst = keys1 + r.x;
    for (uint64_t R = BIN_LIST_LONG; R < n; R <<= 1) {
      const bool last = 2 * R >= n;
      for (uint64_t p = (uint64_t)threadIdx.x * MERGE_ITEMS; p < n;
           p += (uint64_t)blockDim.x * MERGE_ITEMS) {
        const uint64_t a0 = p / (2 * R) * (2 * R);
        const uint64_t a1 = min(a0 + R, n), b1 = min(a0 + 2 * R, n);
        const uint64_t la = a1 - a0, lb = b1 - a1, d = p - a0;
        uint64_t lo = d > lb ? d - lb : 0, hi = min(d, la);
        while (lo < hi) {
          const uint64_t mid = (lo + hi) >> 1;
          if (src[a0 + mid] < src[a1 + d - mid - 1]) lo = mid + 1; else hi = mid;
        }
        uint64_t ia = lo, ib = d - lo;
        for (int k = 0; k < MERGE_ITEMS && p + k < b1; ++k) {
          uint64_t v;
          if (ia < la && (ib >= lb || src[a0 + ia] < src[a1 + ib])) v = src[a0 + ia++];
          else v = src[a1 + ib++];
          if (last) vals[r.x + p + k] = (uint32_t)v;
          else dst[p + k] = v;
        }
      }
      __syncthreads();
      uint64_t *t = src;
      src = dst;
      dst = t;
    }
  }
}

constexpr int SORT_LONG_THREADS = 512, SORT_LONG_ITEMS = BIN_LIST_LONG / SORT_LONG_THREADS;
constexpr size_t SHORT_SMEM = 2 * SORT_SHORT * sizeof(uint64_t);
constexpr size_t MID_SMEM = 2 * SORT_MID * sizeof(uint64_t);
constexpr size_t LONG_SMEM = 2 * (size_t)BIN_LIST_LONG * sizeof(uint64_t);

}  // namespace

void launch_scan_blocks(int64_t nblk, ddgs_workspace &ws, cudaStream_t st) {
  LaunchScope ls(KID_SCAN_BLOCKS, st);
  scan_blocks_kernel<uint32_t><<<1, 1024, 0, st>>>(ws.blk_total, nullptr, nblk, ws.d_pairs);
}

int64_t list_capacity(int64_t tiles, int64_t pairs) {
  // per class at most one entry per tile, plus one per BIN_LIST_LONG pairs for
  // the chunks of long lists
  return LIST_CLASSES * tiles + pairs / BIN_LIST_LONG + 64;
}

int64_t part_capacity(int64_t tiles) { return 2 * ((tiles + 1023) / 1024) + 2; }


cudaError_t prepare_bin_kernels() {
  // the block sorts keep two copies of a list in dynamic shared memory; the
  // attributes are set once per device, outside any stream capture
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(bin_sort_block_kernel<SORT_LONG_THREADS, SORT_LONG_ITEMS, 1>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LONG_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(bin_scatter_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)scatter_smem(BIN_HIST_MAX));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(bin_scatter_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)scatter_smem(BIN_HIST_MAX, true));
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

void launch_binning(const RenderShape &s, uint64_t pair_bound, ddgs_workspace &ws,
                    cudaStream_t st) {
  const int64_t T = s.total_tiles;
  if (T <= 0) return;
  if (prepare_bin_kernels() != cudaSuccess) return;  // surfaces via cudaGetLastError
  const uint64_t cap = (uint64_t)ws.pair_cap;
  const size_t hsm = (size_t)s.hist_area * sizeof(uint32_t);  // <= 32 KiB
  const unsigned sms = (unsigned)device_sms();  // the sorts run persistent blocks per SM
  const bool pairs = pair_bound > 0 && s.n_items > 0;
  if (pairs) {
    LaunchScope ls(KID_BIN_COUNT, st);
    bin_count_kernel<<<(unsigned)s.n_items, BIN_THREADS, hsm, st>>>(
        s, reinterpret_cast<const uint4 *>(ws.rect), ws.hist);
  }
  const int64_t nb = (T + 1023) / 1024;
  uint64_t *part = ws.part, *part_off = ws.part + nb + 1;
  BinLists L;  // at most T entries per class, except the chunks of long lists (last)
  L.item[LIST_WARP] = ws.lists;
  L.item[LIST_SHORT] = ws.lists + T;
  L.item[LIST_MID] = ws.lists + 2 * T;
  L.item[LIST_LONG] = ws.lists + 3 * T;
  L.item[LIST_BLOCK] = ws.lists + 4 * T;
  L.count = ws.list_count;
  cudaMemsetAsync(ws.list_count, 0, LIST_CLASSES * sizeof(uint32_t), st);
  cudaMemsetAsync(part, 0, (size_t)nb * sizeof(uint64_t), st);
  {
    LaunchScope ls(KID_BIN_OFFSETS, st);
    bin_column_kernel<<<(unsigned)((T + 31) / 32), COL_WARPS * 32, 0, st>>>(s, pairs ? 1 : 0, ws.hist,
                                                                          ws.ranges, part);
  }
  {
    LaunchScope ls(KID_BIN_OFFSETS, st);
    scan_blocks_kernel<uint64_t><<<1, 1024, 0, st>>>(part, part_off, nb, nullptr);
  }
  {
    LaunchScope ls(KID_BIN_OFFSETS, st);
    bin_offsets_kernel<<<(unsigned)nb, 1024, 0, st>>>(T, ws.ranges, part_off, cap, L, ws.d_status);
  }
  if (!pairs) return;
  {
    LaunchScope ls(KID_BIN_SCATTER, st);
    // the pair bound (the count, or the capacity without a sync) over the blocks
    const bool direct = pair_bound > 2u * (uint64_t)SCAT_STAGE * (uint64_t)s.n_items;
    if (direct)
      bin_scatter_kernel<true><<<(unsigned)s.n_items, SCAT_THREADS, scatter_smem(s.hist_area, true), st>>>(
          s, reinterpret_cast<const uint4 *>(ws.rect), ws.hist, ws.ranges, ws.keys[0], ws.vals, cap);
    else
      bin_scatter_kernel<false><<<(unsigned)s.n_items, SCAT_THREADS, scatter_smem(s.hist_area), st>>>(
          s, reinterpret_cast<const uint4 *>(ws.rect), ws.hist, ws.ranges, ws.keys[0], ws.vals, cap);
  }
  // A list holds at most one entry per Gaussian of its request, so a render of
  // n_total Gaussians in all cannot fill the classes of longer lists: those
  // sorts (and the merge) are not launched.
  const int64_t nmax = s.n_total;
  if (nmax >= 2) {
    LaunchScope ls(KID_BIN_SORT, st);
    bin_sort_warp_kernel<<<sms * 4, 256, 0, st>>>(L.item[LIST_WARP], L.count + LIST_WARP,
                                                   ws.ranges, ws.keys[0], ws.vals);
  }
  if (nmax > 32) {
    LaunchScope ls(KID_BIN_SORT, st);
    bin_sort_block_kernel<128, SORT_SHORT / 128, 8><<<sms * 8, 128, SHORT_SMEM, st>>>(
        L.item[LIST_SHORT], L.count + LIST_SHORT, ws.ranges, ws.keys[0], ws.vals);
  }
  if (nmax > SORT_SHORT) {
    LaunchScope ls(KID_BIN_SORT, st);
    // six blocks per SM (80 registers, a few bytes spilled): with the padded
    // bucket counters 0.636 -> 0.629 ms for the sorts at 64 poses against five
    // at 96 registers (which led before the padding, 0.69 against 0.72; four
    // at 128 registers measured 0.75)
    bin_sort_block_kernel<128, SORT_MID / 128, 6><<<sms * 6, 128, MID_SMEM, st>>>(
        L.item[LIST_MID], L.count + LIST_MID, ws.ranges, ws.keys[0], ws.vals);
  }
  if (nmax > SORT_MID) {
    LaunchScope ls(KID_BIN_SORT, st);
    bin_sort_block_kernel<SORT_LONG_THREADS, SORT_LONG_ITEMS, 1>
        <<<sms, SORT_LONG_THREADS, LONG_SMEM, st>>>(L.item[LIST_BLOCK], L.count + LIST_BLOCK,
                                                   ws.ranges, ws.keys[0], ws.vals);
  }
  if (nmax > BIN_LIST_LONG) {
    LaunchScope ls(KID_BIN_MERGE, st);
    bin_merge_kernel<<<sms * 2, 256, 0, st>>>(L.item[LIST_LONG], L.count + LIST_LONG, ws.ranges,
                                              ws.keys[0], ws.keys[1], ws.vals);
  }
}

}  // namespace ddgs
