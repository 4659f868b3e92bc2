// sort.cu -- tile binning: prefix sums of tiles touched, a device LSD radix
// sort of the packed (global tile, depth) keys, and per-tile list ranges.
//
// Eq. 1's product runs over the Gaussians "on the ray" in order; the tiled
// renderer orders them once per tile by sorting 64-bit keys
// (global tile << 32 | depth bits) with their Gaussian index as value. Depth
// is positive, so its IEEE bits sort like the number. The sort is a stable
// least-significant-digit radix sort over only the significant key bits, so
// equal keys keep their emission order (ascending Gaussian index).
//
// A prepass reads the keys once and counts every pass's 8-bit digits; a plan
// kernel turns the counts into each digit's global start and marks the
// passes whose digit is the same in every key (skipped). Each pass is then
// one kernel: blocks take tiles of 4096 keys in ticket order, rank their keys
// stably (warp match + per-warp digit counters), publish their digit counts
// and add up the counts of the earlier tiles (decoupled look-back) before
// scattering keys and values. The look-back waits only on tiles whose blocks
// are already running; every wait has an iteration limit, after which the
// pass reports DDGS_ERR_TIMEOUT and writes only in-bounds positions.
#include <algorithm>
#include <mutex>

#include "ddgs_internal.cuh"

namespace ddgs {
namespace {

// ---------------------------------------------------------------------------
// K2: exclusive scan of the preprocess block totals -> block offsets, total
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) scan_blocks_kernel(const uint32_t *in, uint64_t *out,
                                                            int64_t n, uint64_t *total,
                                                            uint64_t *host_total) {
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
      x[k] = j < n ? in[j] : 0;
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
      if (j < n) out[j] = run;
      run += x[k];
    }
    __syncthreads();
    if (tid == 1023) s_carry = run;
    __syncthreads();
  }
  if (tid == 0) {
    *total = s_carry;
    if (host_total) *host_total = s_carry;
  }
}

// ---------------------------------------------------------------------------
// Radix sort
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t pair_count(const uint64_t *d_pairs, uint64_t cap) {
  uint64_t m = *d_pairs;
  return m < cap ? m : cap;
}

// ---- prepass: the digit histograms of every pass from one read of the keys ----
// Warp-private counters in shared memory ([pass][warp][digit]); a grid-stride
// loop over pairs of keys, so that few blocks add their totals to the global
// histograms.
__global__ void __launch_bounds__(SORT_THREADS) radix_hist_kernel(const uint64_t *keys,
                                                                  const uint64_t *d_pairs,
                                                                  uint64_t cap, int passes,
                                                                  SortState *ss) {
  extern __shared__ uint32_t h_smem[];
  constexpr int NW = SORT_THREADS / 32;
  const int tid = threadIdx.x, wid = tid >> 5;
  for (int e = tid; e < passes * NW * RADIX; e += SORT_THREADS) h_smem[e] = 0;
  __syncthreads();
  const uint64_t m = pair_count(d_pairs, cap);
  const ulonglong2 *p2 = reinterpret_cast<const ulonglong2 *>(keys);
  for (uint64_t i = (uint64_t)blockIdx.x * SORT_THREADS + tid; i < m / 2;
       i += (uint64_t)gridDim.x * SORT_THREADS) {
    const ulonglong2 v = p2[i];
    for (int p = 0; p < passes; ++p) {
      uint32_t *hp = h_smem + (p * NW + wid) * RADIX;
      atomicAdd(&hp[(v.x >> (RADIX_BITS * p)) & (RADIX - 1)], 1u);
      atomicAdd(&hp[(v.y >> (RADIX_BITS * p)) & (RADIX - 1)], 1u);
    }
  }
  if ((m & 1) && blockIdx.x == 0 && tid == 0) {
    const uint64_t k = keys[m - 1];
    for (int p = 0; p < passes; ++p) atomicAdd(&h_smem[p * NW * RADIX + ((k >> (RADIX_BITS * p)) & (RADIX - 1))], 1u);
  }
  __syncthreads();
  for (int e = tid; e < passes * RADIX; e += SORT_THREADS) {
    const int p = e / RADIX, d = e % RADIX;
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) c += h_smem[(p * NW + w) * RADIX + d];
    if (c) atomicAdd(&ss->hist[p][d], c);
  }
}

// ---- plan (one block of RADIX threads): per pass, the global start of every
// digit, whether the pass is skipped (one digit holds every key: the pass is
// an identity), the buffer each pass reads, and the tile tickets ----
__global__ void __launch_bounds__(RADIX) radix_plan_kernel(SortState *ss, const uint64_t *d_pairs,
                                                           uint64_t cap, int passes) {
  __shared__ uint32_t s_w[RADIX / 32];
  __shared__ uint32_t s_skip;
  const int d = threadIdx.x, lane = d & 31, wid = d >> 5;
  const uint64_t m = pair_count(d_pairs, cap);
  if (d == 0) s_skip = 0;
  __syncthreads();
  for (int p = 0; p < passes; ++p) {
    const uint32_t c = ss->hist[p][d];
    if ((uint64_t)c == m) atomicOr(&s_skip, 1u << p);
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    uint32_t base = 0;
    for (int w = 0; w < wid; ++w) base += s_w[w];
    ss->off[p][d] = base + inc - c;
    __syncthreads();
  }
  if (d == 0) {
    const uint32_t sk = s_skip;
    ss->skip = sk;
    ss->cur[0] = 0;
    for (int p = 0; p < passes; ++p) {
      ss->cur[p + 1] = ((sk >> p) & 1u) ? ss->cur[p] : ss->cur[p] ^ 1;
      ss->ticket[p] = 0;
    }
  }
}

// Look-back words: flag in the top two bits, a count below.
constexpr uint64_t LB_AGG = 1ull << 62, LB_PREFIX = 2ull << 62, LB_COUNT = (1ull << 62) - 1;
constexpr uint32_t LB_SPIN_LIMIT = 1u << 20;  // then the pass gives up and reports a timeout
constexpr int LB_WINDOW = 8;                  // predecessors read per look-back round trip

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// ---- one radix pass: tiles of 4096 keys taken in ticket order, ranked in the
// block, global offsets from the digits' start plus the counts of the earlier
// tiles (decoupled look-back), written out digit run by digit run ----
// Warp w of the block owns the contiguous segment [w * 512, (w + 1) * 512) of
// the tile and ranks its keys stably with a warp-private counter per digit
// (warp match + leader update). The tile is then staged in shared memory in
// digit order, and each digit's run is written with consecutive threads
// writing consecutive addresses.
constexpr int DS_WARPS = SORT_THREADS / 32;
constexpr int DS_SEG = SORT_TILE / DS_WARPS;  // 512 keys per warp
constexpr size_t DS_DYN_SMEM = SORT_TILE * (sizeof(uint64_t) + sizeof(uint32_t));

__global__ void __launch_bounds__(SORT_THREADS) radix_pass_kernel(
    uint64_t *keys0, uint32_t *vals0, uint64_t *keys1, uint32_t *vals1, const uint64_t *d_pairs,
    uint64_t cap, int shift, int pass, SortState *ss, uint64_t *lookback, int32_t *status,
    int32_t withhold) {
  if ((ss->skip >> pass) & 1u) return;  // block-uniform
  extern __shared__ __align__(16) unsigned char ds_smem[];
  uint64_t *s_keys = reinterpret_cast<uint64_t *>(ds_smem);
  uint32_t *s_vals = reinterpret_cast<uint32_t *>(ds_smem + SORT_TILE * sizeof(uint64_t));
  __shared__ uint32_t s_cnt[DS_WARPS][RADIX];  // per-warp digit counts, then bases
  __shared__ uint32_t s_glob[RADIX];           // global position of the tile's digit run - local start
  __shared__ uint32_t s_wsum[DS_WARPS];
  __shared__ uint32_t s_hist[RADIX];           // the tile's digit counts, published early
  __shared__ uint32_t s_tile;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(&ss->ticket[pass], 1u);
  for (int d = lane; d < RADIX; d += 32) s_cnt[wid][d] = 0;
  s_hist[tid] = 0;  // SORT_THREADS == RADIX
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t m = pair_count(d_pairs, cap);
  const uint64_t start = (uint64_t)tile * SORT_TILE;
  if (start >= m) return;  // block-uniform
  const int count = (int)min((uint64_t)SORT_TILE, m - start);
  const bool from1 = ss->cur[pass] != 0;
  const uint64_t *keys_in = from1 ? keys1 : keys0;
  const uint32_t *vals_in = from1 ? vals1 : vals0;
  uint64_t *keys_out = from1 ? keys0 : keys1;
  uint32_t *vals_out = from1 ? vals0 : vals1;
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint64_t key[SORT_ITEMS];
  uint32_t val[SORT_ITEMS], rank[SORT_ITEMS];
  // issue every load of the thread before ranking
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; ++r) {
    const int li = wid * DS_SEG + r * 32 + lane;  // position in the tile
    const bool ok = li < count;
    key[r] = ok ? keys_in[start + li] : 0;
    val[r] = ok ? vals_in[start + li] : 0;
  }
  // the tile's digit counts go out before the (slower) stable ranking, so that
  // later tiles waiting in their look-back are released early
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; ++r)
    if (wid * DS_SEG + r * 32 + lane < count) atomicAdd(&s_hist[(key[r] >> shift) & (RADIX - 1)], 1u);
  __syncthreads();
  uint64_t *mine = lookback + (uint64_t)tile * RADIX + tid;
  const bool publish = (int64_t)tile != (int64_t)withhold;  // test hook: withhold = -1
  if (publish)
    atomicExch(reinterpret_cast<unsigned long long *>(mine), (tile == 0 ? LB_PREFIX : LB_AGG) | s_hist[tid]);
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; ++r) {
    const int li = wid * DS_SEG + r * 32 + lane;
    const bool ok = li < count;
    const uint32_t digit = ok ? (uint32_t)((key[r] >> shift) & (RADIX - 1)) : RADIX;
    const uint32_t peers = __match_any_sync(0xffffffffu, digit);
    const int leader = __ffs(peers) - 1;
    uint32_t before = 0;
    if (ok && lane == leader) {
      before = s_cnt[wid][digit];
      s_cnt[wid][digit] = before + __popc(peers);
    }
    before = __shfl_sync(0xffffffffu, before, leader);
    rank[r] = before + __popc(peers & lt_mask);
    __syncwarp();
  }
  __syncthreads();
  // per digit d (thread d): bases of each warp's run; the look-back sums the
  // earlier tiles' counts
  const int d = tid;  // SORT_THREADS == RADIX
  uint32_t run = 0;
#pragma unroll
  for (int w = 0; w < DS_WARPS; ++w) {
    const uint32_t c = s_cnt[w][d];
    s_cnt[w][d] = run;
    run += c;
  }
  uint64_t excl = 0;
  if (tile > 0) {
    // read LB_WINDOW predecessors per round trip, newest first; stop at the
    // first inclusive prefix, wait at the first tile that has not published
    int64_t j = (int64_t)tile - 1;
    uint32_t spins = 0;
    bool found = false;
    while (!found && j >= 0) {
      uint64_t w[LB_WINDOW];
#pragma unroll
      for (int k = 0; k < LB_WINDOW; ++k)
        w[k] = j - k >= 0 ? ld_relaxed(lookback + (uint64_t)(j - k) * RADIX + d) : 0ull;
      int used = 0;
#pragma unroll
      for (int k = 0; k < LB_WINDOW; ++k) {
        if (found || used < k || j - k < 0) continue;
        if ((w[k] >> 62) == 0) continue;  // not published yet: resume here
        excl += w[k] & LB_COUNT;
        ++used;
        if ((w[k] & ~LB_COUNT) == LB_PREFIX) found = true;
      }
      j -= used;
      if (!found && used < LB_WINDOW && j >= 0) {
        if (++spins > LB_SPIN_LIMIT) {
          atomicOr(status, ST_TIMEOUT);
          break;
        }
        __nanosleep(32);
      }
    }
    if (publish) atomicExch(reinterpret_cast<unsigned long long *>(mine), LB_PREFIX | (excl + run));
  }
  uint32_t inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_wsum[wid] = inc;
  __syncthreads();
  uint32_t wbase = 0;
#pragma unroll
  for (int w = 0; w < DS_WARPS; ++w) wbase += (w < wid) ? s_wsum[w] : 0u;
  const uint32_t pref = wbase + inc - run;  // first local position of digit d
#pragma unroll
  for (int w = 0; w < DS_WARPS; ++w) s_cnt[w][d] += pref;
  s_glob[d] = ss->off[pass][d] + (uint32_t)excl - pref;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; ++r) {
    const int li = wid * DS_SEG + r * 32 + lane;
    if (li < count) {
      const uint32_t digit = (uint32_t)((key[r] >> shift) & (RADIX - 1));
      const uint32_t pos = s_cnt[wid][digit] + rank[r];
      s_keys[pos] = key[r];
      s_vals[pos] = val[r];
    }
  }
  __syncthreads();
  for (int p = tid; p < count; p += SORT_THREADS) {
    const uint64_t k = s_keys[p];
    const uint32_t digit = (uint32_t)((k >> shift) & (RADIX - 1));
    const uint32_t o = s_glob[digit] + (uint32_t)p;
    if (o < m) {  // always, unless a look-back gave up
      keys_out[o] = k;
      vals_out[o] = s_vals[p];
    }
  }
}

// Tiles outside [0, n_tiles) can only come from a capacity overflow (stale
// keys); they are ignored so that the render stays memory-safe.
__global__ void tile_ranges_kernel(const uint64_t *keys0, const uint64_t *keys1,
                                   const int32_t *sorted, const uint64_t *d_pairs, uint64_t cap,
                                   uint2 *ranges, uint64_t n_tiles) {
  const uint64_t *keys = *sorted ? keys1 : keys0;
  const uint64_t m = pair_count(d_pairs, cap);
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m;
       j += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t t = (uint32_t)(keys[j] >> 32);
    if (t >= n_tiles) continue;
    if (j == 0 || (uint32_t)(keys[j - 1] >> 32) != t) ranges[t].x = (uint32_t)j;
    if (j + 1 == m || (uint32_t)(keys[j + 1] >> 32) != t) ranges[t].y = (uint32_t)(j + 1);
  }
}

}  // namespace

void launch_scan_blocks(int64_t nblk, ddgs_workspace &ws, cudaStream_t st) {
  LaunchScope ls(KID_SCAN_BLOCKS, st);
  scan_blocks_kernel<<<1, 1024, 0, st>>>(ws.blk_total, ws.blk_offset, nblk, ws.d_pairs, nullptr);
}

int64_t sort_blocks(uint64_t pair_bound) {
  return (int64_t)((pair_bound + SORT_TILE - 1) / SORT_TILE);
}

cudaError_t prepare_sort_kernels() {
  // the pass kernel stages a 4096-key tile (48 KiB) and the prepass keeps
  // warp-private histograms of up to 8 passes (64 KiB) in dynamic shared
  // memory; the attributes are set once per device, outside any stream capture
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(radix_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)DS_DYN_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(radix_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(MAX_SORT_PASSES * (SORT_THREADS / 32) * RADIX * sizeof(uint32_t)));
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

void launch_radix_sort(const RenderShape &s, uint64_t pair_bound, ddgs_workspace &ws,
                       cudaStream_t st) {
  const int64_t nblk = sort_blocks(pair_bound);
  if (nblk > 0 && prepare_sort_kernels() != cudaSuccess) return;  // surfaces via cudaGetLastError
  // keys in buffer 0 until the plan says otherwise; histograms start at zero
  cudaMemsetAsync(ws.sort_state, 0, sizeof(SortState), st);
  ws.sort_passes = 0;
  if (nblk == 0) return;
  const int passes = (s.key_bits + RADIX_BITS - 1) / RADIX_BITS;
  {
    LaunchScope ls(KID_RADIX_HIST, st);
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nblk, 152 * 3));
    radix_hist_kernel<<<g, SORT_THREADS, passes * (SORT_THREADS / 32) * RADIX * sizeof(uint32_t), st>>>(
        ws.keys[0], ws.d_pairs, (uint64_t)ws.pair_cap, passes, ws.sort_state);
  }
  {
    LaunchScope ls(KID_RADIX_PLAN, st);
    radix_plan_kernel<<<1, RADIX, 0, st>>>(ws.sort_state, ws.d_pairs, (uint64_t)ws.pair_cap, passes);
  }
  for (int p = 0; p < passes; ++p) {
    cudaMemsetAsync(ws.lookback, 0, (size_t)nblk * RADIX * sizeof(uint64_t), st);
    LaunchScope ls(KID_RADIX_PASS, st);
    radix_pass_kernel<<<(unsigned)nblk, SORT_THREADS, DS_DYN_SMEM, st>>>(
        ws.keys[0], ws.vals[0], ws.keys[1], ws.vals[1], ws.d_pairs, (uint64_t)ws.pair_cap,
        p * RADIX_BITS, p, ws.sort_state, ws.lookback, ws.d_status, ws.debug_withhold_tile);
  }
  ws.sort_passes = passes;
}

void launch_tile_ranges(const RenderShape &s, uint64_t pair_bound, ddgs_workspace &ws,
                        cudaStream_t st) {
  cudaMemsetAsync(ws.ranges, 0, (size_t)s.total_tiles * sizeof(uint2), st);
  if (pair_bound == 0) return;
  int64_t blocks = (int64_t)((pair_bound + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  LaunchScope ls(KID_TILE_RANGES, st);
  tile_ranges_kernel<<<(unsigned)blocks, 256, 0, st>>>(
      ws.keys[0], ws.keys[1], ws.sort_state->cur + ws.sort_passes, ws.d_pairs, (uint64_t)ws.pair_cap,
      ws.ranges, (uint64_t)s.total_tiles);
}

}  // namespace ddgs
