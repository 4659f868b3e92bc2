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
// Each pass: (1) upsweep -- every block histograms the 8-bit digit of its
// tile of 4096 keys and adds the histogram to per-digit totals; (2) scan --
// one block per digit turns the per-block counts into global output offsets;
// (3) downsweep -- every block ranks its keys stably within the tile (warp
// match + per-warp digit counters) and scatters keys and values. No block
// waits on another, so no spin-waits are needed.
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

__global__ void __launch_bounds__(SORT_THREADS) radix_upsweep_kernel(
    const uint64_t *keys, const uint64_t *d_pairs, uint64_t cap, int shift, uint32_t *hist,
    uint32_t *digit_total, int64_t nblk) {
  __shared__ uint32_t s_hist[SORT_THREADS / 32][RADIX];
  const int tid = threadIdx.x, wid = tid >> 5;
  for (int d = tid; d < (SORT_THREADS / 32) * RADIX; d += SORT_THREADS) (&s_hist[0][0])[d] = 0;
  __syncthreads();
  const uint64_t m = pair_count(d_pairs, cap);
  const uint64_t start = (uint64_t)blockIdx.x * SORT_TILE;
#pragma unroll 4
  for (int k = 0; k < SORT_ITEMS; ++k) {
    const uint64_t j = start + (uint64_t)k * SORT_THREADS + tid;
    if (j < m) atomicAdd(&s_hist[wid][(keys[j] >> shift) & (RADIX - 1)], 1u);
  }
  __syncthreads();
  for (int d = tid; d < RADIX; d += SORT_THREADS) {
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < SORT_THREADS / 32; ++w) c += s_hist[w][d];
    hist[(int64_t)d * nblk + blockIdx.x] = c;
    if (c) atomicAdd(&digit_total[d], c);
  }
}

// One block per digit: offsets[d][b] = (keys of smaller digits) + (keys of
// digit d in blocks before b).
__global__ void __launch_bounds__(1024) radix_scan_kernel(uint32_t *hist, const uint32_t *digit_total,
                                                          int64_t nblk) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) {
    uint32_t b = 0;
    for (int e = 0; e < d; ++e) b += digit_total[e];
    s_carry = b;
  }
  __syncthreads();
  uint32_t *h = hist + (int64_t)d * nblk;
  for (int64_t base = 0; base < nblk; base += 1024) {
    const int64_t j = base + tid;
    const uint32_t x = j < nblk ? h[j] : 0;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      uint32_t w = s_warp[lane], wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      s_warp[lane] = wi - w;
    }
    __syncthreads();
    const uint32_t ex = s_carry + s_warp[wid] + inc - x;
    if (j < nblk) h[j] = ex;
    __syncthreads();
    if (tid == 1023) s_carry = ex + x;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SORT_THREADS) radix_downsweep_kernel(
    const uint64_t *keys_in, const uint32_t *vals_in, uint64_t *keys_out, uint32_t *vals_out,
    const uint64_t *d_pairs, uint64_t cap, int shift, const uint32_t *offsets, int64_t nblk) {
  constexpr int NW = SORT_THREADS / 32;
  __shared__ uint32_t s_base[RADIX];     // running output position per digit
  __shared__ uint32_t s_cnt[NW][RADIX];  // per-warp counts of the current round
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint64_t m = pair_count(d_pairs, cap);
  const uint64_t start = (uint64_t)blockIdx.x * SORT_TILE;
  if (start >= m) return;
  for (int d = tid; d < RADIX; d += SORT_THREADS) s_base[d] = offsets[(int64_t)d * nblk + blockIdx.x];
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int k = 0; k < SORT_ITEMS; ++k) {
    const uint64_t j = start + (uint64_t)k * SORT_THREADS + tid;
    const bool ok = j < m;
    uint64_t key = 0;
    uint32_t val = 0;
    if (ok) { key = keys_in[j]; val = vals_in[j]; }
    const uint32_t digit = ok ? (uint32_t)((key >> shift) & (RADIX - 1)) : RADIX;  // RADIX: none
    for (int d = lane; d < RADIX; d += 32) s_cnt[wid][d] = 0;
    __syncthreads();  // s_base ready (first round), s_cnt cleared
    const uint32_t peers = __match_any_sync(0xffffffffu, digit);
    const uint32_t rank_in_warp = __popc(peers & lt_mask);
    const bool leader = (peers & lt_mask) == 0;
    if (ok && leader) s_cnt[wid][digit] = __popc(peers);
    __syncthreads();
    // per digit: exclusive prefix over warps, starting at the running base
    for (int d = tid; d < RADIX; d += SORT_THREADS) {
      uint32_t run = s_base[d];
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        uint32_t c = s_cnt[w][d];
        s_cnt[w][d] = run;
        run += c;
      }
      s_base[d] = run;
    }
    __syncthreads();
    if (ok) {
      const uint32_t pos = s_cnt[wid][digit] + rank_in_warp;
      keys_out[pos] = key;
      vals_out[pos] = val;
    }
    __syncthreads();
  }
}

// K5: [start, end) of every global tile's list.
// Tiles outside [0, n_tiles) can only come from a capacity overflow (stale
// keys); they are ignored so that the render stays memory-safe.
__global__ void tile_ranges_kernel(const uint64_t *keys, const uint64_t *d_pairs, uint64_t cap,
                                   uint2 *ranges, uint64_t n_tiles) {
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

void launch_radix_sort(const RenderShape &s, uint64_t pair_bound, ddgs_workspace &ws,
                       cudaStream_t st) {
  const int64_t nblk = sort_blocks(pair_bound);
  int cur = 0;
  if (nblk > 0) {
    const int passes = (s.key_bits + RADIX_BITS - 1) / RADIX_BITS;
    for (int p = 0; p < passes; ++p) {
      const int shift = p * RADIX_BITS;
      cudaMemsetAsync(ws.digit_total, 0, RADIX * sizeof(uint32_t), st);
      {
        LaunchScope ls(KID_RADIX_UPSWEEP, st);
        radix_upsweep_kernel<<<(unsigned)nblk, SORT_THREADS, 0, st>>>(
            ws.keys[cur], ws.d_pairs, (uint64_t)ws.pair_cap, shift, ws.hist, ws.digit_total, nblk);
      }
      {
        LaunchScope ls(KID_RADIX_SCAN, st);
        radix_scan_kernel<<<RADIX, 1024, 0, st>>>(ws.hist, ws.digit_total, nblk);
      }
      {
        LaunchScope ls(KID_RADIX_DOWNSWEEP, st);
        radix_downsweep_kernel<<<(unsigned)nblk, SORT_THREADS, 0, st>>>(
            ws.keys[cur], ws.vals[cur], ws.keys[cur ^ 1], ws.vals[cur ^ 1], ws.d_pairs,
            (uint64_t)ws.pair_cap, shift, ws.hist, nblk);
      }
      cur ^= 1;
    }
  }
  ws.sorted = cur;
}

void launch_tile_ranges(const RenderShape &s, uint64_t pair_bound, ddgs_workspace &ws,
                        cudaStream_t st) {
  cudaMemsetAsync(ws.ranges, 0, (size_t)s.total_tiles * sizeof(uint2), st);
  if (pair_bound == 0) return;
  int64_t blocks = (int64_t)((pair_bound + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  LaunchScope ls(KID_TILE_RANGES, st);
  tile_ranges_kernel<<<(unsigned)blocks, 256, 0, st>>>(ws.keys[ws.sorted], ws.d_pairs,
                                                       (uint64_t)ws.pair_cap, ws.ranges,
                                                       (uint64_t)s.total_tiles);
}

}  // namespace ddgs
