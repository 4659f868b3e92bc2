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

__global__ void __launch_bounds__(SORT_THREADS) radix_upsweep_kernel(
    const uint64_t *keys0, const uint64_t *keys1, const uint64_t *d_pairs, uint64_t cap, int shift,
    int pass, SortState *ss, uint32_t *hist, uint32_t *digit_total, int64_t nblk) {
  __shared__ uint32_t s_hist[SORT_THREADS / 32][RADIX];
  const int tid = threadIdx.x, wid = tid >> 5;
  if (pass > 0 && ((ss->skip >> pass) & 1u)) return;  // block-uniform
  const uint64_t *keys = ss->cur[pass] ? keys1 : keys0;
  for (int d = tid; d < (SORT_THREADS / 32) * RADIX; d += SORT_THREADS) (&s_hist[0][0])[d] = 0;
  const uint64_t m = pair_count(d_pairs, cap);
  const uint64_t start = (uint64_t)blockIdx.x * SORT_TILE;
  // all of the thread's loads first (two keys per 16-byte load), then count
  uint64_t k[SORT_ITEMS];
  const bool full = start + SORT_TILE <= m;
  if (full) {
    const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(keys + start);
#pragma unroll
    for (int r = 0; r < SORT_ITEMS / 2; ++r) {
      const ulonglong2 v = p[r * SORT_THREADS + tid];
      k[2 * r] = v.x;
      k[2 * r + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int r = 0; r < SORT_ITEMS / 2; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint64_t j = start + 2 * ((uint64_t)r * SORT_THREADS + tid) + h;
        k[2 * r + h] = j < m ? keys[j] : ~0ull;
      }
  }
  __syncthreads();
  unsigned long long k_and = ~0ull, k_or = 0ull;
#pragma unroll
  for (int r = 0; r < SORT_ITEMS; ++r) {
    const uint64_t j = start + 2 * ((uint64_t)(r >> 1) * SORT_THREADS + tid) + (r & 1);
    if (j < m) {
      atomicAdd(&s_hist[wid][(k[r] >> shift) & (RADIX - 1)], 1u);
      k_and &= k[r];
      k_or |= k[r];
    }
  }
  if (pass == 0) {  // the bits that differ between keys decide which passes can be skipped
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      k_and &= __shfl_xor_sync(0xffffffffu, k_and, o);
      k_or |= __shfl_xor_sync(0xffffffffu, k_or, o);
    }
    if ((tid & 31) == 0) {
      atomicAnd(&ss->key_and, k_and);
      atomicOr(&ss->key_or, k_or);
    }
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
// Also decides whether the pass is skipped and which buffer the next pass reads.
__global__ void __launch_bounds__(1024) radix_scan_kernel(uint32_t *hist, const uint32_t *digit_total,
                                                          int64_t nblk, SortState *ss, int pass,
                                                          int passes) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  uint32_t sk;
  if (pass == 0) {  // the AND / OR of every key are complete: a digit that no key varies in
    const unsigned long long diff = ss->key_and ^ ss->key_or;
    sk = 0;
    for (int p = 0; p < passes; ++p)
      if (((diff >> (p * RADIX_BITS)) & (RADIX - 1)) == 0) sk |= 1u << p;
  } else {
    sk = ss->skip;
  }
  const bool skip = (sk >> pass) & 1u;
  if (d == 0 && tid == 0) {
    if (pass == 0) ss->skip = sk;
    ss->cur[pass + 1] = skip ? ss->cur[pass] : ss->cur[pass] ^ 1;
  }
  if (skip) return;  // block-uniform
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

// Downsweep. Warp w of the block owns the contiguous segment
// [w * 512, (w + 1) * 512) of the block's tile of 4096 keys and ranks its keys
// stably with a warp-private counter per digit (warp match + leader update),
// so the tile needs only a few block barriers. The tile is then staged in
// shared memory in digit order and each digit's run is written out with
// consecutive threads writing consecutive addresses.
constexpr int DS_WARPS = SORT_THREADS / 32;
constexpr int DS_SEG = SORT_TILE / DS_WARPS;  // 512 keys per warp
constexpr size_t DS_DYN_SMEM = SORT_TILE * (sizeof(uint64_t) + sizeof(uint32_t));

__global__ void __launch_bounds__(SORT_THREADS) radix_downsweep_kernel(
    uint64_t *keys0, uint32_t *vals0, uint64_t *keys1, uint32_t *vals1, const uint64_t *d_pairs,
    uint64_t cap, int shift, int pass, const SortState *ss, const uint32_t *offsets, int64_t nblk) {
  if ((ss->skip >> pass) & 1u) return;  // block-uniform
  const bool from1 = ss->cur[pass] != 0;
  const uint64_t *keys_in = from1 ? keys1 : keys0;
  const uint32_t *vals_in = from1 ? vals1 : vals0;
  uint64_t *keys_out = from1 ? keys0 : keys1;
  uint32_t *vals_out = from1 ? vals0 : vals1;
  extern __shared__ __align__(16) unsigned char ds_smem[];
  uint64_t *s_keys = reinterpret_cast<uint64_t *>(ds_smem);
  uint32_t *s_vals = reinterpret_cast<uint32_t *>(ds_smem + SORT_TILE * sizeof(uint64_t));
  __shared__ uint32_t s_cnt[DS_WARPS][RADIX];  // per-warp digit counts, then bases
  __shared__ uint32_t s_glob[RADIX];           // global position of the tile's digit run - local start
  __shared__ uint32_t s_wsum[DS_WARPS];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint64_t m = pair_count(d_pairs, cap);
  const uint64_t start = (uint64_t)blockIdx.x * SORT_TILE;
  if (start >= m) return;
  const int count = (int)min((uint64_t)SORT_TILE, m - start);
  for (int d = lane; d < RADIX; d += 32) s_cnt[wid][d] = 0;
  __syncwarp();
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
  // per digit d (thread d): bases of each warp's run, digit total, and the
  // exclusive prefix of the totals over digits
  {
    const int d = tid;  // SORT_THREADS == RADIX
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < DS_WARPS; ++w) {
      const uint32_t c = s_cnt[w][d];
      s_cnt[w][d] = run;
      run += c;
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
    s_glob[d] = offsets[(int64_t)d * nblk + blockIdx.x] - pref;
  }
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
    keys_out[o] = k;
    vals_out[o] = s_vals[p];
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
  // the downsweep stages a 4096-key tile (48 KiB) in dynamic shared memory;
  // the attribute is set once per device, outside any stream capture
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(radix_downsweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)DS_DYN_SMEM);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

void launch_radix_sort(const RenderShape &s, uint64_t pair_bound, ddgs_workspace &ws,
                       cudaStream_t st) {
  const int64_t nblk = sort_blocks(pair_bound);
  if (nblk > 0 && prepare_sort_kernels() != cudaSuccess) return;  // surfaces via cudaGetLastError
  // state: key AND = all ones, key OR = 0, nothing skipped, keys in buffer 0
  cudaMemsetAsync(ws.sort_state, 0, sizeof(SortState), st);
  cudaMemsetAsync(&ws.sort_state->key_and, 0xff, sizeof(unsigned long long), st);
  ws.sort_passes = 0;
  if (nblk > 0) {
    const int passes = (s.key_bits + RADIX_BITS - 1) / RADIX_BITS;
    for (int p = 0; p < passes; ++p) {
      const int shift = p * RADIX_BITS;
      cudaMemsetAsync(ws.digit_total, 0, RADIX * sizeof(uint32_t), st);
      {
        LaunchScope ls(KID_RADIX_UPSWEEP, st);
        radix_upsweep_kernel<<<(unsigned)nblk, SORT_THREADS, 0, st>>>(
            ws.keys[0], ws.keys[1], ws.d_pairs, (uint64_t)ws.pair_cap, shift, p, ws.sort_state,
            ws.hist, ws.digit_total, nblk);
      }
      {
        LaunchScope ls(KID_RADIX_SCAN, st);
        radix_scan_kernel<<<RADIX, 1024, 0, st>>>(ws.hist, ws.digit_total, nblk, ws.sort_state, p,
                                                  passes);
      }
      {
        LaunchScope ls(KID_RADIX_DOWNSWEEP, st);
        radix_downsweep_kernel<<<(unsigned)nblk, SORT_THREADS, DS_DYN_SMEM, st>>>(
            ws.keys[0], ws.vals[0], ws.keys[1], ws.vals[1], ws.d_pairs, (uint64_t)ws.pair_cap,
            shift, p, ws.sort_state, ws.hist, nblk);
      }
    }
    ws.sort_passes = passes;
  }
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
