// rads.cu -- radiodensity-aware dual sampling (RADS, Sec. 3.3): the initial
// point cloud of a DDGS model from a CT volume.
//
//   P^mc  marching-cubes points of the isolevel (min + max) / 2 (Sec. 4.1):
//         one point on every grid edge whose two end voxels lie on opposite
//         sides of it, at the linear interpolation along the edge; n1 of them
//         kept uniformly without replacement (the n1 smallest counter-based
//         keys), in edge order.
//   P^dw  n2 voxel centres drawn with probability proportional to HU - min.
//   Scales: the 3D Gaussian splatting default, the root mean squared distance
//         to the 3 nearest other points.
//
// Every pass over the volume is a memory-bound sweep: blocks own chunks of
// 4096 consecutive voxels; a warp walks 512 of them lane-interleaved (voxel
// base + 32 i + lane), so each load of the voxel and of its +x/+y/+z
// neighbours is one coalesced 64-byte request, and the per-warp crossing
// order is the global edge order. The crossing list is sized by one host
// synchronisation; the n1-th smallest key is found by an 8-pass radix select
// (8 bits a pass) and the kept crossings are compacted in order.
#include <algorithm>
#include <climits>

#include "ddgs_internal.cuh"

namespace ddgs {
namespace {

constexpr int RT = 256;         // threads per block of the sweeps
constexpr int RI = 16;          // voxels (keys) per lane
constexpr int RCH = RT * RI;    // voxels (keys) per block: 4096
constexpr int SUB = 32 * RI;    // voxels per warp (sub-chunk): 512
constexpr int NSUB = RT / 32;   // sub-chunks per chunk
constexpr int KNN_T = 128;      // threads per block of the neighbour search
constexpr int KNN_Q = 2;        // queries per thread
constexpr int SEL_BINS = 2048;  // radix select: 11-bit digits

// Output number i + 1 of SplitMix64 (Steele, Lea and Flood, OOPSLA 2014)
// seeded with `seed`: the state after i + 1 golden-gamma steps, finalised.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct RadsState {
  int32_t hu_min, hu_max;
  uint64_t prefix;   // radix select: the wanted key's digits found so far
  uint64_t rank;     // its rank among the keys sharing that prefix
  uint32_t done;     // blocks finished in the current select pass
  uint32_t hist[SEL_BINS];
};

struct Vol {
  const int16_t *hu;
  int32_t nx, ny, nz;
  int64_t nvox;
  float sx, sy, sz, ox, oy, oz;
};

__device__ __forceinline__ int warp_min(int x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}
__device__ __forceinline__ int warp_max(int x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}
template <class Tv>
__device__ __forceinline__ Tv warp_sum(Tv x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
template <class Tv>
__device__ __forceinline__ Tv warp_incl_scan(Tv x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const Tv y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// ---- pass 1: min and max of the volume ----
__global__ void __launch_bounds__(RT) rads_minmax_kernel(Vol v, RadsState *st) {
  int lo = INT_MAX, hi = INT_MIN;
  const int64_t n8 = v.nvox / 8, stride = (int64_t)gridDim.x * blockDim.x;
  const uint4 *p = reinterpret_cast<const uint4 *>(v.hu);  // 8 voxels, little-endian
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += stride) {
    const uint4 q = p[i];
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int a = (int)(int16_t)(w[k] & 0xffffu), b = (int)(int16_t)(w[k] >> 16);
      lo = min(lo, min(a, b));
      hi = max(hi, max(a, b));
    }
  }
  for (int64_t i = n8 * 8 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < v.nvox; i += stride) {
    const int a = v.hu[i];
    lo = min(lo, a);
    hi = max(hi, a);
  }
  lo = warp_min(lo);
  hi = warp_max(hi);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&st->hu_min, lo);
    atomicMax(&st->hu_max, hi);
  }
}

// Lane-interleaved walk of one warp's 512 voxels: voxel c0 + 32 i + lane.
struct VoxelWalk {
  int64_t v;
  int32_t x, y, z;
  __device__ __forceinline__ VoxelWalk(const Vol &vol, int64_t first) : v(first) {
    const int64_t plane = (int64_t)vol.nx * vol.ny;
    z = (int32_t)(first / plane);
    const int64_t r = first - (int64_t)z * plane;
    y = (int32_t)(r / vol.nx);
    x = (int32_t)(r - (int64_t)y * vol.nx);
  }
  __device__ __forceinline__ void advance(const Vol &vol) {
    v += 32;
    x += 32;
    while (x >= vol.nx) {
      x -= vol.nx;
      if (++y == vol.ny) { y = 0; ++z; }
    }
  }
};

// Crossing edges (bit a = edge to the +a neighbour) of a voxel inside the
// volume; a voxel is above the isolevel when 2 HU > lam2 = min + max.
__device__ __forceinline__ uint32_t crossing_bits(const Vol &vol, const VoxelWalk &w, int lam2,
                                                  int &hu) {
  hu = vol.hu[w.v];
  const bool a = 2 * hu > lam2;
  uint32_t bits = 0;
  if (w.x + 1 < vol.nx) bits |= (uint32_t)((2 * (int)vol.hu[w.v + 1] > lam2) != a);
  if (w.y + 1 < vol.ny) bits |= (uint32_t)((2 * (int)vol.hu[w.v + vol.nx] > lam2) != a) << 1;
  if (w.z + 1 < vol.nz)
    bits |= (uint32_t)((2 * (int)vol.hu[w.v + (int64_t)vol.nx * vol.ny] > lam2) != a) << 2;
  return bits;
}

// 8 consecutive voxels of one row (rows are a multiple of 8 voxels on the
// vector path): int16 values from one 16-byte load, little-endian.
__device__ __forceinline__ void unpack8(const uint4 q, int h[8]) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    h[2 * k] = (int)(int16_t)(w[k] & 0xffffu);
    h[2 * k + 1] = (int)(int16_t)(w[k] >> 16);
  }
}

__device__ __forceinline__ uint32_t above_mask(const int h[8], int lam2) {
  uint32_t m = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) m |= (uint32_t)(2 * h[j] > lam2) << j;
  return m;
}

// Crossing bits of voxels v0 .. v0 + 7 (v0 a multiple of 8, nx a multiple of
// 8): bit 3 j + a for voxel j and axis a, so that the edge id is 3 v0 + bit.
// Adds the group's weights (HU - min) to wsum.
__device__ __forceinline__ uint32_t group_bits(const Vol &vol, int64_t v0, int lam2, int mn,
                                               uint64_t &wsum) {
  // voxel counts stay below 2^32 (edge ids fit 32 bits): 32-bit division
  const uint32_t plane = (uint32_t)vol.nx * (uint32_t)vol.ny, vv = (uint32_t)v0;
  const uint32_t z = vv / plane, r = vv - z * plane, y = r / (uint32_t)vol.nx,
                 x0 = r - y * (uint32_t)vol.nx;
  const uint4 *p = reinterpret_cast<const uint4 *>(vol.hu);
  int h[8];
  unpack8(p[v0 >> 3], h);
  uint32_t ws = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) ws += (uint32_t)(h[j] - mn);
  wsum += ws;
  const uint32_t ab = above_mask(h, lam2);
  uint32_t bx = (ab ^ (ab >> 1)) & 0x7fu, by = 0, bz = 0;
  if (x0 + 8 < (uint32_t)vol.nx) bx |= ((ab >> 7) ^ (uint32_t)(2 * (int)vol.hu[v0 + 8] > lam2)) << 7;
  int hn[8];
  if (y + 1 < (uint32_t)vol.ny) {
    unpack8(p[(v0 + vol.nx) >> 3], hn);
    by = ab ^ above_mask(hn, lam2);
  }
  if (z + 1 < (uint32_t)vol.nz) {
    unpack8(p[(v0 + plane) >> 3], hn);
    bz = ab ^ above_mask(hn, lam2);
  }
  uint32_t bits = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j)
    bits |= (((bx >> j) & 1u) << (3 * j)) | (((by >> j) & 1u) << (3 * j + 1)) |
            (((bz >> j) & 1u) << (3 * j + 2));
  return bits;
}

// ---- pass 2: crossings per chunk and weight per warp sub-chunk (512 voxels) ----
template <bool VEC>
__global__ void __launch_bounds__(RT) rads_count_kernel(Vol vol, const RadsState *st,
                                                        uint32_t *cnt, uint64_t *wsub,
                                                        uint64_t *wsum) {
  __shared__ uint32_t s_c[RT / 32];
  __shared__ uint64_t s_w[RT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int mn = st->hu_min, lam2 = st->hu_min + st->hu_max;
  const int64_t sub0 = (int64_t)blockIdx.x * RCH + wid * SUB;
  uint32_t c = 0;
  uint64_t ws = 0;
  if (VEC) {
#pragma unroll
    for (int i = 0; i < SUB / 256; ++i) {
      const int64_t v0 = sub0 + 256 * i + 8 * lane;
      if (v0 < vol.nvox) c += __popc(group_bits(vol, v0, lam2, mn, ws));
    }
  } else if (sub0 + lane < vol.nvox) {
    VoxelWalk w(vol, sub0 + lane);
    for (int i = 0; i < RI && w.v < vol.nvox; ++i, w.advance(vol)) {
      int hu;
      c += __popc(crossing_bits(vol, w, lam2, hu));
      ws += (uint64_t)(hu - mn);
    }
  }
  c = warp_sum(c);
  ws = warp_sum(ws);
  if (lane == 0) {
    s_c[wid] = c;
    s_w[wid] = ws;
    wsub[(int64_t)blockIdx.x * NSUB + wid] = ws;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tc = 0;
    uint64_t tw = 0;
    for (int k = 0; k < RT / 32; ++k) { tc += s_c[k]; tw += s_w[k]; }
    cnt[blockIdx.x] = tc;
    wsum[blockIdx.x] = tw;
  }
}

// ---- exclusive scans of per-chunk values over many blocks: a[] (uint32)
// and optionally b[] (uint64) into ao[0..n], bo[0..n] (ao[n], bo[n] = totals).
// Local scans of 1024 entries, a one-block scan of their totals, then the add.
constexpr int SCAN_T = 1024;

__device__ __forceinline__ uint64_t block_excl_scan64(uint64_t x, uint64_t *s_w, uint64_t &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint64_t inc = warp_incl_scan(x);
  __syncthreads();
  if (lane == 31) s_w[wid] = inc;
  __syncthreads();
  if (wid == 0) s_w[lane] = warp_incl_scan(lane < (int)(blockDim.x >> 5) ? s_w[lane] : 0ull);
  __syncthreads();
  total = s_w[(blockDim.x >> 5) - 1];
  return (wid ? s_w[wid - 1] : 0ull) + inc - x;
}

__global__ void __launch_bounds__(SCAN_T) rads_scan_local_kernel(const uint32_t *a, const uint64_t *b,
                                                                 int64_t n, uint64_t *ao, uint64_t *bo,
                                                                 uint64_t *tops) {
  __shared__ uint64_t s_w[32];
  const int64_t i = (int64_t)blockIdx.x * SCAN_T + threadIdx.x;
  uint64_t ta, tb;
  const uint64_t ea = block_excl_scan64(i < n ? (uint64_t)a[i] : 0ull, s_w, ta);
  if (i < n) ao[i] = ea;
  if (b) {
    const uint64_t eb = block_excl_scan64(i < n ? b[i] : 0ull, s_w, tb);
    if (i < n) bo[i] = eb;
  }
  if (threadIdx.x == 0) {
    tops[2 * blockIdx.x] = ta;
    tops[2 * blockIdx.x + 1] = b ? tb : 0ull;
  }
}

__global__ void __launch_bounds__(SCAN_T) rads_scan_tops_kernel(uint64_t *tops, int64_t nt, int64_t n,
                                                                uint64_t *ao, uint64_t *bo) {
  __shared__ uint64_t s_w[32];
  const int t = threadIdx.x;  // nt <= SCAN_T
  uint64_t ta, tb;
  const uint64_t xa = t < nt ? tops[2 * t] : 0ull, xb = t < nt ? tops[2 * t + 1] : 0ull;
  const uint64_t ea = block_excl_scan64(xa, s_w, ta);
  const uint64_t eb = block_excl_scan64(xb, s_w, tb);
  if (t < nt) {
    tops[2 * t] = ea;
    tops[2 * t + 1] = eb;
  }
  if (t == 0) {
    ao[n] = ta;
    if (bo) bo[n] = tb;
  }
}

__global__ void __launch_bounds__(SCAN_T) rads_scan_add_kernel(const uint64_t *tops, int64_t n,
                                                               uint64_t *ao, uint64_t *bo) {
  const int64_t i = (int64_t)blockIdx.x * SCAN_T + threadIdx.x;
  if (blockIdx.x == 0 || i >= n) return;
  ao[i] += tops[2 * blockIdx.x];
  if (bo) bo[i] += tops[2 * blockIdx.x + 1];
}

__device__ __forceinline__ uint64_t edge_key(uint64_t seed, uint64_t e) {
  return ((splitmix64(seed, e) >> 32) << 32) | e;
}

// ---- pass 3: the keys of every crossing, in edge order ----
template <bool VEC>
__global__ void __launch_bounds__(RT) rads_emit_kernel(Vol vol, const RadsState *st,
                                                       const uint64_t *coff, uint64_t seed,
                                                       uint64_t *keys, uint64_t cap) {
  __shared__ uint32_t s_c[RT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int mn = st->hu_min, lam2 = st->hu_min + st->hu_max;
  const int64_t sub0 = (int64_t)blockIdx.x * RCH + wid * SUB;
  constexpr int NIT = VEC ? SUB / 256 : RI;
  constexpr int BPI = VEC ? 24 : 3;  // crossing bits per lane and iteration
  uint32_t bits[NIT];
  uint32_t c = 0;
  uint64_t ws = 0;
#pragma unroll
  for (int i = 0; i < NIT; ++i) bits[i] = 0;
  if (VEC) {
#pragma unroll
    for (int i = 0; i < NIT; ++i) {
      const int64_t v0 = sub0 + 256 * i + 8 * lane;
      if (v0 < vol.nvox) {
        bits[i] = group_bits(vol, v0, lam2, mn, ws);
        c += __popc(bits[i]);
      }
    }
  } else if (sub0 + lane < vol.nvox) {
    VoxelWalk w(vol, sub0 + lane);
#pragma unroll
    for (int i = 0; i < NIT; ++i) {
      if (w.v < vol.nvox) {
        int hu;
        bits[i] = crossing_bits(vol, w, lam2, hu);
        c += __popc(bits[i]);
        w.advance(vol);
      }
    }
  }
  (void)BPI;
  const uint32_t wc = warp_sum(c);
  if (lane == 0) s_c[wid] = wc;
  __syncthreads();
  uint64_t run = coff[blockIdx.x];
  for (int k = 0; k < wid; ++k) run += s_c[k];
  if (wc == 0) return;  // warp-uniform: nothing for this warp to write
#pragma unroll
  for (int i = 0; i < NIT; ++i) {
    const uint32_t n = __popc(bits[i]);
    const uint32_t incl = warp_incl_scan(n);
    uint64_t o = run + (incl - n);
    // first edge id of this lane's voxels in iteration i: 3 v0 (+ bit index)
    const uint64_t e0 = VEC ? 3ull * (uint64_t)(sub0 + 256 * i + 8 * lane)
                            : 3ull * (uint64_t)(sub0 + 32 * i + lane);
    uint32_t b = bits[i];
    while (b) {
      const int k = __ffs(b) - 1;
      b &= b - 1;
      if (o < cap) keys[o] = edge_key(seed, e0 + (uint64_t)k);
      ++o;
    }
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
}

// ---- radix select of the rank-th smallest key: 11-bit digits from the top;
// the last block of each pass picks the digit ----
__global__ void rads_select_init_kernel(RadsState *st, uint64_t rank) {
  if (threadIdx.x == 0) {
    st->prefix = 0;
    st->rank = rank;
    st->done = 0;
  }
  for (int k = threadIdx.x; k < SEL_BINS; k += blockDim.x) st->hist[k] = 0;
}

__global__ void __launch_bounds__(RT) rads_select_pass_kernel(const uint64_t *keys, int64_t m,
                                                              RadsState *st, int shift,
                                                              int width) {
  __shared__ uint32_t h[SEL_BINS];
  __shared__ uint32_t s_sum[RT];
  __shared__ bool s_last;
  const int t = threadIdx.x;
  for (int k = t; k < SEL_BINS; k += RT) h[k] = 0;
  __syncthreads();
  const uint64_t mask = shift + width >= 64 ? 0ull : (~0ull << (shift + width));
  const uint64_t prefix = st->prefix;
  const uint32_t dmask = (1u << width) - 1u;
  for (int64_t i = (int64_t)blockIdx.x * RT + t; i < m; i += (int64_t)gridDim.x * RT) {
    const uint64_t k = keys[i];
    if ((k & mask) == prefix) atomicAdd(&h[(uint32_t)(k >> shift) & dmask], 1u);
  }
  __syncthreads();
  for (int k = t; k < SEL_BINS; k += RT)
    if (h[k]) atomicAdd(&st->hist[k], h[k]);
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(&st->done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the last block: the digit whose count interval holds the rank
  constexpr int PER = SEL_BINS / RT;  // 8 bins per thread
  uint32_t hv[PER], sum = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    hv[k] = __ldcg(&st->hist[t * PER + k]);
    sum += hv[k];
  }
  s_sum[t] = sum;
  const uint64_t rank = st->rank;
  __syncthreads();
  for (int o = 1; o < RT; o <<= 1) {
    const uint32_t y = t >= o ? s_sum[t - o] : 0u;
    __syncthreads();
    s_sum[t] += y;
    __syncthreads();
  }
  uint64_t excl = s_sum[t] - sum;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    if (hv[k] && excl <= rank && rank < excl + hv[k]) {
      st->prefix = prefix | ((uint64_t)(t * PER + k) << shift);
      st->rank = rank - excl;
    }
    excl += hv[k];
  }
  for (int k = 0; k < PER; ++k) st->hist[t * PER + k] = 0;
  if (t == 0) st->done = 0;
}

// ---- compaction of the kept crossings (key <= limit), in edge order ----
__global__ void __launch_bounds__(RT) rads_keep_count_kernel(const uint64_t *keys, int64_t m,
                                                             const RadsState *st, int all,
                                                             uint32_t *cnt) {
  __shared__ uint32_t s_c[RT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint64_t limit = all ? ~0ull : st->prefix;
  const int64_t first = (int64_t)blockIdx.x * RCH + wid * (32 * RI) + lane;
  uint32_t c = 0;
  for (int i = 0; i < RI; ++i) {
    const int64_t j = first + 32 * i;
    c += (j < m && keys[j] <= limit) ? 1u : 0u;
  }
  c = warp_sum(c);
  if (lane == 0) s_c[wid] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int k = 0; k < RT / 32; ++k) t += s_c[k];
    cnt[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(RT) rads_keep_emit_kernel(Vol vol, const uint64_t *keys,
                                                            int64_t m, const RadsState *st,
                                                            int all, const uint64_t *off,
                                                            int64_t n_out, float *means,
                                                            int64_t *kept_edges) {
  __shared__ uint32_t s_c[RT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint64_t limit = all ? ~0ull : st->prefix;
  const int lam2 = st->hu_min + st->hu_max;
  const int64_t first = (int64_t)blockIdx.x * RCH + wid * (32 * RI) + lane;
  uint32_t sel = 0;  // bit i: this lane's key of iteration i is kept
  for (int i = 0; i < RI; ++i) {
    const int64_t j = first + 32 * i;
    if (j < m && keys[j] <= limit) sel |= 1u << i;
  }
  const uint32_t wc = warp_sum((uint32_t)__popc(sel));
  if (lane == 0) s_c[wid] = wc;
  __syncthreads();
  uint64_t run = off[blockIdx.x];
  for (int k = 0; k < wid; ++k) run += s_c[k];
  const uint64_t plane = (uint64_t)vol.nx * vol.ny;
  for (int i = 0; i < RI; ++i) {
    const bool kept = (sel >> i) & 1u;
    const uint32_t bal = __ballot_sync(0xffffffffu, kept);
    if (kept) {
      const uint64_t o = run + __popc(bal & ((1u << lane) - 1u));
      if (o < (uint64_t)n_out) {
        const uint64_t e = keys[first + 32 * i] & 0xffffffffull;
        const uint64_t v = e / 3;
        const int axis = (int)(e - 3 * v);
        const uint64_t z = v / plane, r = v - z * plane, y = r / vol.nx, x = r - y * vol.nx;
        const uint64_t step = axis == 0 ? 1ull : (axis == 1 ? (uint64_t)vol.nx : plane);
        const float f0 = (float)vol.hu[v], f1 = (float)vol.hu[v + step];
        const float t = (0.5f * (float)lam2 - f0) / (f1 - f0);
        float c[3] = {(float)x, (float)y, (float)z};
        c[axis] += t;
        means[3 * o] = fmaf(vol.sx, c[0], vol.ox);
        means[3 * o + 1] = fmaf(vol.sy, c[1], vol.oy);
        means[3 * o + 2] = fmaf(vol.sz, c[2], vol.oz);
        if (kept_edges) kept_edges[o] = (int64_t)e;
      }
    }
    run += __popc(bal);
  }
}

// ---- P^dw: one warp per draw ----
template <bool VEC>
__global__ void __launch_bounds__(RT) rads_draw_kernel(Vol vol, const RadsState *st,
                                                       const uint64_t *woff, const uint64_t *wsub,
                                                       int64_t nblk, int32_t n2, uint64_t seed,
                                                       int64_t row0, float *means,
                                                       int64_t *draw_voxels) {
  const int lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * (RT / 32) + (threadIdx.x >> 5);
  if (j >= n2) return;  // warp-uniform
  const uint64_t total = woff[nblk];
  const uint64_t target = __umul64hi(splitmix64(~seed, (uint64_t)j), total);
  // the chunk whose weight interval [woff[c], woff[c+1]) holds the target
  int64_t lo = 0, hi = nblk;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (woff[mid] <= target) lo = mid; else hi = mid;
  }
  uint64_t rem = target - woff[lo];
  // then the warp sub-chunk (512 voxels) inside it
  const uint64_t wsl = lane < NSUB ? wsub[lo * NSUB + lane] : 0ull;
  const uint64_t winc = warp_incl_scan(wsl);
  const uint32_t sub_past = __ballot_sync(0xffffffffu, lane < NSUB && winc > rem);
  const int s = sub_past ? __ffs(sub_past) - 1 : NSUB - 1;
  rem -= __shfl_sync(0xffffffffu, winc - wsl, s);
  const int64_t sub0 = lo * RCH + (int64_t)s * SUB;
  const int mn = st->hu_min;
  uint64_t run = 0;
  int64_t found = -1;
  if (VEC) {
    const uint4 *p = reinterpret_cast<const uint4 *>(vol.hu);
    for (int i = 0; i < SUB / 256; ++i) {
      const int64_t v0 = sub0 + 256 * i + 8 * lane;
      int h[8];
      uint64_t wl = 0;
      if (v0 < vol.nvox) {
        unpack8(p[v0 >> 3], h);
#pragma unroll
        for (int k = 0; k < 8; ++k) wl += (uint64_t)(h[k] - mn);
      }
      const uint64_t incl = warp_incl_scan(wl);
      const uint32_t past = __ballot_sync(0xffffffffu, run + incl > rem);
      if (past) {
        const int L = __ffs(past) - 1;
        int64_t f = -1;
        if (lane == L) {
          uint64_t acc = run + incl - wl;
          for (int k = 0; k < 8; ++k) {
            acc += (uint64_t)(h[k] - mn);
            if (acc > rem) { f = v0 + k; break; }
          }
        }
        found = __shfl_sync(0xffffffffu, f, L);
        break;
      }
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
  } else {
    for (int i = 0; i < SUB / 32; ++i) {
      const int64_t v = sub0 + 32 * i + lane;
      const uint64_t w = v < vol.nvox ? (uint64_t)((int)vol.hu[v] - mn) : 0ull;
      const uint64_t incl = warp_incl_scan(w);
      const uint32_t past = __ballot_sync(0xffffffffu, run + incl > rem);
      if (past) {
        found = sub0 + 32 * i + (__ffs(past) - 1);
        break;
      }
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  if (lane != 0 || found < 0) return;  // found < 0 cannot happen while target < total
  const uint64_t plane = (uint64_t)vol.nx * vol.ny;
  const uint64_t z = (uint64_t)found / plane, r = (uint64_t)found - z * plane;
  const uint64_t y = r / vol.nx, x = r - y * vol.nx;
  const int64_t o = row0 + j;
  means[3 * o] = fmaf(vol.sx, (float)x, vol.ox);
  means[3 * o + 1] = fmaf(vol.sy, (float)y, vol.oy);
  means[3 * o + 2] = fmaf(vol.sz, (float)z, vol.oz);
  if (draw_voxels) draw_voxels[j] = found;
}

// ---- scales: the 3 nearest other points, candidates split over gridDim.y.
// Each thread serves KNN_Q queries; every list keeps the 4 smallest squared
// distances, the point itself included (it contributes exactly one 0, the
// smallest value), so no per-pair self test is needed: the merge drops it. ----
__device__ __forceinline__ void insert4(float d2, float &b0, float &b1, float &b2, float &b3) {
  if (d2 < b3) {
    if (d2 < b2) {
      b3 = b2;
      if (d2 < b1) {
        b2 = b1;
        if (d2 < b0) { b1 = b0; b0 = d2; } else { b1 = d2; }
      } else {
        b2 = d2;
      }
    } else {
      b3 = d2;
    }
  }
}

__global__ void __launch_bounds__(KNN_T) rads_knn_part_kernel(const float *means, int64_t n,
                                                              int64_t slice, float *part) {
  __shared__ float4 s_p[KNN_T];
  const float inf = __int_as_float(0x7f800000);
  const int64_t c0 = (int64_t)blockIdx.y * slice, c1 = min(n, c0 + slice);
  float q[KNN_Q][3], b[KNN_Q][4];
  int64_t qi[KNN_Q];
#pragma unroll
  for (int u = 0; u < KNN_Q; ++u) {
    qi[u] = (int64_t)blockIdx.x * (KNN_T * KNN_Q) + u * KNN_T + threadIdx.x;
    const bool ok = qi[u] < n;
    q[u][0] = ok ? means[3 * qi[u]] : 0.f;
    q[u][1] = ok ? means[3 * qi[u] + 1] : 0.f;
    q[u][2] = ok ? means[3 * qi[u] + 2] : 0.f;
    b[u][0] = b[u][1] = b[u][2] = b[u][3] = inf;
  }
  for (int64_t t0 = c0; t0 < c1; t0 += KNN_T) {
    __syncthreads();
    const int64_t jj = t0 + threadIdx.x;
    if (jj < c1) s_p[threadIdx.x] = make_float4(means[3 * jj], means[3 * jj + 1], means[3 * jj + 2], 0.f);
    __syncthreads();
    const int cnt = (int)min((int64_t)KNN_T, c1 - t0);
#pragma unroll 4
    for (int k = 0; k < cnt; ++k) {
      const float4 p = s_p[k];
#pragma unroll
      for (int u = 0; u < KNN_Q; ++u) {
        const float dx = p.x - q[u][0], dy = p.y - q[u][1], dz = p.z - q[u][2];
        insert4(fmaf(dz, dz, fmaf(dy, dy, dx * dx)), b[u][0], b[u][1], b[u][2], b[u][3]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < KNN_Q; ++u) {
    if (qi[u] >= n) continue;
    float4 *o = reinterpret_cast<float4 *>(part) + (int64_t)blockIdx.y * n + qi[u];
    *o = make_float4(b[u][0], b[u][1], b[u][2], b[u][3]);
  }
}

__global__ void rads_knn_merge_kernel(const float *part, int64_t n, int slices, float *log_scales) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float inf = __int_as_float(0x7f800000);
  float b0 = inf, b1 = inf, b2 = inf, b3 = inf;
  for (int s = 0; s < slices; ++s) {
    const float4 v = reinterpret_cast<const float4 *>(part)[(int64_t)s * n + i];
    insert4(v.x, b0, b1, b2, b3);
    insert4(v.y, b0, b1, b2, b3);
    insert4(v.z, b0, b1, b2, b3);
    insert4(v.w, b0, b1, b2, b3);
  }
  // b0 is the point itself (0); the others are the nearest other points
  const int kk = n - 1 < 3 ? (int)(n - 1) : 3;
  float m = 0.f;
  if (kk >= 1) m += b1;
  if (kk >= 2) m += b2;
  if (kk >= 3) m += b3;
  m = kk > 0 ? m / (float)kk : 0.f;
  const float ls = 0.5f * logf(fmaxf(m, 1e-7f));
  log_scales[3 * i] = ls;
  log_scales[3 * i + 1] = ls;
  log_scales[3 * i + 2] = ls;
}

}  // namespace
}  // namespace ddgs

#define RCK(call)                                                  \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return ddgs::cuda_status(e_, #call);    \
  } while (0)

namespace {

// Reallocate the workspace buffer p (a field of the workspace) for `need`
// bytes. Its capacity is zeroed first, so an allocation that fails leaves the
// buffer marked empty and the next call retries it.
template <class Tp>
ddgs_status grow_bytes(Tp *&p, int64_t &cap, int64_t need) {
  if (need <= cap && p) return DDGS_OK;
  cap = 0;
  if (p) RCK(cudaFree(p));
  p = nullptr;
  const int64_t c = need + need / 4 + 4096;
  RCK(cudaMalloc(reinterpret_cast<void **>(&p), (size_t)c));
  cap = c;
  return DDGS_OK;
}

int64_t align256(int64_t x) { return (x + 255) & ~int64_t(255); }

// Exclusive scans of n per-chunk values (a, and b if not null) with totals at
// [n]; n <= 1024 * 1024.
void scan_chunks(const uint32_t *a, const uint64_t *b, int64_t n, uint64_t *ao, uint64_t *bo,
                 uint64_t *tops, cudaStream_t st) {
  using namespace ddgs;
  const int64_t nt = (n + SCAN_T - 1) / SCAN_T;
  {
    LaunchScope ls(KID_RADS_SCAN, st);
    rads_scan_local_kernel<<<(unsigned)nt, SCAN_T, 0, st>>>(a, b, n, ao, bo, tops);
  }
  {
    LaunchScope ls(KID_RADS_SCAN, st);
    rads_scan_tops_kernel<<<1, SCAN_T, 0, st>>>(tops, nt, n, ao, bo);
  }
  if (nt > 1) {
    LaunchScope ls(KID_RADS_SCAN, st);
    rads_scan_add_kernel<<<(unsigned)nt, SCAN_T, 0, st>>>(tops, n, ao, bo);
  }
}

}  // namespace

extern "C" ddgs_status ddgs_rads(const ddgs_volume *vol, int32_t n1, int32_t n2, uint64_t seed,
                                 ddgs_workspace *ws, float *means, float *log_scales,
                                 int64_t *kept_edges, int64_t *draw_voxels, int64_t *counts,
                                 void *stream) {
  using namespace ddgs;
  if (!vol || !ws || !counts || !vol->hu || n1 < 0 || n2 < 0) return DDGS_ERR_INVALID_ARG;
  int dev = -1;  // the workspace's buffers live on the device current at its creation
  if (cudaGetDevice(&dev) != cudaSuccess || dev != ws->device) return DDGS_ERR_INVALID_ARG;
  if (vol->nx < 1 || vol->ny < 1 || vol->nz < 1) return DDGS_ERR_INVALID_ARG;
  const int64_t nvox = (int64_t)vol->nx * vol->ny * vol->nz;
  if (nvox * 3 >= (int64_t(1) << 32)) return DDGS_ERR_INVALID_ARG;  // edge ids fill the key's low word
  if ((reinterpret_cast<uintptr_t>(vol->hu) & 15u) != 0) return DDGS_ERR_INVALID_ARG;
  if ((int64_t)n1 + n2 > 0 && (!means || !log_scales)) return DDGS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Vol v{vol->hu, vol->nx, vol->ny, vol->nz, nvox, vol->spacing[0], vol->spacing[1],
        vol->spacing[2], vol->origin[0], vol->origin[1], vol->origin[2]};
  const int64_t nblk = (nvox + RCH - 1) / RCH;
  const bool vec = vol->nx % 8 == 0;  // rows of whole 16-byte vectors
  const int64_t n_max = (int64_t)n1 + n2;
  // candidate slices of the neighbour search: enough blocks to fill the GPU
  const int64_t qblk = (n_max + KNN_T * KNN_Q - 1) / (KNN_T * KNN_Q);
  const int slices = (int)std::max<int64_t>(1, std::min<int64_t>(32, qblk ? (8 * device_sms() + qblk - 1) / qblk : 1));

  // scratch: state | cnt u32[nblk] | wsub u64[8 nblk] | wsum u64[nblk] | coff u64[nblk+1] |
  //          woff u64[nblk+1] | scan tops u64[2][1024] | knn partial f32x4[slices][n1+n2]
  const int64_t o_cnt = align256(sizeof(RadsState)), o_ws = o_cnt + align256(4 * nblk),
                o_wsum = o_ws + align256(8 * NSUB * nblk), o_coff = o_wsum + align256(8 * nblk),
                o_woff = o_coff + align256(8 * (nblk + 1)), o_tops = o_woff + align256(8 * (nblk + 1)),
                o_knn = o_tops + align256(16 * SCAN_T),
                bytes = o_knn + align256(16 * (int64_t)slices * std::max<int64_t>(n_max, 1));
  ddgs_status s;
  if ((s = grow_bytes(ws->rads_buf, ws->rads_buf_cap, bytes))) return s;
  unsigned char *b = ws->rads_buf;
  RadsState *state = reinterpret_cast<RadsState *>(b);
  uint32_t *cnt = reinterpret_cast<uint32_t *>(b + o_cnt);
  uint64_t *wsub = reinterpret_cast<uint64_t *>(b + o_ws);
  uint64_t *wsum = reinterpret_cast<uint64_t *>(b + o_wsum);
  uint64_t *tops = reinterpret_cast<uint64_t *>(b + o_tops);
  uint64_t *coff = reinterpret_cast<uint64_t *>(b + o_coff);
  uint64_t *woff = reinterpret_cast<uint64_t *>(b + o_woff);
  float *knn_part = reinterpret_cast<float *>(b + o_knn);

  RCK(cudaMemsetAsync(&state->hu_min, 0x7f, sizeof(int32_t), st));  // > any int16
  RCK(cudaMemsetAsync(&state->hu_max, 0x80, sizeof(int32_t), st));  // < any int16
  {
    LaunchScope ls(KID_RADS_MINMAX, st);
    const int64_t want = (nvox / 8 + RT - 1) / RT;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, 8 * device_sms()));
    rads_minmax_kernel<<<grid, RT, 0, st>>>(v, state);
  }
  {
    LaunchScope ls(KID_RADS_COUNT, st);
    if (vec) rads_count_kernel<true><<<(unsigned)nblk, RT, 0, st>>>(v, state, cnt, wsub, wsum);
    else rads_count_kernel<false><<<(unsigned)nblk, RT, 0, st>>>(v, state, cnt, wsub, wsum);
  }
  scan_chunks(cnt, wsum, nblk, coff, woff, tops, st);
  RCK(cudaGetLastError());
  uint64_t tot[2] = {0, 0};
  RCK(cudaMemcpyAsync(&tot[0], coff + nblk, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  RCK(cudaMemcpyAsync(&tot[1], woff + nblk, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  RCK(cudaStreamSynchronize(st));
  const int64_t M = (int64_t)tot[0];
  const int64_t m1 = std::min<int64_t>(n1, M), m2 = tot[1] > 0 ? n2 : 0;

  if (m1 > 0) {
    // keys u64[M] | off u64[nkb+1] | cnt u32[nkb]
    const int64_t nkb = (M + RCH - 1) / RCH;
    const int64_t k_off = align256(8 * M), k_cnt = k_off + align256(8 * (nkb + 1)),
                  kbytes = k_cnt + align256(4 * nkb);
    if ((s = grow_bytes(ws->rads_keys, ws->rads_key_cap, kbytes))) return s;
    unsigned char *kb = reinterpret_cast<unsigned char *>(ws->rads_keys);
    uint64_t *keys = ws->rads_keys;
    uint64_t *koff = reinterpret_cast<uint64_t *>(kb + k_off);
    uint32_t *kcnt = reinterpret_cast<uint32_t *>(kb + k_cnt);
    {
      LaunchScope ls(KID_RADS_EMIT, st);
      if (vec) rads_emit_kernel<true><<<(unsigned)nblk, RT, 0, st>>>(v, state, coff, seed, keys, (uint64_t)M);
      else rads_emit_kernel<false><<<(unsigned)nblk, RT, 0, st>>>(v, state, coff, seed, keys, (uint64_t)M);
    }
    const int all = M <= n1 ? 1 : 0;
    if (!all) {
      {
        LaunchScope ls(KID_RADS_SELECT, st);
        rads_select_init_kernel<<<1, RT, 0, st>>>(state, (uint64_t)(n1 - 1));
      }
      const unsigned hg = (unsigned)std::max<int64_t>(1, std::min<int64_t>((M + RT - 1) / RT, 2 * device_sms()));
      // digits of 11 bits from the top: shifts 53, 42, 31, 20, 9 and a last 9-bit digit
      for (int shift = 53; shift >= 0; shift -= 11) {
        LaunchScope ls(KID_RADS_SELECT, st);
        rads_select_pass_kernel<<<hg, RT, 0, st>>>(keys, M, state, shift, 11);
      }
      {
        LaunchScope ls(KID_RADS_SELECT, st);
        rads_select_pass_kernel<<<hg, RT, 0, st>>>(keys, M, state, 0, 9);
      }
    }
    {
      LaunchScope ls(KID_RADS_SELECT, st);
      rads_keep_count_kernel<<<(unsigned)nkb, RT, 0, st>>>(keys, M, state, all, kcnt);
    }
    scan_chunks(kcnt, nullptr, nkb, koff, nullptr, tops, st);
    {
      LaunchScope ls(KID_RADS_SELECT, st);
      rads_keep_emit_kernel<<<(unsigned)nkb, RT, 0, st>>>(v, keys, M, state, all, koff, m1, means,
                                                          kept_edges);
    }
    RCK(cudaGetLastError());
  }
  if (m2 > 0) {
    LaunchScope ls(KID_RADS_DRAW, st);
    const unsigned g = (unsigned)((m2 + RT / 32 - 1) / (RT / 32));
    if (vec)
      rads_draw_kernel<true><<<g, RT, 0, st>>>(v, state, woff, wsub, nblk, (int32_t)m2, seed, m1,
                                               means, draw_voxels);
    else
      rads_draw_kernel<false><<<g, RT, 0, st>>>(v, state, woff, wsub, nblk, (int32_t)m2, seed, m1,
                                                means, draw_voxels);
    RCK(cudaGetLastError());
  }
  const int64_t n = m1 + m2;
  if (n > 0) {
    const int64_t slice = (n + slices - 1) / slices;
    {
      LaunchScope ls(KID_RADS_KNN, st);
      const unsigned qb = (unsigned)((n + KNN_T * KNN_Q - 1) / (KNN_T * KNN_Q));
      rads_knn_part_kernel<<<dim3(qb, (unsigned)slices), KNN_T, 0, st>>>(means, n, slice, knn_part);
    }
    {
      LaunchScope ls(KID_RADS_KNN, st);
      rads_knn_merge_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(knn_part, n, slices, log_scales);
    }
    RCK(cudaGetLastError());
  }
  counts[0] = m1;
  counts[1] = m2;
  counts[2] = M;
  return DDGS_OK;
}
