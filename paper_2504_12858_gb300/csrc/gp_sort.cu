// Stable LSD radix sort of (key, uint32 value) pairs, 8-bit digits; keys are
// uint32 (one run) or uint64 (a batch of runs, whose cell keys exceed 32 bits).
//
// One histogram kernel reads the keys once and counts every digit of every
// pass.  Each pass is then a single kernel ("onesweep", after Adinets & Merrill,
// "Onesweep: a faster least significant digit radix sort for GPUs", 2022):
// a CTA ranks a tile of keys (3072 of 32 bits or 2560 of 64 bits) in shared memory
// (warp-level match ranking, stable in input order; the values are loaded with the
// keys), obtains the global offset of each digit for its tile by
// decoupled look-back over the per-tile digit counts of the preceding tiles, and
// scatters the tile through a shared-memory staging buffer so that equal digits
// leave as contiguous runs.  Tiles are numbered by an atomic ticket, so a CTA
// only ever waits for tiles whose CTAs are already resident; every wait is
// bounded and reports ERR_TIMEOUT instead of spinning forever.
#include <algorithm>

#include "gp_internal.cuh"

namespace gp {

namespace {

// Counts every digit of every pass: 32-bit keys, four per 16-byte load.  With
// n_dev the key count is read on the device.
__global__ void __launch_bounds__(256) k_hist32(const uint32_t* __restrict__ keys, int64_t n,
                                                const unsigned long long* n_dev, int npass,
                                                uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[4 * 256];
  if (n_dev) n = (int64_t)*n_dev;
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n4 = n >> 2;
  const uint4* k4 = reinterpret_cast<const uint4*>(keys);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    uint4 v = __ldg(k4 + i);
    uint32_t kk[4] = {v.x, v.y, v.z, v.w};
    const uint32_t m = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      for (int p = 0; p < npass; ++p) {
        // the keys are nearly sorted, so the high digits are mostly the same across
        // a warp: one shared atomic then, else one per lane (3.6x faster than
        // grouping the lanes by digit with a match)
        const uint32_t d = (kk[q] >> (8 * p)) & 255u;
        if (__all_sync(m, d == __shfl_sync(m, d, leader))) {
          if (lane == leader) atomicAdd(&sh[p * 256 + d], (uint32_t)__popc(m));
        } else {
          atomicAdd(&sh[p * 256 + d], 1u);
        }
      }
  }
  for (int64_t i = (n4 << 2) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint32_t k = keys[i];
    for (int p = 0; p < npass; ++p) atomicAdd(&sh[p * 256 + ((k >> (8 * p)) & 255u)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npass * 256; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// the same for 64-bit keys (up to kSortMaxPasses digits), two per 16-byte load
__global__ void __launch_bounds__(256) k_hist64(const uint64_t* __restrict__ keys, int64_t n,
                                                const unsigned long long* n_dev, int npass,
                                                uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[kSortMaxPasses * 256];
  if (n_dev) n = (int64_t)*n_dev;
  for (int i = threadIdx.x; i < kSortMaxPasses * 256; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n2 = n >> 1;
  const uint4* k2 = reinterpret_cast<const uint4*>(keys);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
    uint4 v = __ldg(k2 + i);
    uint64_t kk[2] = {(uint64_t)v.x | ((uint64_t)v.y << 32), (uint64_t)v.z | ((uint64_t)v.w << 32)};
    const uint32_t m = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
#pragma unroll
    for (int q = 0; q < 2; ++q)
      for (int p = 0; p < npass; ++p) {
        const uint32_t d = (uint32_t)(kk[q] >> (8 * p)) & 255u;
        if (__all_sync(m, d == __shfl_sync(m, d, leader))) {
          if (lane == leader) atomicAdd(&sh[p * 256 + d], (uint32_t)__popc(m));
        } else {
          atomicAdd(&sh[p * 256 + d], 1u);
        }
      }
  }
  for (int64_t i = (n2 << 1) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t k = keys[i];
    for (int p = 0; p < npass; ++p)
      atomicAdd(&sh[p * 256 + ((uint32_t)(k >> (8 * p)) & 255u)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npass * 256; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// exclusive scan of 256 values held one per thread (blockDim.x == 256)
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t v, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < 8 ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < 8) s_warp[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  uint32_t base = warp ? s_warp[warp - 1] : 0;
  uint32_t r = base + x - v;
  __syncthreads();
  return r;
}

template <class K>
__global__ void __launch_bounds__(kSortThreads, SortTile<K>::ctas) k_onesweep(
    const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n, const unsigned long long* n_dev, int shift,
    const uint32_t* __restrict__ hist, uint32_t* status, uint32_t* ticket, uint32_t* err) {
  constexpr int W = kSortThreads / 32;
  constexpr int kItems = SortTile<K>::items;
  constexpr int kTile = SortTile<K>::tile;
  __shared__ uint32_t s_whist[W][256];
  __shared__ K s_keys[kTile];
  __shared__ uint32_t s_vals[kTile];
  __shared__ uint32_t s_start[256];  // tile-local start of each digit
  __shared__ uint32_t s_gofs[256];   // global position of tile-local index 0 of each digit
  __shared__ uint32_t s_tmp[8];
  __shared__ uint32_t s_tile;

  if (n_dev) n = (int64_t)*n_dev;
  const int64_t ntiles = (n + kTile - 1) / kTile;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // a CTA takes tiles in ticket order until none is left (one tile per CTA when the
  // grid covers all tiles; a persistent grid otherwise)
  while (true) {
    if (tid == 0) s_tile = atomicAdd(ticket, 1u);
    for (int i = tid; i < W * 256; i += kSortThreads) (&s_whist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    if ((int64_t)tile >= ntiles) break;
    const int64_t base = (int64_t)tile * kTile;

    // keys, values and ranks live in registers (digits are recomputed); the values
    // are loaded with the keys, so that both are in flight during the ranking
    K k[kItems];
    uint32_t rk[kItems], v[kItems];
    const int64_t wbase = base + (int64_t)warp * kItems * 32;
    const int64_t nvalid = n - wbase;  // items of this warp's run that exist
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      int64_t idx = wbase + r * 32 + lane;
      k[r] = idx < n ? kin[idx] : ~K(0);
      v[r] = idx < n ? __ldg(vin + idx) : 0u;
    }
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int d = (r * 32 + lane) < nvalid ? (int)((uint32_t)(k[r] >> shift) & 255u) : 256;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      uint32_t before = 0;
      if (d < 256) before = s_whist[warp][d];
      rk[r] = before + __popc(peers & lt_mask);
      __syncwarp();
      if (d < 256 && lane == __ffs(peers) - 1) s_whist[warp][d] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();

    // per digit (one thread each): warp-exclusive offsets and the tile count
    const int d = tid;
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      uint32_t c = s_whist[w][d];
      s_whist[w][d] = cnt;
      cnt += c;
    }
    const uint32_t start = block_excl_scan_256(cnt, s_tmp);
    s_start[d] = start;

    // global digit base: exclusive scan of the whole-array histogram
    const uint32_t dbase = block_excl_scan_256(hist[d], s_tmp);

    // decoupled look-back over preceding tiles, digit d
    uint32_t* my = status + (size_t)tile * 256 + d;
    uint32_t excl = 0;
    if (tile == 0) {
      atomicExch(my, kFlagInc | cnt);
    } else {
      atomicExch(my, kFlagAgg | cnt);
      excl = lookback_excl(status, (int64_t)tile, d, kSpinLimit, err);
      atomicExch(my, kFlagInc | ((excl + cnt) & kValMask));
    }
    s_gofs[d] = dbase + excl - start;  // wraps modulo 2^32; the sum below is exact
    __syncthreads();

#pragma unroll
    for (int r = 0; r < kItems; ++r) {
      const int64_t idx = wbase + r * 32 + lane;
      if (idx < n) {
        const uint32_t d = (uint32_t)(k[r] >> shift) & 255u;
        const uint32_t lp = s_start[d] + s_whist[warp][d] + rk[r];
        s_keys[lp] = k[r];
        s_vals[lp] = v[r];
      }
    }
    __syncthreads();
    const int64_t rem = n - base;
    const int tn = rem < kTile ? (int)rem : kTile;
    for (int i = tid; i < tn; i += kSortThreads) {
      const K key = s_keys[i];
      uint32_t g = s_gofs[(uint32_t)(key >> shift) & 255u] + (uint32_t)i;
      if ((int64_t)g < n) {
        kout[g] = key;
        vout[g] = s_vals[i];
      } else {
        atomicOr(err, ERR_TIMEOUT);
      }
    }
    __syncthreads();  // the shared arrays are reused by the next tile
  }
}

}  // namespace

size_t radix_status_words(int64_t n, int key_bytes) {
  const int tile = key_bytes == 8 ? SortTile<uint64_t>::tile : SortTile<uint32_t>::tile;
  const int64_t tiles = (n + tile - 1) / tile;
  return (size_t)(tiles < 1 ? 1 : tiles) * 256;
}

template <class K>
int radix_sort(const SortBufs& B, int64_t n, int nbits, cudaStream_t st) {
  const bool dev = B.n_dev != nullptr;  // n is then an upper bound only
  if ((!dev && n <= 1) || nbits <= 0) return 0;
  const int npass = (nbits + 7) / 8;
  if (npass > kSortMaxPasses || 8 * (int)sizeof(K) < nbits) return -1;
  constexpr int kTile = SortTile<K>::tile;
  const int64_t nmax = dev ? B.max_n : n;
  const int64_t tiles = (nmax + kTile - 1) / kTile;
  // one tile per CTA, or a persistent grid of the resident CTAs
  const int64_t grid = dev ? std::min<int64_t>(tiles, SortTile<K>::ctas * (int64_t)B.sms) : tiles;
  cudaMemsetAsync(B.hist, 0, sizeof(uint32_t) * 256 * npass, st);
  cudaMemsetAsync(B.ticket, 0, sizeof(uint32_t) * kSortMaxPasses, st);
  int hblocks = (int)((nmax / 4 + 255) / 256);
  if (hblocks > B.sms * 8) hblocks = B.sms * 8;
  if (hblocks < 1) hblocks = 1;
  K* keys[2] = {static_cast<K*>(B.keys[0]), static_cast<K*>(B.keys[1])};
  if (B.prof) B.prof->begin(K_HIST);
  if constexpr (sizeof(K) == 4)
    k_hist32<<<hblocks, 256, 0, st>>>(keys[0], n, B.n_dev, npass, B.hist);
  else
    k_hist64<<<hblocks, 256, 0, st>>>(keys[0], n, B.n_dev, npass, B.hist);
  if (B.prof) B.prof->end(K_HIST, (double)n);
  int cur = 0;
  for (int p = 0; p < npass; ++p) {
    cudaMemsetAsync(B.status, 0, sizeof(uint32_t) * 256 * (size_t)tiles, st);
    if (B.prof) B.prof->begin(K_ONESWEEP);
    k_onesweep<K><<<(unsigned)grid, kSortThreads, 0, st>>>(
        keys[cur], B.vals[cur], keys[cur ^ 1], B.vals[cur ^ 1], n, B.n_dev, 8 * p,
        B.hist + 256 * p, B.status, B.ticket + p, B.err);
    if (B.prof) B.prof->end(K_ONESWEEP, (double)n);
    cur ^= 1;
  }
  return cur;
}

template int radix_sort<uint32_t>(const SortBufs&, int64_t, int, cudaStream_t);
template int radix_sort<uint64_t>(const SortBufs&, int64_t, int, cudaStream_t);

}  // namespace gp
