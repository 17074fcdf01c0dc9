// gp_hash_build_static: the spatial hash of gp_hash_build for callers that
// cannot allocate device memory.
//
// Some host programs cannot hand this library a workspace and cannot let it call
// cudaMalloc: a solver embedded in another code whose device memory is owned and
// budgeted by that code's own pool allocator, or a caller on a latency-critical
// path that must not pay the implicit device synchronisation of an allocation.
// This entry point therefore takes its scratch (sort buffers, look-back words,
// histograms, compaction arrays) from one statically sized device array defined
// in this file.  Every GPU that loads the library holds that array until the
// process exits.
//
// Limits and sharing rules:
//  - at most GP_STATIC_SCRATCH_MAX_POINTS points per call; larger n is refused
//    with GP_ERR_CAPACITY before any device work;
//  - the array is shared by all calls on a device and keeps what the previous
//    call left in it; each call clears the counters that must start at zero
//    (histograms, tile tickets, look-back words, error word, cell counter);
//  - two calls whose device work overlaps (different streams, or different
//    host threads on one stream without ordering) race on the array: callers
//    must order them;
//  - the first call on a device looks up the device address of the array
//    (cudaGetSymbolAddress, with that device current) and caches it, so that
//    first call should come before any stream capture on that device.
#include <cmath>
#include <mutex>

#include "../../include/gp.h"
#include "gp_kernels.cuh"

using namespace gp;

namespace {

constexpr int64_t kMaxPoints = GP_STATIC_SCRATCH_MAX_POINTS;
constexpr size_t kA = 256;
constexpr size_t up(size_t x) { return (x + kA - 1) / kA * kA; }
constexpr size_t kTiles = (kMaxPoints + SortTile<uint32_t>::tile - 1) / SortTile<uint32_t>::tile;

// byte offsets of the scratch regions
constexpr size_t kKeys0 = 0;
constexpr size_t kKeys1 = kKeys0 + up(4 * kMaxPoints + 16);
constexpr size_t kVals0 = kKeys1 + up(4 * kMaxPoints + 16);
constexpr size_t kVals1 = kVals0 + up(4 * kMaxPoints + 16);
constexpr size_t kStatus = kVals1 + up(4 * kMaxPoints + 16);
constexpr size_t kHist = kStatus + up(4 * 256 * kTiles);
constexpr size_t kTickets = kHist + up(4 * kSortMaxPasses * 256);
constexpr size_t kErr = kTickets + up(64);
constexpr size_t kFlags = kErr + up(64);
constexpr size_t kOfs = kFlags + up(4 * kMaxPoints);
constexpr size_t kBsum = kOfs + up(4 * kMaxPoints);
constexpr size_t kNcell = kBsum + up(4 * (kMaxPoints / 256 + 1) + 16);
constexpr size_t kBytes = kNcell + up(64);

// 6,390,784 bytes: the size include/gp.h states
static_assert(kBytes == 6390784, "scratch size stated in gp.h");
static __device__ __align__(256) unsigned char g_scratch[kBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// device address of g_scratch on the current device (looked up once per device)
gp_status scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GP_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return GP_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return GP_ERR_CUDA;
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return GP_OK;
}

}  // namespace

extern "C" gp_status gp_hash_build_static(const float* x3, int64_t n, const gp_domain* domain,
                                          double h, uint32_t* keys_sorted, int32_t* ids_sorted,
                                          uint32_t* cell_keys, int32_t* cell_start,
                                          int64_t* n_cells, void* cuda_stream) {
  if (!domain || n < 0 || !(h > 0)) return GP_ERR_ARG;
  if (n > kMaxPoints) return GP_ERR_CAPACITY;
  if (n > 0 && (!x3 || !keys_sorted || !ids_sorted || !cell_keys || !cell_start))
    return GP_ERR_ARG;
  if (n == 0) {
    if (n_cells) *n_cells = 0;
    return GP_OK;
  }
  // hash grid: the definition gp_hash_build uses (cell edge h (1 + 2^-9))
  Params P{};
  uint64_t ncells = 1;
  if (!hash_cells(domain->lo, domain->hi, h, P.geo.nc, &ncells)) return GP_ERR_ARG;
  for (int a = 0; a < 3; ++a) {
    P.geo.lo[a] = (float)domain->lo[a];
    P.geo.hi[a] = (float)domain->hi[a];
  }
  P.inv_c = (float)(1.0 / cell_edge(h));
  for (int a = 0; a < 3; ++a) P.geo.inv[a] = P.inv_c;
  float hf = (float)h;
  P.rc2 = hf * hf;

  unsigned char* b = nullptr;
  gp_status s = scratch_address(&b);
  if (s != GP_OK) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  SortBufs sb{};
  uint32_t* keys[2] = {reinterpret_cast<uint32_t*>(b + kKeys0),
                       reinterpret_cast<uint32_t*>(b + kKeys1)};
  sb.keys[0] = keys[0];
  sb.keys[1] = keys[1];
  sb.vals[0] = reinterpret_cast<uint32_t*>(b + kVals0);
  sb.vals[1] = reinterpret_cast<uint32_t*>(b + kVals1);
  sb.status = reinterpret_cast<uint32_t*>(b + kStatus);
  sb.hist = reinterpret_cast<uint32_t*>(b + kHist);
  sb.ticket = reinterpret_cast<uint32_t*>(b + kTickets);
  sb.err = reinterpret_cast<uint32_t*>(b + kErr);
  sb.max_n = kMaxPoints;
  int dev = 0;
  cudaGetDevice(&dev);
  sb.sms = 152;
  cudaDeviceGetAttribute(&sb.sms, cudaDevAttrMultiProcessorCount, dev);
  sb.prof = nullptr;
  // counters that must start at zero (the sort clears its own histograms,
  // tickets and look-back words on every pass)
  if (cudaMemsetAsync(b + kErr, 0, 64, st) != cudaSuccess ||
      cudaMemsetAsync(b + kNcell, 0, 64, st) != cudaSuccess)
    return GP_ERR_CUDA;
  launch_keys_pos(P, x3, nullptr, n, keys[0], sb.vals[0], st);
  uint64_t nm1 = ncells - 1;
  int nbits = 0;
  while (nm1) {
    ++nbits;
    nm1 >>= 1;
  }
  const int w = radix_sort<uint32_t>(sb, n, nbits, st);
  if (w < 0) return GP_ERR_ARG;
  if (cudaMemcpyAsync(keys_sorted, keys[w], 4 * n, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(ids_sorted, sb.vals[w], 4 * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return GP_ERR_CUDA;
  launch_cells(keys[w], n, (uint32_t)ncells, reinterpret_cast<uint32_t*>(b + kFlags),
               reinterpret_cast<uint32_t*>(b + kOfs), reinterpret_cast<uint32_t*>(b + kBsum),
               cell_keys, cell_start, reinterpret_cast<unsigned long long*>(b + kNcell), st);
  unsigned long long nc = 0;
  uint32_t err = 0;
  if (cudaMemcpyAsync(&nc, b + kNcell, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&err, b + kErr, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return GP_ERR_CUDA;
  if (err) return GP_ERR_TIMEOUT;
  if (n_cells) *n_cells = (int64_t)nc;
  return GP_OK;
}
