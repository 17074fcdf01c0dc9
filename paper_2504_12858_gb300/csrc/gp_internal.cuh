// Internal device-side definitions of the grain-envelope particle library.
//
// Device state is binary32.  Notation follows Sec. 2.1.2 of the paper: a
// particle of grain g at lattice site s (crystal frame, relative to the nucleus
// c_g) moving in direction k with progress ell sits at
//     x = c_g + h R_g s + ell * sigma_k * h R_g e_{a_k}
// where a_k = k >> 1 is the axis and sigma_k = +1 for even k, -1 for odd k.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace gp {

// ---------------------------------------------------------------------------------
// constants
// ---------------------------------------------------------------------------------
enum : int { ST_ACTIVE = 0, ST_FROZEN = 1, ST_REMOVED = 2 };

// sticky device error bits (reported in gp_stats_t.error_flags)
enum : uint32_t {
  ERR_CAPACITY = 1u,      // particle store full
  ERR_HASH_FULL = 2u,     // claim table probe limit / load exceeded
  ERR_TIMEOUT = 4u,       // a bounded look-back wait gave up
  ERR_REACHED_CAP = 8u,   // reached-site list full
  ERR_CELL_OVERFLOW = 16u,// 32767 or more particles in one segment of 16 hash cells
  ERR_GRAINS = 32u,       // grain table full
  ERR_SITE_RANGE = 64u,   // lattice site outside [-4095, 4095]
};

constexpr int kSiteMax = 4095;
constexpr int kClaimProbeLimit = 4096;
constexpr uint32_t kSpinLimit = 1u << 22;  // polls (~seconds) before a look-back wait gives up
constexpr int kBrickWords = 128;           // 8^3 sites, one byte each, 4 per word
constexpr int kSegShift = 4;               // the cell table has one entry per 16 cells of a row
constexpr int kSegCells = 1 << kSegShift;
constexpr uint32_t kSegMaxCount = 0x7fffu;  // particles per segment (15-bit count)
// tiles of the particle step's cell order: 16 x 2^kTileYShift x 2^kTileZShift cells
constexpr int kTileYShift = 3;
constexpr int kTileZShift = 3;
// a single run groups its records by key >> kGroupShift (one tile: 1024 cells, 64
// segments) and orders them by cell inside each group, in place of the radix sort
constexpr int kGroupShift = 10;
constexpr int kGroupCells = 1 << kGroupShift;

// ---------------------------------------------------------------------------------
// hash grid (host side): cells of edge h (1 + 2^-9), the contact radius enlarged so
// that binary32 rounding of the cell coordinate can never separate two points closer
// than h by more than one cell (up to 4096 cells per axis).  Cells per axis
// n_a = max(1, ceil((hi_a - lo_a) / edge)); false if an extent is not finite and
// non-negative, an axis needs more than 4096 cells or the grid 2^32 cells or more.
// ---------------------------------------------------------------------------------
inline double cell_edge(double h) { return h * (1.0 + 1.0 / 512.0); }

inline bool hash_cells(const double lo[3], const double hi[3], double h, int nc[3],
                       uint64_t* ncells) {
  const double e = cell_edge(h);
  uint64_t tot = 1;
  for (int a = 0; a < 3; ++a) {
    const double ext = hi[a] - lo[a];
    if (!(ext >= 0) || !std::isfinite(ext)) return false;
    const double v = std::ceil(ext / e);
    if (v > 4096.0) return false;
    nc[a] = v < 1 ? 1 : (int)v;
    tot *= (uint64_t)nc[a];
  }
  *ncells = tot;
  return tot < (1ull << 32);
}

// ---------------------------------------------------------------------------------
// particle record: 16 bytes, loaded and stored as one int4
//   x: grain id
//   y: sx (int16, low half) | sy (int16, high half)
//   z: sz (int16, bits 0..15) | dir (bits 16..18) | state (bits 20..21) |
//      crossing flag (bit 24: the particle reached its target this step)
//   w: ell (binary32 bits)
// ---------------------------------------------------------------------------------
struct Rec {
  int grain;
  int sx, sy, sz;
  int dir;
  int state;
  int cross;
  float ell;
};

__host__ __device__ inline int4 rec_pack(const Rec& r) {
  int4 v;
  v.x = r.grain;
  v.y = (int)((uint32_t)(uint16_t)(int16_t)r.sx | ((uint32_t)(uint16_t)(int16_t)r.sy << 16));
  v.z = (int)((uint32_t)(uint16_t)(int16_t)r.sz | ((uint32_t)(r.dir & 7) << 16) |
              ((uint32_t)(r.state & 3) << 20) | ((uint32_t)(r.cross & 1) << 24));
#ifdef __CUDA_ARCH__
  v.w = __float_as_int(r.ell);
#else
  union { float f; int i; } u;
  u.f = r.ell;
  v.w = u.i;
#endif
  return v;
}

__host__ __device__ inline Rec rec_unpack(int4 v) {
  Rec r;
  r.grain = v.x;
  r.sx = (int16_t)(uint16_t)((uint32_t)v.y & 0xFFFFu);
  r.sy = (int16_t)(uint16_t)((uint32_t)v.y >> 16);
  r.sz = (int16_t)(uint16_t)((uint32_t)v.z & 0xFFFFu);
  r.dir = ((uint32_t)v.z >> 16) & 7;
  r.state = ((uint32_t)v.z >> 20) & 3;
  r.cross = ((uint32_t)v.z >> 24) & 1;
#ifdef __CUDA_ARCH__
  r.ell = __int_as_float(v.w);
#else
  union { float f; int i; } u;
  u.i = v.w;
  r.ell = u.f;
#endif
  return r;
}

// ---------------------------------------------------------------------------------
// simulation constants (passed by value to every kernel)
// ---------------------------------------------------------------------------------
// Domain, hash geometry and analytic field of one simulation ("run").  A context
// holds either one run (Params::geo) or a batch of independent runs (the table
// Params::runs, indexed by the run id that each grain's table entry carries).
// The runs of a batch take consecutive ranges of the cell keys, of the cell table
// and of the reached-site heads.
struct Geo {
  float lo[3], hi[3];
  int nc[3];                 // hash cells per axis
  float inv[3];              // 1 / cell edge per axis (the contact search's cells)
  int nsx;                   // segments of kSegCells cells per x row of the hash grid
  int tx, ty;                // tiles along x and y (tiled cell order)
  unsigned long long key0;   // cell key of the run's cell 0
  unsigned long long seg0;   // first cell-table entry of the run
  unsigned long long head0;  // first reached-site head of the run
  float G[3], xref[3];       // analytic field: T = T0 + G . (x - xref) + Tdot t
  float dT_base;             // T_L - T0 - Tdot t_n
  float dT_base1;            // T_L - T0 - Tdot t_{n+1} (nucleation)
};

struct Params {
  Geo geo;           // the run of a single-run context
  const Geo* runs;   // batch: one entry per run
  float inv_c;       // (float)(1/edge): cell index scale
  float rc2;         // contact radius squared, hf * hf with hf = (float)h
  float dt_over_h;   // (float)(dt / h)
  int nterms;
  float a[2], b[2];
  int bint[2];       // b as a small integer exponent (1..8), else -1 (powf)
  float TL;
  int thermal;       // 0 none, 1 analytic, 2 grid
  const float* grid;
  int gn[3];
  float ginv[3];     // 1 / spacing
  const float4* gtab;// grain table: 4 float4 per grain (c with the run id in w, rows of h R)
  int hshift;        // one reached-site head per 2^hshift cells along each axis
  // periodic axes of a single run (bit a): positions wrap into [lo, hi), distances
  // take the nearest image, no clip; per_L = hi - lo
  int periodic;
  float per_L[3];
  // local liquidus T_m + m_L w(x) from a composition grid (solute != 0)
  int solute;
  const float* wgrid;
  int wn[3];
  float winv[3];
  float Tm, mL;
  // grids of the device-sized (batch) launches, in CTAs over the whole GPU
  struct {
    int build_ctas, advance_ctas, emit_ctas;
  } launch;
};

// per-step constants of the gridded field (computed on the host in double)
struct StepArgs {
  float gshift[3];   // grid: origin + frame_vel t
  float wshift[3];   // composition grid: origin + frame_vel t
  int parity;        // step & 1: which claimant bits of a site byte are live
};

// geometry of run `run` (a single-run context has only run 0)
template <bool BATCH>
__device__ __forceinline__ const Geo& geo_of(const Params& P, int run) {
  if constexpr (BATCH) return P.runs[run];
  else return P.geo;
}

// pos4.w / grain-table w word: grain id in the low 24 bits, run id in the high 8
constexpr int kRunShift = 24;
constexpr int kGrainMask = (1 << kRunShift) - 1;
constexpr int kMaxRuns = 256;

// ---------------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void grain_load(const float4* gtab, int g, float4& c, float4& r0,
                                           float4& r1, float4& r2) {
  const float4* p = gtab + 4 * (size_t)g;
  c = __ldg(p);
  r0 = __ldg(p + 1);
  r1 = __ldg(p + 2);
  r2 = __ldg(p + 3);
}

// x = c + hR s, evaluated with explicit fused multiply-adds so every kernel that
// needs a position obtains the same binary32 value.
__device__ __forceinline__ float3 site_pos_g(float4 c, float4 r0, float4 r1, float4 r2, int sx,
                                             int sy, int sz) {
  float fx = (float)sx, fy = (float)sy, fz = (float)sz;
  float3 p;
  p.x = __fmaf_rn(r0.z, fz, __fmaf_rn(r0.y, fy, __fmaf_rn(r0.x, fx, c.x)));
  p.y = __fmaf_rn(r1.z, fz, __fmaf_rn(r1.y, fy, __fmaf_rn(r1.x, fx, c.y)));
  p.z = __fmaf_rn(r2.z, fz, __fmaf_rn(r2.y, fy, __fmaf_rn(r2.x, fx, c.z)));
  return p;
}

__device__ __forceinline__ float3 add_dir(float3 p, float4 r0, float4 r1, float4 r2, int dir,
                                          float ell) {
  int a = dir >> 1;
  float sl = (dir & 1) ? -ell : ell;
  float cx = a == 0 ? r0.x : (a == 1 ? r0.y : r0.z);
  float cy = a == 0 ? r1.x : (a == 1 ? r1.y : r1.z);
  float cz = a == 0 ? r2.x : (a == 1 ? r2.y : r2.z);
  p.x = __fmaf_rn(sl, cx, p.x);
  p.y = __fmaf_rn(sl, cy, p.y);
  p.z = __fmaf_rn(sl, cz, p.z);
  return p;
}

__device__ __forceinline__ float3 part_pos(const float4* gtab, int g, int sx, int sy, int sz,
                                           int dir, float ell) {
  float4 c, r0, r1, r2;
  grain_load(gtab, g, c, r0, r1, r2);
  return add_dir(site_pos_g(c, r0, r1, r2, sx, sy, sz), r0, r1, r2, dir, ell);
}

__device__ __forceinline__ int cell1(float x, float lo, float inv, int n) {
  float u = __fmul_rn(__fsub_rn(x, lo), inv);
  int c = __float2int_rd(u);
  return min(max(c, 0), n - 1);
}

// cell of p in its run's hash grid (clamped) and the run-local linear cell index
__device__ __forceinline__ uint32_t cell_local(const Geo& g, float3 p, int& cx, int& cy,
                                               int& cz) {
  cx = cell1(p.x, g.lo[0], g.inv[0], g.nc[0]);
  cy = cell1(p.y, g.lo[1], g.inv[1], g.nc[1]);
  cz = cell1(p.z, g.lo[2], g.inv[2], g.nc[2]);
  return (uint32_t)(((uint64_t)cz * g.nc[1] + cy) * g.nc[0] + cx);
}

// position wrapped into [lo, hi) along the periodic axes (single-run contexts)
__device__ __forceinline__ float wrap1(float x, float lo, float L) {
  float u = __fsub_rn(x, lo);
  u = __fsub_rn(u, __fmul_rn(L, floorf(__fdiv_rn(u, L))));
  return __fadd_rn(lo, u);
}
__device__ __forceinline__ float3 wrap_pos(const Params& P, const Geo& g, float3 p) {
  if (P.periodic & 1) p.x = wrap1(p.x, g.lo[0], P.per_L[0]);
  if (P.periodic & 2) p.y = wrap1(p.y, g.lo[1], P.per_L[1]);
  if (P.periodic & 4) p.z = wrap1(p.z, g.lo[2], P.per_L[2]);
  return p;
}
// difference a - b along axis a_ taken to the nearest image on a periodic axis
__device__ __forceinline__ float dmin1(float d, float L, bool per) {
  if (per) {
    if (d > 0.5f * L) d = __fsub_rn(d, L);
    else if (d < -0.5f * L) d = __fadd_rn(d, L);
  }
  return d;
}
__device__ __forceinline__ float dist2_per(const Params& P, float3 a, float3 b) {
  const float dx = dmin1(__fsub_rn(a.x, b.x), P.per_L[0], P.periodic & 1);
  const float dy = dmin1(__fsub_rn(a.y, b.y), P.per_L[1], P.periodic & 2);
  const float dz = dmin1(__fsub_rn(a.z, b.z), P.per_L[2], P.periodic & 4);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ bool inside(const Geo& g, float3 p) {
  return p.x >= g.lo[0] && p.x <= g.hi[0] && p.y >= g.lo[1] && p.y <= g.hi[1] &&
         p.z >= g.lo[2] && p.z <= g.hi[2];
}

// squared distance with every product and sum rounded separately (no contraction)
__device__ __forceinline__ float dist2_rn(float3 a, float3 b) {
  float dx = __fsub_rn(a.x, b.x);
  float dy = __fsub_rn(a.y, b.y);
  float dz = __fsub_rn(a.z, b.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// outer direction at site s (increases |s|_1): s_a == 0 or sign(s_a) == sigma
__device__ __forceinline__ bool is_outer(int sx, int sy, int sz, int k) {
  int a = k >> 1;
  int sa = a == 0 ? sx : (a == 1 ? sy : sz);
  return sa == 0 || ((sa > 0) == ((k & 1) == 0));
}

__device__ __forceinline__ void step_site(int& sx, int& sy, int& sz, int k) {
  int d = (k & 1) ? -1 : 1;
  if ((k >> 1) == 0) sx += d;
  else if ((k >> 1) == 1) sy += d;
  else sz += d;
}

// ---------------------------------------------------------------------------------
// thermal field and growth law
// ---------------------------------------------------------------------------------
// trilinear sample of a node-centred binary32 grid g (n nodes per axis, 1/spacing
// inv) whose node 0 sits at shift; clamped to the table
__device__ __forceinline__ float trilinear(const float* __restrict__ g, const int n[3],
                                           const float inv[3], const float shift[3], float3 p) {
  float u[3] = {__fmul_rn(__fsub_rn(p.x, shift[0]), inv[0]),
                __fmul_rn(__fsub_rn(p.y, shift[1]), inv[1]),
                __fmul_rn(__fsub_rn(p.z, shift[2]), inv[2])};
  int i0[3];
  float f[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float um = (float)(n[a] - 1);
    float v = fminf(fmaxf(u[a], 0.f), um);
    int i = min(__float2int_rd(v), n[a] - 2);
    i0[a] = i;
    f[a] = v - (float)i;
  }
  const int nx = n[0];
  const size_t plane = (size_t)n[0] * n[1];
  const float* b = g + (size_t)i0[2] * plane + (size_t)i0[1] * nx + i0[0];
  float t000 = __ldg(b), t100 = __ldg(b + 1);
  float t010 = __ldg(b + nx), t110 = __ldg(b + nx + 1);
  float t001 = __ldg(b + plane), t101 = __ldg(b + plane + 1);
  float t011 = __ldg(b + plane + nx), t111 = __ldg(b + plane + nx + 1);
  float c00 = __fmaf_rn(f[0], t100 - t000, t000);
  float c10 = __fmaf_rn(f[0], t110 - t010, t010);
  float c01 = __fmaf_rn(f[0], t101 - t001, t001);
  float c11 = __fmaf_rn(f[0], t111 - t011, t011);
  float e0 = __fmaf_rn(f[1], c10 - c00, c00);
  float e1 = __fmaf_rn(f[1], c11 - c01, c01);
  return __fmaf_rn(f[2], e1 - e0, e0);
}

__device__ __forceinline__ float grid_T(const Params& P, const StepArgs& S, float3 p) {
  return trilinear(P.grid, P.gn, P.ginv, S.gshift, p);
}

// undercooling at p; base = T_L - T0 - Tdot t of the analytic field at the time
// of the sample (Geo::dT_base or Geo::dT_base1)
__device__ __forceinline__ float undercooling(const Params& P, const Geo& g, const StepArgs& S,
                                             float3 p, float base) {
  float dT = 0.f;
  if (P.thermal == 1) {
    float v = __fmul_rn(g.G[0], __fsub_rn(p.x, g.xref[0]));
    v = __fmaf_rn(g.G[1], __fsub_rn(p.y, g.xref[1]), v);
    v = __fmaf_rn(g.G[2], __fsub_rn(p.z, g.xref[2]), v);
    dT = base - v;
  } else if (P.thermal == 2) {
    dT = P.TL - grid_T(P, S, p);
  } else {
    return 0.f;
  }
  if (P.solute) {  // local liquidus: add T_m + m_L w(x) - T_L
    const float liq = __fmaf_rn(P.mL, trilinear(P.wgrid, P.wn, P.winv, S.wshift, p), P.Tm);
    dT = __fadd_rn(__fsub_rn(liq, P.TL), dT);
  }
  return dT;
}

__device__ __forceinline__ float ipow(float x, int n) {
  float r = x;
  for (int i = 1; i < n; ++i) r *= x;
  return r;
}

// Eq. (1) / Eq. (2); zero velocity without undercooling
__device__ __forceinline__ float growth_v(const Params& P, float dT) {
  if (!(dT > 0.f)) return 0.f;
  float v = 0.f;
  for (int i = 0; i < P.nterms; ++i) {
    float pw = P.bint[i] > 0 ? ipow(dT, P.bint[i]) : powf(dT, P.b[i]);
    v = __fmaf_rn(P.a[i], pw, v);
  }
  return v;
}

// Explicit Euler step of a particle's progress (Sec. 2.1.2, Eq. 1/2, reading r2): the
// undercooling at its position x_n at t_n, the growth law, dl = v dt / h capped at one
// spacing (capped is set), and e = ell + dl.  The advance and the adjoint's replay of
// the taped steps both call it, so the two obtain the same binary32 values.
__device__ __forceinline__ float euler_ell(const Params& P, const Geo& gm, const StepArgs& S,
                                           float3 x, float ell, bool& capped) {
  const float dT = undercooling(P, gm, S, x, gm.dT_base);
  float dl = __fmul_rn(growth_v(P, dT), P.dt_over_h);
  capped = dl > 1.f;
  if (capped) dl = 1.f;
  return __fadd_rn(ell, dl);
}

// the target counts as reached within 2^-20 of a full spacing (reading r6), so that a
// step commensurate with h does not lose a step to binary32 rounding
__device__ __forceinline__ bool reaches_target(float e) { return e >= 1.f - 0x1p-20f; }

// ---------------------------------------------------------------------------------
// lattice-site claim table: open addressing over 8^3-site blocks of a grain; each
// block holds one byte per site: bit 7 = claimed, bits 0..2 = claimant axes of an
// even step, bits 3..5 = claimant axes of an odd step, bit 6 = reached and not
// melted (maintained by the melting pass only).
// ---------------------------------------------------------------------------------
// The blocks live in a dense pool, handed out in order of first claim (so blocks
// claimed by nearby particles sit close together in memory); an open-addressing
// hash maps each block key to its pool slot.  A bucket is {key, slot + 1}: the
// thread whose compare-and-swap puts the key into an empty bucket reserves the
// pool slot and publishes it in the second word; until then the bucket is
// "pending" (key set, slot word 0).  Claims are made by whole warps together
// (warp_claim_word): each warp first inserts and publishes everything it
// inserts, and only then waits, with a bound, for slots other warps are
// publishing, so no wait can close a cycle.
struct Claims {
  ulonglong2* bucket;         // {block key, pool slot + 1}; {0, 0} = empty
  uint32_t* data;             // pool: kBrickWords words per block
  uint32_t mask;              // buckets - 1
  uint32_t pool_cap;          // blocks in the pool
  unsigned long long* used;   // pool blocks handed out
  uint32_t* err;
};

constexpr unsigned long long kSlotFull = ~0ull;  // published when the pool is full

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z ^= z >> 33;
  z *= 0xff51afd7ed558ccdull;
  z ^= z >> 33;
  z *= 0xc4ceb9fe1a85ec53ull;
  z ^= z >> 33;
  return z;
}

__device__ __forceinline__ unsigned long long block_key(int g, int bx, int by, int bz) {
  return ((unsigned long long)(g + 1) << 30) | ((unsigned long long)(bx + 512) << 20) |
         ((unsigned long long)(by + 512) << 10) | (unsigned long long)(bz + 512);
}

__device__ __forceinline__ int64_t slot_of(unsigned long long v) {
  return v == kSlotFull ? -1 : (int64_t)(v - 1);
}

// Looks up (and with insert, inserts) block `key` without waiting.  Returns its
// pool slot; -1 if absent (insert == false) or if the table or pool is full;
// -2 - b if bucket b holds the key but another thread has not yet published the
// slot.  Linear probing from a mixed hash of the full key: a home bucket with
// spatial locality (grain offset + Morton code of the block) clusters the
// occupied buckets into long runs and multiplies the probe lengths by two orders
// of magnitude at the loads used here.
// A bucket only ever goes from empty to {key, 0} to {key, slot + 1}, so a key or a slot
// that a plain (cacheable) load shows is final; an empty bucket or slot that it shows
// may be an older copy and is read again from memory before it is acted on.  The plain
// load serves most probes from L1: the warps of an SM look up the same few blocks.
__device__ inline int64_t claim_probe(const Claims& C, unsigned long long key, bool insert) {
  uint32_t b = (uint32_t)mix64(key) & C.mask;
  for (int i = 0; i < kClaimProbeLimit; ++i) {
    volatile unsigned long long* kv = &C.bucket[b].x;
    volatile unsigned long long* sv = &C.bucket[b].y;
    const ulonglong2 seen = C.bucket[b];
    unsigned long long k = seen.x;
    if (k == 0ull) k = *kv;
    if (k == 0ull) {
      if (!insert) return -1;
      k = atomicCAS(&C.bucket[b].x, 0ull, key);
      if (k == 0ull) {
        const unsigned long long s = atomicAdd(C.used, 1ull);
        if (s >= C.pool_cap) {
          atomicOr(C.err, ERR_HASH_FULL);
          atomicExch(&C.bucket[b].y, kSlotFull);
          return -1;
        }
        atomicExch(&C.bucket[b].y, s + 1ull);
        return (int64_t)s;
      }
    }
    if (k == key) {
      const unsigned long long v = seen.x == key && seen.y ? seen.y : *sv;
      return v ? slot_of(v) : -2 - (int64_t)b;
    }
    b = (b + 1) & C.mask;
  }
  atomicOr(C.err, ERR_HASH_FULL);
  return -1;
}

// bounded wait for the slot of bucket b: at most `limit` polls, then ERR_TIMEOUT
__device__ inline int64_t claim_wait(const Claims& C, uint32_t b, uint32_t limit = kSpinLimit) {
  volatile unsigned long long* sv = &C.bucket[b].y;
  for (uint32_t spins = 0; spins < limit; ++spins) {
    const unsigned long long v = *sv;
    if (v) return slot_of(v);
  }
  atomicOr(C.err, ERR_TIMEOUT);
  return -1;
}

// ---------------------------------------------------------------------------------
// decoupled look-back of a onesweep pass: each tile publishes, per digit, a status
// word {flag, value}: kFlagAgg with its own count, then kFlagInc with the inclusive
// prefix.  A tile sums the preceding tiles' words from the nearest one backwards until
// it meets an inclusive prefix.  A predecessor that has not published yet is polled;
// after `limit` polls in all the wait gives up, sets ERR_TIMEOUT in *err and returns
// the partial sum (the sort's result is then invalid and the host reports the error).
// ---------------------------------------------------------------------------------
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;

__device__ inline uint32_t lookback_excl(const uint32_t* status, int64_t tile, int d,
                                         uint32_t limit, uint32_t* err) {
  uint32_t excl = 0, spins = 0;
  int64_t pred = tile - 1;
  while (pred >= 0) {
    const uint32_t s = *((volatile const uint32_t*)(status + (size_t)pred * 256 + d));
    const uint32_t flag = s & ~kValMask;
    if (flag == 0u) {
      if (++spins > limit) {
        atomicOr(err, ERR_TIMEOUT);
        break;
      }
      continue;
    }
    excl += s & kValMask;
    if (flag == kFlagInc) break;
    --pred;
  }
  return excl;
}

// The targets of one particle are the neighbours of one site, so they nearly
// always share its 8^3 block: the block lookup is remembered between calls.
struct BlockCache {
  int bx = 0x7fffffff, by = 0, bz = 0;
  int64_t b = -1;
};

__device__ __forceinline__ bool site_in_range(int tx, int ty, int tz) {
  return tx >= -kSiteMax && tx <= kSiteMax && ty >= -kSiteMax && ty <= kSiteMax &&
         tz >= -kSiteMax && tz <= kSiteMax;
}

__device__ __forceinline__ uint32_t* block_word(const Claims& C, int64_t slot, int tx, int ty,
                                                int tz, int& shift) {
  const int local = (((tz & 7) << 3) | (ty & 7)) << 3 | (tx & 7);
  shift = (local & 3) << 3;
  return C.data + (size_t)slot * kBrickWords + (local >> 2);
}

// Word holding the claim byte of site t of grain g (shift: its bit offset) for
// every lane with `have`; nullptr for the others, or if the block is absent / the
// table is full.  Must be called by all 32 lanes of the warp together (converged,
// none exited).  Lanes asking for the same block share one probe; inserts made by
// the warp are published before any lane waits for another warp's insert.
__device__ inline uint32_t* warp_claim_word(const Claims& C, bool have, int g, int tx, int ty,
                                            int tz, bool insert, int& shift, BlockCache& bc) {
  const int lane = threadIdx.x & 31;
  if (have && !site_in_range(tx, ty, tz)) {
    atomicOr(C.err, ERR_SITE_RANGE);
    have = false;
  }
  const int bx = tx >> 3, by = ty >> 3, bz = tz >> 3;
  const bool cached = have && bx == bc.bx && by == bc.by && bz == bc.bz &&
                      (bc.b >= 0 || !insert);
  const bool need = have && !cached;
  if (__any_sync(0xffffffffu, need)) {  // most targets share the cached block
    const unsigned long long key = need ? block_key(g, bx, by, bz) : 0ull;
    const uint32_t peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    long long r = -1;
    if (need && lane == leader) r = claim_probe(C, key, insert);
    __syncwarp();
    if (need && lane == leader && r <= -2) r = claim_wait(C, (uint32_t)(-2 - r));
    r = __shfl_sync(0xffffffffu, r, leader);
    if (need) {
      bc.bx = bx;
      bc.by = by;
      bc.bz = bz;
      bc.b = r;
    }
  }
  if (!have || bc.b < 0) return nullptr;
  return block_word(C, bc.b, tx, ty, tz, shift);
}

// Lookup only, by one thread (no waiting; for use after the inserting kernel).
__device__ inline uint32_t* claim_lookup(const Claims& C, int g, int tx, int ty, int tz,
                                         int& shift, BlockCache& bc) {
  if (!site_in_range(tx, ty, tz)) return nullptr;
  const int bx = tx >> 3, by = ty >> 3, bz = tz >> 3;
  if (bx != bc.bx || by != bc.by || bz != bc.bz) {
    const int64_t r = claim_probe(C, block_key(g, bx, by, bz), false);
    bc.bx = bx;
    bc.by = by;
    bc.bz = bz;
    bc.b = r < 0 ? -1 : r;
  }
  if (bc.b < 0) return nullptr;
  return block_word(C, bc.b, tx, ty, tz, shift);
}

// ---------------------------------------------------------------------------------
// reached lattice sites: append-only list, linked per hash cell for range queries
// ---------------------------------------------------------------------------------
// an entry of the reached-site list whose site has melted (never a packed site: the
// grain field would exceed every grain id)
constexpr unsigned long long kDeadSite = ~0ull;

struct Reached {
  unsigned long long* key;  // packed (grain, site)
  uint32_t* next;           // next entry in the same cell, 0xFFFFFFFF ends
  uint32_t* head;           // per hash cell
  unsigned long long* count;
  unsigned long long cap;
  uint32_t* err;
};

__host__ __device__ __forceinline__ unsigned long long pack_site(int g, int sx, int sy, int sz) {
  return ((unsigned long long)(uint32_t)g << 39) |
         ((unsigned long long)(uint32_t)(sx + 4096) << 26) |
         ((unsigned long long)(uint32_t)(sy + 4096) << 13) | (unsigned long long)(uint32_t)(sz + 4096);
}
__host__ __device__ __forceinline__ void unpack_site(unsigned long long k, int& g, int& sx, int& sy,
                                                     int& sz) {
  g = (int)(k >> 39);
  sx = (int)((k >> 26) & 8191) - 4096;
  sy = (int)((k >> 13) & 8191) - 4096;
  sz = (int)(k & 8191) - 4096;
}

// ---------------------------------------------------------------------------------
// device counters
// ---------------------------------------------------------------------------------
struct DevStats {
  unsigned long long particle_steps;
  unsigned long long frozen_new;
  unsigned long long spawned;
  unsigned long long claims_lost;
  unsigned long long clipped;
  unsigned long long clamped;
  unsigned long long nucleated;
  unsigned long long n_out;        // particles written by the last emit
  unsigned long long n_frozen;     // FROZEN among them
  unsigned long long n_grains;
  unsigned long long reached;      // reached-site count (== Reached::count target)
  unsigned long long claim_used;   // occupied claim buckets
  unsigned long long n_live;       // after nucleation
  uint32_t err;
  uint32_t n_actx;                 // ACTIVE particles listed from the back of the list
  unsigned long long linked;       // reached sites linked into the per-cell lists
  unsigned long long n_act;        // ACTIVE particles listed by the last build
  unsigned long long step;         // batch: index n of the step being computed
  unsigned long long stamp;        // batch: cell-table stamp of the current build
  unsigned long long melted;       // reached sites melted (cumulative)
  unsigned long long walkback;     // particles re-activated by the walk-back (cumulative)
  unsigned long long n_dormant;    // grains melted entirely whose seed waits
  unsigned long long n_mlist;      // sites melted by the last melting pass
  unsigned long long removed;      // particles removed by the last melting pass
  unsigned long long renucleated;  // re-nucleations of dormant seeds (cumulative)
  unsigned long long obs_new;      // FROZEN records listed by the last obstacle flush
};

// ---------------------------------------------------------------------------------
// obstacle store of a single run.  A FROZEN particle never moves again (Sec. 2.1.2:
// points of two grains that meet stop for good and form the grain boundary), so its
// record need not be regrouped, gathered and re-emitted every step.  Flushes move the
// FROZEN records into an obstacle store ordered by cell key (records, positions, keys);
// every step's ordering copies the obstacles' positions and keys into the cell-ordered
// sequence that the contact search reads, beside the moving records.
// ---------------------------------------------------------------------------------

// warp-aggregated 64-bit counter increment
__device__ __forceinline__ void warp_add(unsigned long long* ctr, unsigned int v) {
  unsigned int m = __activemask();
  unsigned int s = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(m, s, o);
  // all active lanes hold the sum only if m is full; fall back to per-lane atomics
  if (m == 0xffffffffu) {
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(ctr, (unsigned long long)s);
  } else if (v) {
    atomicAdd(ctr, (unsigned long long)v);
  }
}

// ---------------------------------------------------------------------------------
// host-side launchers (defined in the .cu files)
// ---------------------------------------------------------------------------------
// kernel ids for the optional CUDA-event timing
enum KernelId : int {
  K_HIST = 0, K_ONESWEEP, K_KEYS, K_BUILD, K_ADVANCE, K_EMIT, K_NUCLEATE, K_GRAIN_MAP,
  K_SEED, K_CONTACT, K_CELLS, K_FINALIZE, K_GROUP, K_OBS, K_COUNT
};

struct ProfHook {
  virtual void begin(int kid) = 0;
  // kernels: how many kernel launches the timed segment holds
  virtual void end(int kid, double units, int kernels = 1) = 0;
  virtual ~ProfHook() {}
};

struct SortBufs {
  void* keys[2];             // uint32 or uint64 keys, per the instantiation of radix_sort
  uint32_t* vals[2];
  uint32_t* status;          // look-back words: max_tiles * 256
  uint32_t* hist;            // kSortMaxPasses * 256
  uint32_t* ticket;          // kSortMaxPasses counters
  uint32_t* err;
  int64_t max_n;
  int sms;
  ProfHook* prof;
  // device-sized sort: the key count is read from *n_dev when the kernels run
  // (persistent CTAs, look-back words cleared for max_n keys), so that the launches
  // need no host round trip and can be captured in a CUDA graph
  const unsigned long long* n_dev;
};

constexpr int kSortThreads = 256;
constexpr int kSortMaxPasses = 5;   // keys of up to 40 bits
template <class K> struct SortTile;
// keys per thread, keys per tile and resident CTAs per SM of a onesweep pass
template <> struct SortTile<uint32_t> {
  static constexpr int items = 12, tile = 256 * 12, ctas = 6;
};
template <> struct SortTile<uint64_t> {
  static constexpr int items = 10, tile = 256 * 10, ctas = 4;
};

// radix sort of (keys[0], vals[0]) over the low nbits of the keys; returns the
// buffer index (0 or 1) holding the sorted result, or -1 if nbits exceeds the
// key type or kSortMaxPasses digits.
template <class K>
int radix_sort(const SortBufs& B, int64_t n, int nbits, cudaStream_t st);
size_t radix_status_words(int64_t n, int key_bytes);  // look-back words for n keys

}  // namespace gp
