// Step kernels of the grain-envelope particle library (sm_103a).
//
// Per timestep (all on the context stream):
//   k_keys      cell keys of the store (only after host-side edits; the emit
//               kernel writes them otherwise)
//   radix sort  (key, store index), gp_sort.cu
//   k_build     gather the store into cell order, positions + grain as float4,
//               dense cell table (start, count) stamped with the build number
//   k_advance   contact freeze over the 27 neighbour cells, thermal sample,
//               growth law, explicit Euler advance, spawn claims
//   k_emit      claim resolution, reached sites, domain clip, compaction of the
//               surviving particles and their children (single-pass scan with
//               decoupled look-back), next-step cell keys
//   k_nucleate  nucleation activation at t_{n+1}
// plus seeding, state decode, grain-id voxelisation and the stand-alone
// hash / contact entry points.
#include "gp_kernels.cuh"

namespace gp {

namespace {

constexpr unsigned long long kF64Agg = 1ull << 62;
constexpr unsigned long long kF64Inc = 2ull << 62;
constexpr unsigned long long kV64Mask = (1ull << 62) - 1;
constexpr uint32_t kNoEntry = 0xffffffffu;

// ---------------------------------------------------------------------------------
// shared helpers
// ---------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long cell_entry(uint32_t stamp, uint32_t cnt,
                                                         uint32_t start) {
  return ((unsigned long long)stamp << 48) | ((unsigned long long)cnt << 32) | start;
}

// [start, end) of the sorted particles in cells x0..x1 of one row; false if empty
__device__ __forceinline__ bool row_range(const unsigned long long* __restrict__ tab,
                                          uint32_t stamp, size_t rowbase, int x0, int x1,
                                          uint32_t& start, uint32_t& end) {
  bool any = false;
  for (int x = x0; x <= x1; ++x) {
    unsigned long long e = __ldg(tab + rowbase + x);
    if ((uint32_t)(e >> 48) != stamp) continue;
    uint32_t s = (uint32_t)e;
    uint32_t c = (uint32_t)(e >> 32) & 0xffffu;
    if (!any) start = s;
    end = s + c;
    any = true;
  }
  return any;
}

__device__ __forceinline__ void reached_append(const Reached& R, const Params& P, int g, int sx,
                                               int sy, int sz, float3 sp) {
  unsigned long long r = atomicAdd(R.count, 1ull);
  if (r >= R.cap) {
    atomicOr(R.err, ERR_REACHED_CAP);
    return;
  }
  int cx, cy, cz;
  uint32_t key = cell_key(P, sp, cx, cy, cz);
  R.key[r] = pack_site(g, sx, sy, sz);
  R.next[r] = atomicExch(R.head + key, (uint32_t)r);
}

// nearest reached site strictly closer than sqrt(rc2); ties to the smaller grain.
// Returns the grain or -1.  If any_only, returns on the first hit.
__device__ int nearest_reached(const Params& P, const Reached& R, float3 p, bool any_only) {
  int c[3];
  c[0] = __float2int_rd(__fmul_rn(__fsub_rn(p.x, P.lo[0]), P.inv_c));
  c[1] = __float2int_rd(__fmul_rn(__fsub_rn(p.y, P.lo[1]), P.inv_c));
  c[2] = __float2int_rd(__fmul_rn(__fsub_rn(p.z, P.lo[2]), P.inv_c));
  float best = P.rc2;
  int bg = -1;
  unsigned long long guard = *R.count + 1;
  for (int dz = -1; dz <= 1; ++dz) {
    int z = min(max(c[2] + dz, 0), P.nc[2] - 1);
    if (dz > -1 && z == min(max(c[2] + dz - 1, 0), P.nc[2] - 1)) continue;  // clamped repeat
    for (int dy = -1; dy <= 1; ++dy) {
      int y = min(max(c[1] + dy, 0), P.nc[1] - 1);
      if (dy > -1 && y == min(max(c[1] + dy - 1, 0), P.nc[1] - 1)) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        int x = min(max(c[0] + dx, 0), P.nc[0] - 1);
        if (dx > -1 && x == min(max(c[0] + dx - 1, 0), P.nc[0] - 1)) continue;
        uint32_t key = (uint32_t)(((uint64_t)z * P.nc[1] + y) * P.nc[0] + x);
        uint32_t r = R.head[key];
        unsigned long long steps = 0;
        while (r != kNoEntry && steps++ < guard) {
          int g, sx, sy, sz;
          unpack_site(R.key[r], g, sx, sy, sz);
          float4 gc, r0, r1, r2;
          grain_load(P.gtab, g, gc, r0, r1, r2);
          float3 q = site_pos_g(gc, r0, r1, r2, sx, sy, sz);
          float d2 = dist2_rn(p, q);
          if (d2 < P.rc2) {
            if (any_only) return g;
            if (d2 < best || (d2 == best && g < bg)) {
              best = d2;
              bg = g;
            }
          }
          r = R.next[r];
        }
      }
    }
  }
  return bg;
}

// block-wide exclusive scan of one uint32 per thread (blockDim.x == 256)
__device__ __forceinline__ uint32_t bscan256(uint32_t v, uint32_t* s_warp, uint32_t& total) {
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
    if (lane < 8) s_warp[lane] = w;
  }
  __syncthreads();
  uint32_t r = (warp ? s_warp[warp - 1] : 0) + x - v;
  total = s_warp[7];
  __syncthreads();
  return r;
}

// decoupled look-back of a 64-bit tile aggregate (called by warp 0 of the CTA);
// returns the exclusive prefix of this tile.
__device__ unsigned long long lookback64(unsigned long long* status, uint32_t tile,
                                         unsigned long long agg, uint32_t* err) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) {
    if (lane == 0) atomicExch(status, kF64Inc | agg);
    return 0;
  }
  if (lane == 0) atomicExch(status + tile, kF64Agg | agg);
  unsigned long long excl = 0;
  long long pred = (long long)tile - 1;
  uint32_t spins = 0;
  while (true) {
    long long idx = pred - lane;
    unsigned long long s = 2ull << 62;  // before tile 0: an inclusive prefix of 0
    if (idx >= 0) s = *((volatile unsigned long long*)(status + idx));
    unsigned long long flag = s & ~kV64Mask;
    if (__any_sync(0xffffffffu, flag == 0ull)) {
      if (++spins > kSpinLimit) {
        if (lane == 0) atomicOr(err, ERR_TIMEOUT);
        break;
      }
      continue;
    }
    uint32_t inc = __ballot_sync(0xffffffffu, flag == kF64Inc);
    unsigned long long v = s & kV64Mask;
    int first = inc ? __ffs(inc) - 1 : 32;
    if (lane > first) v = 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (inc) break;
    pred -= 32;
  }
  if (lane == 0) atomicExch(status + tile, kF64Inc | ((excl + agg) & kV64Mask));
  return excl;
}

// ---------------------------------------------------------------------------------
// k_keys: cell key and identity value of every stored particle
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_keys(Params P, const int4* __restrict__ rec, int64_t n,
                                              uint32_t* __restrict__ keys,
                                              uint32_t* __restrict__ vals) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Rec r = rec_unpack(__ldg(rec + i));
  float3 p = part_pos(P.gtab, r.grain, r.sx, r.sy, r.sz, r.dir, r.ell);
  int cx, cy, cz;
  keys[i] = cell_key(P, p, cx, cy, cz);
  vals[i] = (uint32_t)i;
}

// ---------------------------------------------------------------------------------
// k_build: sorted store, sorted positions, cell table
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_build(Params P, const uint32_t* __restrict__ skeys,
                                               const uint32_t* __restrict__ svals,
                                               const int4* __restrict__ rin,
                                               int4* __restrict__ rout, float4* __restrict__ pos4,
                                               unsigned long long* __restrict__ tab,
                                               uint32_t stamp, int64_t n, uint32_t ncells,
                                               uint32_t* err) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint32_t id = __ldg(svals + j);
  const uint32_t key = __ldg(skeys + j);
  if ((int64_t)id >= n || key >= ncells) {  // only after a failed sort
    atomicOr(err, ERR_TIMEOUT);
    return;
  }
  const int4 rv = __ldg(rin + id);
  rout[j] = rv;
  Rec r = rec_unpack(rv);
  float3 p = part_pos(P.gtab, r.grain, r.sx, r.sy, r.sz, r.dir, r.ell);
  pos4[j] = make_float4(p.x, p.y, p.z, __int_as_float(r.grain));
  if (j == 0 || __ldg(skeys + j - 1) != key) {
    uint32_t c = 1;
    while (j + c < n && __ldg(skeys + j + c) == key) {
      if (++c == 0xffffu) {
        atomicOr(err, ERR_CELL_OVERFLOW);
        break;
      }
    }
    tab[key] = cell_entry(stamp, c, (uint32_t)j);
  }
}

// ---------------------------------------------------------------------------------
// k_advance: contact freeze, growth, advance, spawn claims (sorted store, in place)
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_advance(Params P, StepArgs S, int4* __restrict__ rs,
                                                 const float4* __restrict__ pos4,
                                                 const unsigned long long* __restrict__ tab,
                                                 uint32_t stamp, int64_t n, Claims C,
                                                 DevStats* st) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool active = false, froze = false, clamped = false;
  if (j < n) {
    Rec r = rec_unpack(rs[j]);
    if (r.state == ST_ACTIVE) {
      active = true;
      const float4 q = __ldg(pos4 + j);
      const float3 p = make_float3(q.x, q.y, q.z);
      const int g = r.grain;
      int cx, cy, cz;
      cell_key(P, p, cx, cy, cz);
      const int x0 = max(cx - 1, 0), x1 = min(cx + 1, P.nc[0] - 1);
      bool hit = false;
      for (int dz = -1; dz <= 1 && !hit; ++dz) {
        const int z = cz + dz;
        if (z < 0 || z >= P.nc[2]) continue;
        for (int dy = -1; dy <= 1 && !hit; ++dy) {
          const int y = cy + dy;
          if (y < 0 || y >= P.nc[1]) continue;
          uint32_t s0, s1;
          if (!row_range(tab, stamp, ((size_t)z * P.nc[1] + y) * P.nc[0], x0, x1, s0, s1))
            continue;
          if ((int64_t)s1 > n) s1 = (uint32_t)n;
          for (uint32_t i = s0; i < s1; ++i) {
            const float4 o = __ldg(pos4 + i);
            if (__float_as_int(o.w) == g) continue;
            if (dist2_rn(p, make_float3(o.x, o.y, o.z)) < P.rc2) {
              hit = true;
              break;
            }
          }
        }
      }
      if (hit) {
        froze = true;
        r.state = ST_FROZEN;
      } else {
        // thermal sample at (x_n, t_n), growth law, explicit Euler step of ell
        const float dT = undercooling(P, S, p);
        float dl = __fmul_rn(growth_v(P, dT), P.dt_over_h);
        if (dl > 1.f) {
          dl = 1.f;
          clamped = true;
        }
        const float e = __fadd_rn(r.ell, dl);
        // the target is reached within 2^-20 of a full spacing, so a step
        // commensurate with h does not lose a step to binary32 rounding
        if (e >= 1.f - 0x1p-20f) {
          r.cross = 1;
          r.ell = fmaxf(__fsub_rn(e, 1.f), 0.f);
          int sx = r.sx, sy = r.sy, sz = r.sz;
          step_site(sx, sy, sz, r.dir);
          for (int k = 0; k < 6; ++k) {
            if (!is_outer(sx, sy, sz, k)) continue;
            int tx = sx, ty = sy, tz = sz;
            step_site(tx, ty, tz, k);
            int sh;
            uint32_t* w = claim_word(C, g, tx, ty, tz, true, sh);
            if (w) atomicOr(w, (1u << ((k >> 1) + 3 * S.parity)) << sh);
          }
        } else {
          r.ell = e;
        }
      }
      rs[j] = rec_pack(r);
    }
  }
  warp_add(&st->particle_steps, active ? 1u : 0u);
  warp_add(&st->frozen_new, froze ? 1u : 0u);
  warp_add(&st->clamped, clamped ? 1u : 0u);
}

// ---------------------------------------------------------------------------------
// k_emit: claim resolution, reached sites, clip, compaction, next keys
// ---------------------------------------------------------------------------------
constexpr int kEmitItems = 4;
constexpr int kEmitTile = 256 * kEmitItems;

__global__ void __launch_bounds__(256) k_emit(Params P, StepArgs S, const int4* __restrict__ rs,
                                              int64_t n, int4* __restrict__ rout,
                                              uint32_t* __restrict__ keys,
                                              uint32_t* __restrict__ vals, int64_t cap,
                                              Claims C, Reached R,
                                              unsigned long long* status, uint32_t* ticket,
                                              uint32_t ntiles, DevStats* st) {
  __shared__ uint32_t s_warp[8];
  __shared__ uint32_t s_tile;
  __shared__ unsigned long long s_base;
  const int tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t base = (int64_t)tile * kEmitTile;

  // phase A: decide what every record emits.  mask bit 6 = the record itself,
  // bits 0..5 = children in direction k.
  uint32_t mask[kEmitItems];
  Rec rec[kEmitItems];
  uint32_t n_frozen = 0, n_spawn = 0, n_lost = 0, n_clip = 0;
#pragma unroll
  for (int it = 0; it < kEmitItems; ++it) {
    const int64_t j = base + it * 256 + tid;
    mask[it] = 0;
    if (j >= n) continue;
    Rec r = rec_unpack(__ldg(rs + j));
    rec[it] = r;
    if (r.state == ST_FROZEN) {
      mask[it] = 1u << 6;
      ++n_frozen;
      continue;
    }
    if (r.state != ST_ACTIVE) continue;
    float4 gc, r0, r1, r2;
    grain_load(P.gtab, r.grain, gc, r0, r1, r2);
    if (!r.cross) {
      float3 p = add_dir(site_pos_g(gc, r0, r1, r2, r.sx, r.sy, r.sz), r0, r1, r2, r.dir, r.ell);
      if (inside(P, p)) mask[it] = 1u << 6;
      else ++n_clip;
      continue;
    }
    int sx = r.sx, sy = r.sy, sz = r.sz;
    step_site(sx, sy, sz, r.dir);
    const float3 sp = site_pos_g(gc, r0, r1, r2, sx, sy, sz);
    reached_append(R, P, r.grain, sx, sy, sz, sp);
    for (int k = 0; k < 6; ++k) {
      if (!is_outer(sx, sy, sz, k)) continue;
      int tx = sx, ty = sy, tz = sz;
      step_site(tx, ty, tz, k);
      int sh;
      uint32_t* w = claim_word(C, r.grain, tx, ty, tz, false, sh);
      bool win = false;
      if (w) {
        const uint32_t byte = (*((volatile uint32_t*)w) >> sh) & 0xffu;
        const uint32_t live = (byte >> (3 * S.parity)) & 7u;
        win = !(byte & 0x80u) && live && (__ffs(live) - 1) == (k >> 1);
        if (win) atomicOr(w, 0x80u << sh);
      }
      if (!win) {
        ++n_lost;
        continue;
      }
      if (k != r.dir) ++n_spawn;
      const float3 cp = add_dir(sp, r0, r1, r2, k, r.ell);
      if (inside(P, cp)) mask[it] |= 1u << k;
      else ++n_clip;
    }
  }

  // phase B: offsets.  Output order within the tile is (item, thread).
  uint32_t ofs[kEmitItems];
  uint32_t run = 0;
#pragma unroll
  for (int it = 0; it < kEmitItems; ++it) {
    uint32_t tot;
    ofs[it] = run + bscan256((uint32_t)__popc(mask[it]), s_warp, tot);
    run += tot;
  }
  if (tid < 32) {
    unsigned long long excl = lookback64(status, tile, run, st == nullptr ? nullptr : &st->err);
    if (tid == 0) {
      s_base = excl;
      if (tile == ntiles - 1) {
        st->n_out = excl + run;
        if (excl + run > (unsigned long long)cap) atomicOr(&st->err, ERR_CAPACITY);
      }
    }
  }
  __syncthreads();
  const unsigned long long obase = s_base;

  // phase C: write the records and next-step keys
  for (int it = 0; it < kEmitItems; ++it) {
    uint32_t m = mask[it];
    if (!m) continue;
    unsigned long long o = obase + ofs[it];
    const Rec r = rec[it];
    float4 gc, r0, r1, r2;
    grain_load(P.gtab, r.grain, gc, r0, r1, r2);
    if (m & (1u << 6)) {
      if (o < (unsigned long long)cap) {
        Rec w = r;
        w.cross = 0;
        rout[o] = rec_pack(w);
        float3 p = add_dir(site_pos_g(gc, r0, r1, r2, r.sx, r.sy, r.sz), r0, r1, r2, r.dir, r.ell);
        int cx, cy, cz;
        keys[o] = cell_key(P, p, cx, cy, cz);
        vals[o] = (uint32_t)o;
      }
      continue;
    }
    int sx = r.sx, sy = r.sy, sz = r.sz;
    step_site(sx, sy, sz, r.dir);
    const float3 sp = site_pos_g(gc, r0, r1, r2, sx, sy, sz);
    for (int k = 0; k < 6; ++k) {
      if (!(m & (1u << k))) continue;
      if (o < (unsigned long long)cap) {
        Rec w;
        w.grain = r.grain;
        w.sx = sx;
        w.sy = sy;
        w.sz = sz;
        w.dir = k;
        w.state = ST_ACTIVE;
        w.cross = 0;
        w.ell = r.ell;
        rout[o] = rec_pack(w);
        float3 p = add_dir(sp, r0, r1, r2, k, r.ell);
        int cx, cy, cz;
        keys[o] = cell_key(P, p, cx, cy, cz);
        vals[o] = (uint32_t)o;
      }
      ++o;
    }
  }
  warp_add(&st->n_frozen, n_frozen);
  warp_add(&st->spawned, n_spawn);
  warp_add(&st->claims_lost, n_lost);
  warp_add(&st->clipped, n_clip);
}

// ---------------------------------------------------------------------------------
// k_nucleate: one CTA; activation test for every pending site against the state
// after the emit, then activation in registration order.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_nucleate(Params P, StepArgs S1, const float4* npos,
                                                  const float4* ngrain, int* nstate, int m,
                                                  float4* gtab, int max_grains, int4* rout,
                                                  uint32_t* keys, uint32_t* vals, int64_t cap,
                                                  Claims C, Reached R, DevStats* st) {
  __shared__ uint32_t s_warp[8];
  __shared__ uint32_t s_run;
  // phase 1: candidates (nstate: 0 pending, 1 candidate, 2 done)
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    if (nstate[j] != 0) continue;
    const float4 q = npos[j];
    const float3 p = make_float3(q.x, q.y, q.z);
    if (undercooling(P, S1, p) >= q.w && nearest_reached(P, R, p, true) < 0) nstate[j] = 1;
  }
  __threadfence_block();
  __syncthreads();
  if (threadIdx.x == 0) s_run = 0;
  __syncthreads();
  const unsigned long long nout = st->n_out;
  const unsigned long long g0 = st->n_grains;
  for (int c0 = 0; c0 < m; c0 += blockDim.x) {
    const int j = c0 + threadIdx.x;
    const uint32_t cand = (j < m && nstate[j] == 1) ? 1u : 0u;
    uint32_t tot;
    const uint32_t rank = bscan256(cand, s_warp, tot) + s_run;
    if (cand) {
      nstate[j] = 2;
      const unsigned long long g = g0 + rank;
      if (g >= (unsigned long long)max_grains) {
        atomicOr(&st->err, ERR_GRAINS);
      } else {
        for (int q = 0; q < 4; ++q) gtab[4 * g + q] = ngrain[4 * j + q];
        const float4 cq = ngrain[4 * j];
        const float3 c = make_float3(cq.x, cq.y, cq.z);
        // nucleus site reached and claimed; six first targets claimed
        unsigned long long r = atomicAdd(R.count, 1ull);
        if (r < R.cap) {
          int cx, cy, cz;
          uint32_t key = cell_key(P, c, cx, cy, cz);
          R.key[r] = pack_site((int)g, 0, 0, 0);
          R.next[r] = atomicExch(R.head + key, (uint32_t)r);
        } else {
          atomicOr(R.err, ERR_REACHED_CAP);
        }
        int sh;
        uint32_t* w = claim_word(C, (int)g, 0, 0, 0, true, sh);
        if (w) atomicOr(w, 0x80u << sh);
        int cx, cy, cz;
        const uint32_t key = cell_key(P, c, cx, cy, cz);
        for (int k = 0; k < 6; ++k) {
          int tx = 0, ty = 0, tz = 0;
          step_site(tx, ty, tz, k);
          w = claim_word(C, (int)g, tx, ty, tz, true, sh);
          if (w) atomicOr(w, 0x80u << sh);
          const unsigned long long o = nout + 6ull * rank + k;
          if (o < (unsigned long long)cap) {
            Rec rr;
            rr.grain = (int)g;
            rr.sx = rr.sy = rr.sz = 0;
            rr.dir = k;
            rr.state = ST_ACTIVE;
            rr.cross = 0;
            rr.ell = 0.f;
            rout[o] = rec_pack(rr);
            keys[o] = key;
            vals[o] = (uint32_t)o;
          } else {
            atomicOr(&st->err, ERR_CAPACITY);
          }
        }
      }
    }
    if (threadIdx.x == 0) s_run += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    unsigned long long add = s_run;
    unsigned long long ng = g0 + add;
    st->n_grains = ng > (unsigned long long)max_grains ? (unsigned long long)max_grains : ng;
    st->nucleated += add;
    unsigned long long nl = nout + 6ull * add;
    st->n_live = nl > (unsigned long long)cap ? (unsigned long long)cap : nl;
  }
}

__global__ void k_finalize(DevStats* st, int64_t cap) {
  unsigned long long nl = st->n_out;
  st->n_live = nl > (unsigned long long)cap ? (unsigned long long)cap : nl;
}

// ---------------------------------------------------------------------------------
// seeding
// ---------------------------------------------------------------------------------
// appends m records given on the device at store positions base..base+m-1
__global__ void k_append(const int4* __restrict__ src, int64_t m, int4* __restrict__ rout,
                         int64_t base) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) rout[base + i] = src[i];
}

// marks m sites (grain, s) reached and/or claimed
__global__ void k_mark_sites(Params P, const int4* __restrict__ sites, int64_t m, int reached,
                             int claimed, Claims C, Reached R) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int4 s = sites[i];
  if (claimed) {
    int sh;
    uint32_t* w = claim_word(C, s.x, s.y, s.z, s.w, true, sh);
    if (w) atomicOr(w, 0x80u << sh);
  }
  if (reached) {
    float4 gc, r0, r1, r2;
    grain_load(P.gtab, s.x, gc, r0, r1, r2);
    reached_append(R, P, s.x, s.y, s.z, s.w, site_pos_g(gc, r0, r1, r2, s.y, s.z, s.w));
  }
}

// shell seeding: for every (grain, target offset t with |t|_1 = n0 + 1) one ACTIVE
// particle at the site reached from the lowest axis with t_a != 0.
__global__ void k_seed_shell(Params P, const int32_t* __restrict__ grains, int64_t ng,
                             const short4* __restrict__ toff, int64_t nt, float ell0,
                             int4* __restrict__ rout, int64_t cap, unsigned long long* counter,
                             Claims C, uint32_t* err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ng * nt) return;
  const int g = grains[i / nt];
  const short4 t = toff[i % nt];
  int ts[3] = {t.x, t.y, t.z};
  int a = ts[0] != 0 ? 0 : (ts[1] != 0 ? 1 : 2);
  int sg = ts[a] > 0 ? 1 : -1;
  int s[3] = {ts[0], ts[1], ts[2]};
  s[a] -= sg;
  const int dir = 2 * a + (sg > 0 ? 0 : 1);
  float3 p = part_pos(P.gtab, g, s[0], s[1], s[2], dir, ell0);
  if (!inside(P, p)) return;
  unsigned long long o = atomicAdd(counter, 1ull);
  if (o >= (unsigned long long)cap) {
    atomicOr(err, ERR_CAPACITY);
    return;
  }
  Rec r;
  r.grain = g;
  r.sx = s[0];
  r.sy = s[1];
  r.sz = s[2];
  r.dir = dir;
  r.state = ST_ACTIVE;
  r.cross = 0;
  r.ell = ell0;
  rout[o] = rec_pack(r);
  int sh;
  uint32_t* w = claim_word(C, g, ts[0], ts[1], ts[2], true, sh);
  if (w) atomicOr(w, 0x80u << sh);
}

// reached + claimed shell sites |s|_1 = n0 of every listed grain
__global__ void k_seed_shell_sites(Params P, const int32_t* __restrict__ grains, int64_t ng,
                                   const short4* __restrict__ soff, int64_t ns, Claims C,
                                   Reached R) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ng * ns) return;
  const int g = grains[i / ns];
  const short4 s = soff[i % ns];
  int sh;
  uint32_t* w = claim_word(C, g, s.x, s.y, s.z, true, sh);
  if (w) atomicOr(w, 0x80u << sh);
  float4 gc, r0, r1, r2;
  grain_load(P.gtab, g, gc, r0, r1, r2);
  reached_append(R, P, g, s.x, s.y, s.z, site_pos_g(gc, r0, r1, r2, s.x, s.y, s.z));
}

// ---------------------------------------------------------------------------------
// state decode, grain map
// ---------------------------------------------------------------------------------
__global__ void k_positions(Params P, const int4* __restrict__ rec, int64_t n,
                            float* __restrict__ x3) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Rec r = rec_unpack(rec[i]);
  float3 p = part_pos(P.gtab, r.grain, r.sx, r.sy, r.sz, r.dir, r.ell);
  x3[3 * i] = p.x;
  x3[3 * i + 1] = p.y;
  x3[3 * i + 2] = p.z;
}

__global__ void k_grain_map(Params P, Reached R, double ox, double oy, double oz, double sx,
                            double sy, double sz, int nx, int ny, int nz, int32_t* out,
                            int64_t v0, int64_t nv) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  const int64_t v = v0 + i;
  const int ix = (int)(v % nx);
  const int iy = (int)((v / nx) % ny);
  const int iz = (int)(v / ((int64_t)nx * ny));
  float3 p = make_float3((float)(ox + (ix + 0.5) * sx), (float)(oy + (iy + 0.5) * sy),
                         (float)(oz + (iz + 0.5) * sz));
  out[i] = nearest_reached(P, R, p, false);
}

// ---------------------------------------------------------------------------------
// stand-alone hash / contact
// ---------------------------------------------------------------------------------
__global__ void k_keys_pos(Params P, const float* __restrict__ x3, const uint8_t* __restrict__ state,
                           int64_t n, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float3 p = make_float3(x3[3 * i], x3[3 * i + 1], x3[3 * i + 2]);
  int cx, cy, cz;
  uint32_t k = cell_key(P, p, cx, cy, cz);
  if (state && state[i] == ST_REMOVED) k = 0xffffffffu;
  keys[i] = k;
  vals[i] = (uint32_t)i;
}

// cell starts: flags[i] = 1 where a new key begins
__global__ void k_cell_flags(const uint32_t* __restrict__ keys, int64_t n, uint32_t* flags) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

// exclusive scan of flags (n <= 256 * 256 * 1024) into ofs; two-level, simple
__global__ void k_scan_blocks(const uint32_t* __restrict__ in, int64_t n, uint32_t* out,
                              uint32_t* bsum) {
  __shared__ uint32_t s_warp[8];
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t v = i < n ? in[i] : 0u;
  uint32_t tot;
  uint32_t e = bscan256(v, s_warp, tot);
  if (i < n) out[i] = e;
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}
__global__ void k_scan_sums(uint32_t* bsum, int64_t nb) {
  // single CTA, sequential over chunks of 256
  __shared__ uint32_t s_warp[8];
  __shared__ uint32_t s_run;
  if (threadIdx.x == 0) s_run = 0;
  __syncthreads();
  for (int64_t c = 0; c < nb; c += 256) {
    int64_t i = c + threadIdx.x;
    uint32_t v = i < nb ? bsum[i] : 0u;
    uint32_t tot;
    uint32_t e = bscan256(v, s_warp, tot);
    if (i < nb) bsum[i] = e + s_run;
    __syncthreads();
    if (threadIdx.x == 0) s_run += tot;
    __syncthreads();
  }
}
__global__ void k_cell_write(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ flags,
                             const uint32_t* __restrict__ ofs, const uint32_t* __restrict__ bsum,
                             int64_t n, uint32_t nvalid_key, uint32_t* cell_keys,
                             int32_t* cell_start, unsigned long long* ncell) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!flags[i]) return;
  if (keys[i] >= nvalid_key) return;
  uint32_t o = ofs[i] + bsum[i / 256];
  cell_keys[o] = keys[i];
  cell_start[o] = (int32_t)i;
  atomicAdd(ncell, 1ull);
}

__global__ void k_contact_sa(Params P, const float4* __restrict__ pos4,
                             const uint8_t* __restrict__ sstate, const uint32_t* __restrict__ ids,
                             const unsigned long long* __restrict__ tab, int64_t n,
                             uint8_t* freeze, int32_t* pairs, int64_t pair_cap,
                             unsigned long long* npairs) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint8_t stj = sstate[j];
  if (stj == ST_REMOVED) return;
  const float4 q = pos4[j];
  const float3 p = make_float3(q.x, q.y, q.z);
  const int g = __float_as_int(q.w);
  const uint32_t idj = ids[j];
  int cx, cy, cz;
  cell_key(P, p, cx, cy, cz);
  const int x0 = max(cx - 1, 0), x1 = min(cx + 1, P.nc[0] - 1);
  bool hit = false;
  for (int dz = -1; dz <= 1; ++dz) {
    const int z = cz + dz;
    if (z < 0 || z >= P.nc[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int y = cy + dy;
      if (y < 0 || y >= P.nc[1]) continue;
      uint32_t s0, s1;
      if (!row_range(tab, 1u, ((size_t)z * P.nc[1] + y) * P.nc[0], x0, x1, s0, s1)) continue;
      if ((int64_t)s1 > n) s1 = (uint32_t)n;
      for (uint32_t i = s0; i < s1; ++i) {
        if (sstate[i] == ST_REMOVED) continue;
        const float4 o = pos4[i];
        if (__float_as_int(o.w) == g) continue;
        if (!(dist2_rn(p, make_float3(o.x, o.y, o.z)) < P.rc2)) continue;
        hit = true;
        if (!pairs) break;
        const uint32_t idi = ids[i];
        if (idj < idi) {
          unsigned long long k = atomicAdd(npairs, 1ull);
          if ((int64_t)k < pair_cap) {
            pairs[2 * k] = (int32_t)idj;
            pairs[2 * k + 1] = (int32_t)idi;
          }
        }
      }
      if (hit && !pairs) break;
    }
    if (hit && !pairs) break;
  }
  if (freeze) freeze[idj] = (hit && stj == ST_ACTIVE) ? 1 : 0;
}

__global__ void k_build_sa(Params P, const float* __restrict__ x3, const int32_t* __restrict__ grain,
                           const uint8_t* __restrict__ state, const uint32_t* __restrict__ skeys,
                           const uint32_t* __restrict__ svals, int64_t n, float4* pos4,
                           uint8_t* sstate, unsigned long long* tab, uint32_t* err) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint32_t id = svals[j];
  if ((int64_t)id >= n) {  // only after a failed sort
    atomicOr(err, ERR_TIMEOUT);
    return;
  }
  pos4[j] = make_float4(x3[3 * id], x3[3 * id + 1], x3[3 * id + 2], __int_as_float(grain[id]));
  sstate[j] = state[id];
  const uint32_t key = skeys[j];
  if (key >= (uint32_t)((uint64_t)P.nc[0] * P.nc[1] * P.nc[2])) return;  // removed points
  if (j == 0 || skeys[j - 1] != key) {
    uint32_t c = 1;
    while (j + c < n && skeys[j + c] == key) {
      if (++c == 0xffffu) {
        atomicOr(err, ERR_CELL_OVERFLOW);
        break;
      }
    }
    tab[key] = cell_entry(1u, c, (uint32_t)j);
  }
}

inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------
void launch_keys(const Params& P, const int4* rec, int64_t n, uint32_t* keys, uint32_t* vals,
                 cudaStream_t st) {
  if (n > 0) k_keys<<<blocks(n), 256, 0, st>>>(P, rec, n, keys, vals);
}

void launch_build(const Params& P, const uint32_t* skeys, const uint32_t* svals, const int4* rin,
                  int4* rout, float4* pos4, unsigned long long* tab, uint32_t stamp, int64_t n,
                  uint32_t* err, cudaStream_t st) {
  const uint32_t ncells = (uint32_t)((uint64_t)P.nc[0] * P.nc[1] * P.nc[2]);
  if (n > 0)
    k_build<<<blocks(n), 256, 0, st>>>(P, skeys, svals, rin, rout, pos4, tab, stamp, n, ncells,
                                       err);
}

void launch_advance(const Params& P, const StepArgs& S, int4* rs, const float4* pos4,
                    const unsigned long long* tab, uint32_t stamp, int64_t n, const Claims& C,
                    DevStats* dst, cudaStream_t st) {
  if (n > 0) k_advance<<<blocks(n), 256, 0, st>>>(P, S, rs, pos4, tab, stamp, n, C, dst);
}

int64_t emit_tiles(int64_t n) { return (n + kEmitTile - 1) / kEmitTile; }

void launch_emit(const Params& P, const StepArgs& S, const int4* rs, int64_t n, int4* rout,
                 uint32_t* keys, uint32_t* vals, int64_t cap, const Claims& C, const Reached& R,
                 unsigned long long* status, uint32_t* ticket, DevStats* dst, cudaStream_t st) {
  const int64_t nt = emit_tiles(n);
  if (nt == 0) return;
  cudaMemsetAsync(status, 0, sizeof(unsigned long long) * nt, st);
  cudaMemsetAsync(ticket, 0, sizeof(uint32_t), st);
  k_emit<<<(unsigned)nt, 256, 0, st>>>(P, S, rs, n, rout, keys, vals, cap, C, R, status, ticket,
                                       (uint32_t)nt, dst);
}

void launch_nucleate(const Params& P, const StepArgs& S1, const float4* npos, const float4* ngrain,
                     int* nstate, int m, float4* gtab, int max_grains, int4* rout, uint32_t* keys,
                     uint32_t* vals, int64_t cap, const Claims& C, const Reached& R, DevStats* dst,
                     cudaStream_t st) {
  k_nucleate<<<1, 256, 0, st>>>(P, S1, npos, ngrain, nstate, m, gtab, max_grains, rout, keys,
                                vals, cap, C, R, dst);
}

void launch_finalize(DevStats* dst, int64_t cap, cudaStream_t st) {
  k_finalize<<<1, 1, 0, st>>>(dst, cap);
}

void launch_append(const int4* src, int64_t m, int4* rout, int64_t base, cudaStream_t st) {
  if (m > 0) k_append<<<blocks(m), 256, 0, st>>>(src, m, rout, base);
}

void launch_mark_sites(const Params& P, const int4* sites, int64_t m, int reached, int claimed,
                       const Claims& C, const Reached& R, cudaStream_t st) {
  if (m > 0) k_mark_sites<<<blocks(m), 256, 0, st>>>(P, sites, m, reached, claimed, C, R);
}

void launch_seed_shell(const Params& P, const int32_t* grains, int64_t ng, const short4* toff,
                       int64_t nt, float ell0, int4* rout, int64_t cap,
                       unsigned long long* counter, const Claims& C, uint32_t* err,
                       cudaStream_t st) {
  if (ng * nt > 0)
    k_seed_shell<<<blocks(ng * nt), 256, 0, st>>>(P, grains, ng, toff, nt, ell0, rout, cap,
                                                  counter, C, err);
}

void launch_seed_shell_sites(const Params& P, const int32_t* grains, int64_t ng,
                             const short4* soff, int64_t ns, const Claims& C, const Reached& R,
                             cudaStream_t st) {
  if (ng * ns > 0)
    k_seed_shell_sites<<<blocks(ng * ns), 256, 0, st>>>(P, grains, ng, soff, ns, C, R);
}

void launch_positions(const Params& P, const int4* rec, int64_t n, float* x3, cudaStream_t st) {
  if (n > 0) k_positions<<<blocks(n), 256, 0, st>>>(P, rec, n, x3);
}

void launch_grain_map(const Params& P, const Reached& R, const double o[3], const double s[3],
                      const int nvox[3], int32_t* out, int64_t v0, int64_t nv, cudaStream_t st) {
  if (nv > 0)
    k_grain_map<<<blocks(nv), 256, 0, st>>>(P, R, o[0], o[1], o[2], s[0], s[1], s[2], nvox[0],
                                            nvox[1], nvox[2], out, v0, nv);
}

void launch_keys_pos(const Params& P, const float* x3, const uint8_t* state, int64_t n,
                     uint32_t* keys, uint32_t* vals, cudaStream_t st) {
  if (n > 0) k_keys_pos<<<blocks(n), 256, 0, st>>>(P, x3, state, n, keys, vals);
}

void launch_cells(const uint32_t* skeys, int64_t n, uint32_t nvalid_key, uint32_t* flags,
                  uint32_t* ofs, uint32_t* bsum, uint32_t* cell_keys, int32_t* cell_start,
                  unsigned long long* ncell, cudaStream_t st) {
  if (n <= 0) return;
  const unsigned nb = blocks(n);
  k_cell_flags<<<nb, 256, 0, st>>>(skeys, n, flags);
  k_scan_blocks<<<nb, 256, 0, st>>>(flags, n, ofs, bsum);
  k_scan_sums<<<1, 256, 0, st>>>(bsum, nb);
  k_cell_write<<<nb, 256, 0, st>>>(skeys, flags, ofs, bsum, n, nvalid_key, cell_keys, cell_start,
                                   ncell);
}

void launch_build_sa(const Params& P, const float* x3, const int32_t* grain, const uint8_t* state,
                     const uint32_t* skeys, const uint32_t* svals, int64_t n, float4* pos4,
                     uint8_t* sstate, unsigned long long* tab, uint32_t* err, cudaStream_t st) {
  if (n > 0)
    k_build_sa<<<blocks(n), 256, 0, st>>>(P, x3, grain, state, skeys, svals, n, pos4, sstate, tab,
                                          err);
}

void launch_contact_sa(const Params& P, const float4* pos4, const uint8_t* sstate,
                       const uint32_t* ids, const unsigned long long* tab, int64_t n,
                       uint8_t* freeze, int32_t* pairs, int64_t pair_cap,
                       unsigned long long* npairs, cudaStream_t st) {
  if (n > 0)
    k_contact_sa<<<blocks(n), 256, 0, st>>>(P, pos4, sstate, ids, tab, n, freeze, pairs, pair_cap,
                                            npairs);
}

}  // namespace gp
