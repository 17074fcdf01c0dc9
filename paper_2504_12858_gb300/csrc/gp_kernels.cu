// Step kernels of the grain-envelope particle library (sm_103a).
//
// Per timestep (all on the context stream):
//   k_keys      cell keys of the store (only after host-side edits; the emit
//               kernel writes them otherwise)
//   ordering    one run: k_group_count, k_group_scatter, k_group_order and
//               k_group_gather group the records by tile of the cell order and order
//               them by cell inside each tile; a batch: radix sort of (key, store
//               index), gp_sort.cu, then k_build.  Either way the store lands in cell
//               order with positions + grain as float4, the segment table of the cell
//               runs (stamped with the build number) and the list of ACTIVE particles
//   k_advance   contact freeze over the 27 neighbour cells, thermal sample,
//               growth law, explicit Euler advance, spawn claims
//   k_emit      claim resolution, reached sites, domain clip, compaction of the
//               surviving particles and their children (block scan + one atomic
//               reservation per CTA), next-step cell keys
//   k_nucleate  nucleation activation at t_{n+1}
// plus seeding, state decode, grain-id voxelisation and the stand-alone
// hash / contact entry points.
#include <algorithm>

#include "gp_kernels.cuh"

namespace gp {

namespace {

constexpr uint32_t kNoEntry = 0xffffffffu;

// ---------------------------------------------------------------------------------
// shared helpers
// ---------------------------------------------------------------------------------
// Cell table.  The sorted particles of each run of kSegCells = 16 cells along x of
// one row of the hash grid ("segment") are contiguous.  The table holds one
// 16-byte entry per segment:
//   x: sorted index of the segment's first particle
//   y: build stamp (high 16 bits) | saturation flag (bit 15) | particle count of
//      the segment (low 15 bits)
//   z, w: particle count of each of the 16 cells, 4 bits each (cell 0 in the low
//         nibble of z), saturated at 15; the flag is set when any count saturates
// An entry whose stamp is not the current build's is an empty segment.  A query
// turns the 3 cells x-1..x+1 of a neighbour row into a candidate range directly
// from the nibble counts; when a count is saturated it scans the segment's keys.
// Two cell orders.  Linear (the stand-alone hash): local = (z ny + y) nx + x, segments
// of 16 cells along x, nsx per row.  Tiled (the particle step): tiles of 16 x 8 x 8
// cells in (z, y, x) order, x fastest inside a tile, so that a cell's nine neighbour
// rows are segments of one tile (or of its neighbours) and their particles lie close
// together in the sorted store: local = tile * 1024 + ((z & 7) * 8 + (y & 7)) * 16 +
// (x & 15), and the segment of a cell is local / 16.  On the 4 x 2 x 1 mm weld plate the
// step ran 15 % faster than with linear rows (build, emit and advance all gain from the
// 3D locality of consecutive records); 16 x 2 x 2 gained 7 %, 16 x 4 x 4 13 %, and
// 16 x 16 x 16 as much as 16 x 8 x 8.
// run-local segment of a run-local cell key (and the cell's x within its segment)
template <bool TILED>
__device__ __forceinline__ uint32_t seg_of(const Geo& g, uint32_t local, uint32_t& xcell) {
  if constexpr (TILED) {
    xcell = local & (kSegCells - 1);
    return local >> kSegShift;
  } else {
    const uint32_t row = local / (uint32_t)g.nc[0];
    xcell = local - row * (uint32_t)g.nc[0];
    return row * (uint32_t)g.nsx + (xcell >> kSegShift);
  }
}

template <bool TILED>
__device__ __forceinline__ uint32_t ncells_of(const Geo& g) {
  if constexpr (TILED)
    return (uint32_t)((uint64_t)g.tx * g.ty *
                      ((g.nc[2] + (1 << kTileZShift) - 1) >> kTileZShift)
                      << (kSegShift + kTileYShift + kTileZShift));
  else
    return (uint32_t)((uint64_t)g.nc[0] * g.nc[1] * g.nc[2]);
}

// tiled segment of neighbour row (y, z) in x segment sx16 (the tile column)
__device__ __forceinline__ uint32_t seg_tiled(const Geo& g, int sx16, int y, int z) {
  constexpr int ym = (1 << kTileYShift) - 1, zm = (1 << kTileZShift) - 1;
  return ((((uint32_t)(z >> kTileZShift) * (uint32_t)g.ty + (uint32_t)(y >> kTileYShift)) *
               (uint32_t)g.tx + (uint32_t)sx16) << (kTileYShift + kTileZShift)) |
         (uint32_t)(((z & zm) << kTileYShift) | (y & ym));
}

// tiled run-local cell of cell coordinates
__device__ __forceinline__ uint32_t local_tiled(const Geo& g, int cx, int cy, int cz) {
  return (seg_tiled(g, cx >> kSegShift, cy, cz) << kSegShift) | (uint32_t)(cx & (kSegCells - 1));
}

// Writes the entry of the segment that starts at sorted index j (if one does).
// The keys of the run are key0 + local; a key outside that range ends the run.
template <class K, bool TILED>
__device__ __forceinline__ void seg_build(const Geo& gm, const K* __restrict__ skeys, int64_t j,
                                          int64_t n, K key, uint4* __restrict__ tab,
                                          uint32_t stamp, uint32_t* err) {
  const K k0 = (K)gm.key0;
  const uint32_t nvalid = ncells_of<TILED>(gm);
  uint32_t x0;
  const uint32_t sg = seg_of<TILED>(gm, (uint32_t)(key - k0), x0);
  if (j > 0) {
    const K kp = __ldg(skeys + j - 1);
    uint32_t xp;
    if (kp >= k0 && (K)(kp - k0) < (K)nvalid && seg_of<TILED>(gm, (uint32_t)(kp - k0), xp) == sg)
      return;
  }
  unsigned long long nib = 0;
  uint32_t c = 0;
  K k = key;
  while (true) {
    uint32_t x;
    seg_of<TILED>(gm, (uint32_t)(k - k0), x);
    const int sh = 4 * (int)(x & (kSegCells - 1));
    if (((nib >> sh) & 15ull) < 15ull) nib += 1ull << sh;
    if (++c == kSegMaxCount) {
      atomicOr(err, ERR_CELL_OVERFLOW);
      break;
    }
    if (j + c >= n) break;
    k = __ldg(skeys + j + c);
    uint32_t xk;
    if (k < k0 || (K)(k - k0) >= (K)nvalid || seg_of<TILED>(gm, (uint32_t)(k - k0), xk) != sg)
      break;
  }
  const bool sat = ((nib & (nib >> 1) & (nib >> 2) & (nib >> 3)) & 0x1111111111111111ull) != 0;
  tab[gm.seg0 + sg] = make_uint4((uint32_t)j, (stamp << 16) | (sat ? 0x8000u : 0u) | c,
                                 (uint32_t)nib, (uint32_t)(nib >> 32));
}

// the eight 4-bit counts of v summed in pairs, one pair per byte (at most 30 each)
__device__ __forceinline__ uint32_t nib_pairs(uint32_t v) {
  return (v & 0x0f0f0f0fu) + ((v >> 4) & 0x0f0f0f0fu);
}
// sum of the four bytes of b (exact while that sum is below 256)
__device__ __forceinline__ uint32_t byte_sum(uint32_t b) { return (b * 0x01010101u) >> 24; }
// sum of the eight 4-bit counts in v
__device__ __forceinline__ uint32_t nib_sum8(uint32_t v) { return byte_sum(nib_pairs(v)); }
// mask of the low q 4-bit counts of a word (q >= 0)
__device__ __forceinline__ uint32_t low_nibbles(int q) {
  return q >= 8 ? 0xffffffffu : ((1u << (4 * q)) - 1u);
}
// sum of the 4-bit counts of cells 0..p-1 (p <= 16) of an entry's z (cells 0-7)
// and w (cells 8-15)
__device__ __forceinline__ uint32_t nib_prefix(uint32_t z, uint32_t w, int p) {
  return nib_sum8(z & low_nibbles(p)) + nib_sum8(w & low_nibbles(max(p - 8, 0)));
}

// Candidate range [i, end) of the cells c0..c1 of one row of a segment whose table entry
// is e: from the 4-bit counts (masks mz0/mw0 of the cells before c0, rz/rw of the cells
// c0..c1), or, when a count is saturated, by scanning the segment's keys for klo..khi.
// Returns false when the range is empty.
template <class K>
__device__ __forceinline__ bool row_range(const uint4 e, uint32_t mz0, uint32_t mw0, uint32_t rz,
                                          uint32_t rw, K klo, K khi, const K* __restrict__ skeys,
                                          int64_t n, uint32_t& i, uint32_t& end) {
  if (!(e.y & 0x8000u)) {
    const uint32_t cnt = byte_sum(nib_pairs(e.z & rz) + nib_pairs(e.w & rw));
    if (cnt == 0) return false;  // cells c0..c1 of this row are empty
    i = e.x + byte_sum(nib_pairs(e.z & mz0) + nib_pairs(e.w & mw0));
    end = i + cnt;
  } else {
    // a cell holds 15 or more particles: locate the cells by their keys
    i = e.x;
    end = e.x + (e.y & kSegMaxCount);
    while (i < end && __ldg(skeys + i) < klo) ++i;
    uint32_t e2 = i;
    while (e2 < end && __ldg(skeys + e2) <= khi) ++e2;
    end = e2;
  }
  if ((int64_t)end > n) end = (uint32_t)n;
  return i < end;
}

// Finds the sorted particles i of another grain strictly closer than the contact
// radius to p, among the particles of the 3x3x3 cells around (cx, cy, cz) of run
// geometry gm.  gw is the pos4.w word of the querying particle (grain and run):
// particles with the same word belong to the same grain.
// PAIRS == false: returns at the first one.  PAIRS == true: visits all of them and
// appends the pairs (idj, ids[i]) with idj < ids[i] to pairs (up to pair_cap,
// counted in *npairs).  Returns whether any was found.
template <bool PAIRS, class K, bool TILED>
__device__ __forceinline__ bool contact_scan(const Params& P, const Geo& gm,
                                             const uint4* __restrict__ tab, uint32_t stamp,
                                             const K* __restrict__ skeys,
                                             const float4* __restrict__ pos4, int64_t n,
                                             float3 p, int gw, int cx, int cy, int cz,
                                             const uint32_t* __restrict__ ids = nullptr,
                                             uint32_t idj = 0, int32_t* pairs = nullptr,
                                             int64_t pair_cap = 0,
                                             unsigned long long* npairs = nullptr) {
  bool hit = false;
  const int x0 = max(cx - 1, 0), x1 = min(cx + 1, gm.nc[0] - 1);
  const int y0 = max(cy - 1, 0), y1 = min(cy + 1, gm.nc[1] - 1);
  const int z0 = max(cz - 1, 0), z1 = min(cz + 1, gm.nc[2] - 1);
  const uint4* __restrict__ rtab = tab + gm.seg0;
  // segments outermost: the cells c0..c1 of a segment, and so the masks of the counts
  // before c0 and up to c1, are the same in all nine rows
  for (int sgi = x0 >> kSegShift; sgi <= (x1 >> kSegShift); ++sgi) {
    const int base = sgi << kSegShift;
    const int c0 = max(x0, base) - base, c1 = min(x1, base + kSegCells - 1) - base;
    const uint32_t mz0 = low_nibbles(c0), mw0 = low_nibbles(max(c0 - 8, 0));
    const uint32_t rz = low_nibbles(c1 + 1) & ~mz0, rw = low_nibbles(max(c1 - 7, 0)) & ~mw0;
    for (int z = z0; z <= z1; ++z) {
      for (int y = y0; y <= y1; ++y) {
        const uint32_t sg = TILED ? seg_tiled(gm, sgi, y, z)
                                  : ((uint32_t)z * (uint32_t)gm.nc[1] + (uint32_t)y) *
                                            (uint32_t)gm.nsx + (uint32_t)sgi;
        const K klo = (K)gm.key0 +
                      (K)(TILED ? (sg << kSegShift) + (uint32_t)c0
                                : ((uint32_t)z * (uint32_t)gm.nc[1] + (uint32_t)y) *
                                          (uint32_t)gm.nc[0] + (uint32_t)(base + c0));
        const K khi = klo + (K)(c1 - c0);
        const uint4 e = __ldg(rtab + sg);
        uint32_t i, end;
        if ((e.y >> 16) == stamp && row_range<K>(e, mz0, mw0, rz, rw, klo, khi, skeys, n, i, end)) {
          for (; i < end; ++i) {
            const float4 o = __ldg(pos4 + i);
            if (__float_as_int(o.w) == gw) continue;
            if (dist2_rn(p, make_float3(o.x, o.y, o.z)) < P.rc2) {
              if (!PAIRS) return true;
              hit = true;
              const uint32_t idi = ids[i];
              if (idj < idi) {
                const unsigned long long k = atomicAdd(npairs, 1ull);
                if ((int64_t)k < pair_cap) {
                  pairs[2 * k] = (int32_t)idj;
                  pairs[2 * k + 1] = (int32_t)idi;
                }
              }
            }
          }
        }
      }
    }
  }
  return hit;
}

// contact_scan (first hit only) for a single run with periodic axes: neighbour rows
// and cells wrap around the periodic faces and distances take the nearest image.
// With at least three cells per periodic axis the 27 cells are distinct.
template <class K>
__device__ bool contact_scan_per(const Params& P, const Geo& gm, const uint4* __restrict__ tab,
                                 uint32_t stamp, const K* __restrict__ skeys,
                                 const float4* __restrict__ pos4, int64_t n, float3 p, int gw,
                                 int cx, int cy, int cz) {
  // x windows of consecutive cells (two where the neighbourhood wraps)
  int wx0[2], wx1[2], nw = 1;
  const int nx = gm.nc[0];
  if (!(P.periodic & 1)) {
    wx0[0] = max(cx - 1, 0);
    wx1[0] = min(cx + 1, nx - 1);
  } else if (cx == 0) {
    wx0[0] = 0; wx1[0] = 1; wx0[1] = nx - 1; wx1[1] = nx - 1; nw = 2;
  } else if (cx == nx - 1) {
    wx0[0] = nx - 2; wx1[0] = nx - 1; wx0[1] = 0; wx1[1] = 0; nw = 2;
  } else {
    wx0[0] = cx - 1;
    wx1[0] = cx + 1;
  }
  const uint4* __restrict__ rtab = tab + gm.seg0;
  for (int dz = -1; dz <= 1; ++dz) {
    int z = cz + dz;
    if (P.periodic & 4) z = (z + gm.nc[2]) % gm.nc[2];
    else if (z < 0 || z >= gm.nc[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      int y = cy + dy;
      if (P.periodic & 2) y = (y + gm.nc[1]) % gm.nc[1];
      else if (y < 0 || y >= gm.nc[1]) continue;
      for (int wi = 0; wi < nw; ++wi) {
        const int x0 = wx0[wi], x1 = wx1[wi];
        for (int sgi = x0 >> kSegShift; sgi <= (x1 >> kSegShift); ++sgi) {
          const uint32_t sg = seg_tiled(gm, sgi, y, z);
          const uint4 e = __ldg(rtab + sg);
          if ((e.y >> 16) != stamp) continue;
          const int base = sgi << kSegShift;
          const int c0 = max(x0, base) - base, c1 = min(x1, base + kSegCells - 1) - base;
          uint32_t i, end;
          if (!(e.y & 0x8000u)) {
            i = e.x + nib_prefix(e.z, e.w, c0);
            end = e.x + nib_prefix(e.z, e.w, c1 + 1);
          } else {
            const K klo = (K)gm.key0 + (K)((sg << kSegShift) + (uint32_t)c0);
            const K khi = klo + (K)(c1 - c0);
            i = e.x;
            end = e.x + (e.y & kSegMaxCount);
            while (i < end && __ldg(skeys + i) < klo) ++i;
            uint32_t e2 = i;
            while (e2 < end && __ldg(skeys + e2) <= khi) ++e2;
            end = e2;
          }
          if ((int64_t)end > n) end = (uint32_t)n;
          for (; i < end; ++i) {
            const float4 o = __ldg(pos4 + i);
            if (__float_as_int(o.w) == gw) continue;
            if (dist2_per(P, p, make_float3(o.x, o.y, o.z)) < P.rc2) return true;
          }
        }
      }
    }
  }
  return false;
}

// appends one reached site to the list (linking into the per-cell lists happens
// lazily, before a query needs it: k_link_reached)
__device__ __forceinline__ void reached_append(const Reached& R, int g, int sx, int sy, int sz) {
  unsigned long long r = atomicAdd(R.count, 1ull);
  if (r >= R.cap) {
    atomicOr(R.err, ERR_REACHED_CAP);
    return;
  }
  R.key[r] = pack_site(g, sx, sy, sz);
}

// reached-site head of the brick (2^hshift cells per axis) holding cell (x, y, z)
__device__ __forceinline__ uint64_t head_index(const Geo& gm, int hs, int x, int y, int z) {
  const int m = (1 << hs) - 1;
  const uint64_t nbx = (uint64_t)((gm.nc[0] + m) >> hs), nby = (uint64_t)((gm.nc[1] + m) >> hs);
  return gm.head0 + ((uint64_t)(z >> hs) * nby + (uint64_t)(y >> hs)) * nbx + (uint64_t)(x >> hs);
}

// nearest reached site of run gm strictly closer than sqrt(rc2); ties to the
// smaller grain.  Returns the grain or -1.  If any_only, returns on the first hit.
// The sites within the contact radius of p lie in the cells c-1..c+1 of p's cell
// c along each axis (the cell edge exceeds the radius), hence in the bricks
// holding those cells.
// the same over wrapped cells and nearest-image distances (periodic axes of a single
// run, one head per cell)
__device__ int nearest_reached_per(const Params& P, const Geo& gm, const Reached& R, float3 p,
                                   bool any_only) {
  p = wrap_pos(P, gm, p);
  int c[3];
  cell_local(gm, p, c[0], c[1], c[2]);
  int cl[3][3], nl[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    nl[a] = 0;
    for (int d = -1; d <= 1; ++d) {
      int v = c[a] + d;
      if ((P.periodic >> a) & 1) v = (v + gm.nc[a]) % gm.nc[a];
      else if (v < 0 || v >= gm.nc[a]) continue;
      cl[a][nl[a]++] = v;
    }
  }
  float best = P.rc2;
  int bg = -1;
  const unsigned long long guard = *R.count + 1;
  for (int iz = 0; iz < nl[2]; ++iz)
    for (int iy = 0; iy < nl[1]; ++iy)
      for (int ix = 0; ix < nl[0]; ++ix) {
        uint32_t r = R.head[head_index(gm, 0, cl[0][ix], cl[1][iy], cl[2][iz])];
        unsigned long long steps = 0;
        while (r != kNoEntry && steps++ < guard) {
          const unsigned long long key = R.key[r];
          if (key != kDeadSite) {
            int g, sx, sy, sz;
            unpack_site(key, g, sx, sy, sz);
            float4 gc, r0, r1, r2;
            grain_load(P.gtab, g, gc, r0, r1, r2);
            const float d2 = dist2_per(P, p, site_pos_g(gc, r0, r1, r2, sx, sy, sz));
            if (d2 < P.rc2) {
              if (any_only) return g;
              if (d2 < best || (d2 == best && g < bg)) {
                best = d2;
                bg = g;
              }
            }
          }
          r = R.next[r];
        }
      }
  return bg;
}

__device__ int nearest_reached(const Params& P, const Geo& gm, const Reached& R, float3 p,
                               bool any_only) {
  if (P.periodic) return nearest_reached_per(P, gm, R, p, any_only);
  int c[3];
  c[0] = __float2int_rd(__fmul_rn(__fsub_rn(p.x, gm.lo[0]), gm.inv[0]));
  c[1] = __float2int_rd(__fmul_rn(__fsub_rn(p.y, gm.lo[1]), gm.inv[1]));
  c[2] = __float2int_rd(__fmul_rn(__fsub_rn(p.z, gm.lo[2]), gm.inv[2]));
  const int hs = P.hshift;
  int lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = max(c[a] - 1, 0) >> hs;
    hi[a] = min(c[a] + 1, gm.nc[a] - 1) >> hs;
  }
  float best = P.rc2;
  int bg = -1;
  const unsigned long long guard = *R.count + 1;
  for (int bz = lo[2]; bz <= hi[2]; ++bz)
    for (int by = lo[1]; by <= hi[1]; ++by)
      for (int bx = lo[0]; bx <= hi[0]; ++bx) {
        uint32_t r = R.head[head_index(gm, hs, bx << hs, by << hs, bz << hs)];
        unsigned long long steps = 0;
        while (r != kNoEntry && steps++ < guard) {
          const unsigned long long key = R.key[r];
          if (key == kDeadSite) {  // melted
            r = R.next[r];
            continue;
          }
          int g, sx, sy, sz;
          unpack_site(key, g, sx, sy, sz);
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

// run of grain g (the w word of its table entry)
template <bool BATCH>
__device__ __forceinline__ int run_of(const float4& gc) {
  if constexpr (BATCH) return __float_as_int(gc.w);
  else return 0;
}

// cell key (key0 of the run + run-local cell) of a position
template <class K>
__device__ __forceinline__ K cell_key(const Params& P, const Geo& gm, float3 p) {
  int cx, cy, cz;
  if (P.periodic) p = wrap_pos(P, gm, p);
  cell_local(gm, p, cx, cy, cz);
  return (K)gm.key0 + (K)local_tiled(gm, cx, cy, cz);
}

// inside the domain along the axes that are not periodic
__device__ __forceinline__ bool inside_np(const Params& P, const Geo& g, float3 p) {
  return ((P.periodic & 1) || (p.x >= g.lo[0] && p.x <= g.hi[0])) &&
         ((P.periodic & 2) || (p.y >= g.lo[1] && p.y <= g.hi[1])) &&
         ((P.periodic & 4) || (p.z >= g.lo[2] && p.z <= g.hi[2]));
}

// ---------------------------------------------------------------------------------
// k_keys: cell key and identity value of every stored particle
// ---------------------------------------------------------------------------------
template <bool BATCH, class K>
__global__ void __launch_bounds__(256) k_keys(Params P, const int4* __restrict__ rec, int64_t n,
                                              K* __restrict__ keys, uint32_t* __restrict__ vals) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Rec r = rec_unpack(__ldg(rec + i));
  float4 gc, r0, r1, r2;
  grain_load(P.gtab, r.grain, gc, r0, r1, r2);
  const float3 p = add_dir(site_pos_g(gc, r0, r1, r2, r.sx, r.sy, r.sz), r0, r1, r2, r.dir, r.ell);
  keys[i] = cell_key<K>(P, geo_of<BATCH>(P, run_of<BATCH>(gc)), p);
  vals[i] = (uint32_t)i;
}

// ---------------------------------------------------------------------------------
// k_build: sorted store, sorted positions (+ grain and run word), cell table
// ---------------------------------------------------------------------------------
constexpr int kBuildItems = 4;  // records per thread and tile of k_build

template <bool BATCH, class K>
__global__ void __launch_bounds__(256) k_build(Params P, const K* __restrict__ skeys,
                                               const uint32_t* __restrict__ svals,
                                               const int4* __restrict__ rin,
                                               int4* __restrict__ rout, float4* __restrict__ pos4,
                                               uint4* __restrict__ tab,
                                               uint32_t stamp, int64_t n, K key_end,
                                               uint32_t* __restrict__ act, DevStats* st) {
  __shared__ uint32_t s_icnt[8 * kBuildItems];
  __shared__ unsigned long long s_base;
  static_assert(8 * kBuildItems <= 32, "one warp scans the item counts");
  if constexpr (BATCH) {  // sizes of a batch step live on the device (graph capture)
    n = (int64_t)st->n_live;
    stamp = (uint32_t)st->stamp;
  }
  const int lane = threadIdx.x & 31;
  for (int64_t j0 = (int64_t)blockIdx.x * (256 * kBuildItems); j0 < n;
       j0 += (int64_t)gridDim.x * (256 * kBuildItems)) {
    uint32_t amask = 0;  // bit it: record j0 + 256 it + tid is ACTIVE
#pragma unroll 1
    for (int it = 0; it < kBuildItems; ++it) {
      const int64_t j = j0 + it * 256 + threadIdx.x;
      if (j < n) {
        const uint32_t id = __ldg(svals + j);
        const K key = __ldg(skeys + j);
        if ((int64_t)id >= n || key >= key_end) {  // only after a failed sort
          atomicOr(&st->err, ERR_TIMEOUT);
        } else {
          const int4 rv = __ldg(rin + id);
          rout[j] = rv;
          const Rec r = rec_unpack(rv);
          float4 gc, r0, r1, r2;
          grain_load(P.gtab, r.grain, gc, r0, r1, r2);
          const float3 p =
              add_dir(site_pos_g(gc, r0, r1, r2, r.sx, r.sy, r.sz), r0, r1, r2, r.dir, r.ell);
          const int run = run_of<BATCH>(gc);
          const float3 pw = P.periodic ? wrap_pos(P, P.geo, p) : p;
          pos4[j] = make_float4(pw.x, pw.y, pw.z, __int_as_float(r.grain | (run << kRunShift)));
          seg_build<K, true>(geo_of<BATCH>(P, run), skeys, j, n, key, tab, stamp, &st->err);
          if (r.state == ST_ACTIVE) amask |= 1u << it;
        }
      }
    }
    // list of the ACTIVE sorted indices, so that the advance runs on full warps: a
    // CTA appends its share with one reservation per tile, in ascending j (the advance
    // gives a warp 32 consecutive entries, neighbours in space when in record order):
    // item it of warp w starts after items 0..it-1 of all warps and item it of warps < w
    const int warp = threadIdx.x >> 5;
    uint32_t bal[kBuildItems];
#pragma unroll
    for (int it = 0; it < kBuildItems; ++it) {
      bal[it] = __ballot_sync(0xffffffffu, (amask >> it) & 1u);
      if (lane == 0) s_icnt[it * 8 + warp] = (uint32_t)__popc(bal[it]);
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the 8 * kBuildItems counts, item-major
      uint32_t v = lane < 8 * kBuildItems ? s_icnt[lane] : 0u, x = v;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
      }
      if (lane < 8 * kBuildItems) s_icnt[lane] = x - v;
      const uint32_t tot = __shfl_sync(0xffffffffu, x, 31);
      if (lane == 0) s_base = tot ? atomicAdd(&st->n_act, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kBuildItems; ++it)
      if ((amask >> it) & 1u)
        act[s_base + s_icnt[it * 8 + warp] + __popc(bal[it] & ((1u << lane) - 1u))] =
            (uint32_t)(j0 + it * 256 + threadIdx.x);
    __syncthreads();  // s_icnt and s_base are rewritten by the next tile
  }
}

// ---------------------------------------------------------------------------------
// k_advance: contact freeze, growth, advance, spawn claims (sorted store, in place)
// ---------------------------------------------------------------------------------
// A batch: rs and pos4 share the sorted index.  A single run: rs is in grouped order and
// mpos[j] is the position of record j in the cell-ordered sequence (pos4, skeys, tab) that
// also holds the obstacle store; n is that sequence's length; the list act of nrec entries
// holds n_act indices at its front and n_actx at its back (k_act_list).
template <bool BATCH, class K, bool PER = false>
__global__ void __launch_bounds__(256, 8) k_advance(Params P, StepArgs S, int4* __restrict__ rs,
                                                 const float4* __restrict__ pos4,
                                                 const K* __restrict__ skeys,
                                                 const uint4* __restrict__ tab,
                                                 uint32_t stamp, int64_t n,
                                                 const uint32_t* __restrict__ act, Claims C,
                                                 int32_t* __restrict__ site_slot, DevStats* st,
                                                 const uint32_t* __restrict__ mpos,
                                                 int64_t nrec) {
  if constexpr (BATCH) {
    n = (int64_t)st->n_live;
    stamp = (uint32_t)st->stamp;
    S.parity = (int)(st->step & 1ull);
  }
  // step statistics: summed per CTA, one update of each counter per CTA (updates by
  // every warp of these three counters took 15 % of the kernel on the weld plate)
  __shared__ uint32_t s_ctr[3];
  if (threadIdx.x < 3) s_ctr[threadIdx.x] = 0;
  __syncthreads();
  uint32_t c_act = 0, c_froze = 0, c_clamp = 0;
  // thread i advances the i-th listed ACTIVE particle (sorted index j); the loop is
  // uniform over a CTA so that every lane reaches the warp-wide claims
  const int64_t ma = (int64_t)st->n_act;
  const int64_t m = BATCH ? ma : ma + (int64_t)st->n_actx;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < m;
       i0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = i0 + threadIdx.x;
    const int64_t j = i < ma ? (int64_t)__ldg(act + i)
                             : (i < m ? (int64_t)__ldg(act + (nrec - 1 - (i - ma))) : -1);
    bool active = false, froze = false, clamped = false;
    bool crossing = false;
    int g = 0, sx = 0, sy = 0, sz = 0;
    // a single run lists ACTIVE records only (the build's state bytes); a batch checks the
    // state word.  The record is read after the contact search, so that it does not occupy
    // registers during the search
    if (j >= 0 && (!BATCH || ((((uint32_t)__ldg(&rs[j].z)) >> 20) & 3u) == (uint32_t)ST_ACTIVE)) {
      active = true;
      const float4 q = __ldg(pos4 + (BATCH ? j : (int64_t)__ldg(mpos + j)));
      const float3 p = make_float3(q.x, q.y, q.z);
      const int gw = __float_as_int(q.w);
      const Geo& gm = geo_of<BATCH>(P, (int)((uint32_t)gw >> kRunShift));
      int cx, cy, cz;
      cell_local(gm, p, cx, cy, cz);
      bool hit;
      if constexpr (PER)
        hit = contact_scan_per<K>(P, gm, tab, stamp, skeys, pos4, n, p, gw, cx, cy, cz);
      else
        hit = contact_scan<false, K, true>(P, gm, tab, stamp, skeys, pos4, n, p, gw, cx, cy, cz);
      Rec r = rec_unpack(rs[j]);
      g = r.grain;
      if (hit) {
        froze = true;
        r.state = ST_FROZEN;
      } else {
        // thermal sample at (x_n, t_n), growth law, explicit Euler step of ell
        const float e = euler_ell(P, gm, S, p, r.ell, clamped);
        if (reaches_target(e)) {
          r.cross = 1;
          r.ell = fmaxf(__fsub_rn(e, 1.f), 0.f);
          crossing = true;
          sx = r.sx;
          sy = r.sy;
          sz = r.sz;
          step_site(sx, sy, sz, r.dir);
        } else {
          r.ell = e;
        }
      }
      rs[j] = rec_pack(r);
    }
    // spawn claims: every outer direction k' at the reached site s' claims the target
    // s' + e_k' for this step (claimant bit of its axis).  All lanes take part.
    // The warp looks up the block of every s' once (s' was claimed as a target, so its
    // block exists); a target inside that block is claimed directly, and the warp looks
    // up the others (on a face of the block: about one lane in three has one) one per
    // lane and round.  The slot of the block of s' is kept for the resolution in k_emit.
    if (__any_sync(0xffffffffu, crossing)) {
      BlockCache b0;
      int sh = 0;
      warp_claim_word(C, crossing && site_in_range(sx, sy, sz), g, sx, sy, sz, false, sh, b0);
      // outer directions at s' (is_outer: +a where s_a >= 0, -a where s_a <= 0); those
      // whose target leaves the block of s' (s' on that face) or the site range need a
      // lookup of their own
      uint32_t face = 0, same = 0;
      if (crossing) {
        const uint32_t outer = (sx >= 0 ? 1u : 0u) | (sx <= 0 ? 2u : 0u) | (sy >= 0 ? 4u : 0u) |
                               (sy <= 0 ? 8u : 0u) | (sz >= 0 ? 16u : 0u) | (sz <= 0 ? 32u : 0u);
        const uint32_t off = ((sx & 7) == 7 ? 1u : 0u) | ((sx & 7) == 0 || sx <= -kSiteMax ? 2u : 0u) |
                             ((sy & 7) == 7 ? 4u : 0u) | ((sy & 7) == 0 || sy <= -kSiteMax ? 8u : 0u) |
                             ((sz & 7) == 7 ? 16u : 0u) | ((sz & 7) == 0 || sz <= -kSiteMax ? 32u : 0u);
        face = b0.b >= 0 ? (outer & off) : outer;
        same = outer & ~face;
      }
      while (same) {  // per lane: the targets inside the block of s'
        const int k = __ffs(same) - 1;
        same &= same - 1u;
        int tx = sx, ty = sy, tz = sz;
        step_site(tx, ty, tz, k);
        int st2;
        uint32_t* w = block_word(C, b0.b, tx, ty, tz, st2);
        atomicOr(w, (1u << ((k >> 1) + 3 * S.parity)) << st2);
      }
      BlockCache bf;
      while (__any_sync(0xffffffffu, face != 0)) {  // warp-uniform
        const bool have = face != 0;
        const int k = have ? __ffs(face) - 1 : 0;
        face &= face - 1u;
        int tx = sx, ty = sy, tz = sz;
        step_site(tx, ty, tz, k);
        uint32_t* w = warp_claim_word(C, have, g, tx, ty, tz, true, sh, bf);
        if (w) atomicOr(w, (1u << ((k >> 1) + 3 * S.parity)) << sh);
      }
      if (crossing) site_slot[j] = (int32_t)b0.b;
    }
    c_act += active ? 1u : 0u;
    c_froze += froze ? 1u : 0u;
    c_clamp += clamped ? 1u : 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c_act += __shfl_xor_sync(0xffffffffu, c_act, o);
    c_froze += __shfl_xor_sync(0xffffffffu, c_froze, o);
    c_clamp += __shfl_xor_sync(0xffffffffu, c_clamp, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (c_act) atomicAdd(&s_ctr[0], c_act);
    if (c_froze) atomicAdd(&s_ctr[1], c_froze);
    if (c_clamp) atomicAdd(&s_ctr[2], c_clamp);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_ctr[0]) atomicAdd(&st->particle_steps, (unsigned long long)s_ctr[0]);
    if (s_ctr[1]) atomicAdd(&st->frozen_new, (unsigned long long)s_ctr[1]);
    if (s_ctr[2]) atomicAdd(&st->clamped, (unsigned long long)s_ctr[2]);
  }
}

// ---------------------------------------------------------------------------------
// k_emit: claim resolution, reached sites, clip, compaction, next keys.
// A CTA handles a tile of 256 x ITEMS records (ITEMS per thread, strided by 256).  Its
// outputs are placed by a block scan and one atomic reservation per CTA on the
// output counter, so the store order varies from run to run; every result of the
// method is independent of that order.  A large single run takes large tiles (8192
// records) because the reservation on the one shared counter and the scan barrier are
// paid per tile: on the 4 x 2 x 1 mm weld plate, 32 records per thread ran 1.6x faster
// than 4.  A smaller run takes the largest tiles that still fill one wave of CTAs, as a
// thread walks its records one after another.  A batch step holds few records per run
// and takes small tiles, to fill the GPU.
// ---------------------------------------------------------------------------------
constexpr int kEmitItems = 32;      // records per thread, large single run
constexpr int kEmitItemsMid = 8;    // records per thread, single run of one wave at 8
constexpr int kEmitItemsSmall = 2;  // records per thread, smaller single run
constexpr int kEmitItemsBatch = 4;  // records per thread, batch of runs

// decides what record j emits: bit 6 = the record itself, bits 0..5 = children in
// direction k; counts the statistics; appends the reached site of a crossing
template <bool BATCH>
__device__ __forceinline__ uint32_t emit_decide(const Params& P, const StepArgs& S, const Rec& r,
                                                bool valid, int32_t sslot, const Claims& C,
                                                const Reached& R,
                                                uint32_t& n_frozen, uint32_t& n_spawn,
                                                uint32_t& n_lost, uint32_t& n_clip) {
  const int lane = threadIdx.x & 31;
  uint32_t mask = 0;
  const bool crossing = valid && r.state == ST_ACTIVE && r.cross;
  int sx = r.sx, sy = r.sy, sz = r.sz;
  if (crossing) step_site(sx, sy, sz, r.dir);
  // reached site of every crossing particle: one counter update per warp
  const uint32_t want = __ballot_sync(0xffffffffu, crossing);
  if (want) {
    unsigned long long rb = 0;
    if (lane == __ffs(want) - 1) rb = atomicAdd(R.count, (unsigned long long)__popc(want));
    rb = __shfl_sync(0xffffffffu, rb, __ffs(want) - 1);
    if (crossing) {
      const unsigned long long ri = rb + __popc(want & ((1u << lane) - 1u));
      if (ri < R.cap) R.key[ri] = pack_site(r.grain, sx, sy, sz);
      else atomicOr(R.err, ERR_REACHED_CAP);
    }
  }
  if (!valid) return 0;
  if (r.state == ST_FROZEN) {
    ++n_frozen;
    return 1u << 6;
  }
  if (r.state != ST_ACTIVE) return 0;
  if (!crossing) {
    float4 gc, r0, r1, r2;
    grain_load(P.gtab, r.grain, gc, r0, r1, r2);
    const Geo& gm = geo_of<BATCH>(P, run_of<BATCH>(gc));
    const float3 p = add_dir(site_pos_g(gc, r0, r1, r2, r.sx, r.sy, r.sz), r0, r1, r2, r.dir, r.ell);
    if (inside_np(P, gm, p)) return 1u << 6;
    ++n_clip;
    return 0;
  }
  // claims first, the geometry of the winners after: the grain's frame is not held in
  // registers across the claim-word reads
  uint32_t wins = 0;
  BlockCache bc;
  if (sslot >= 0) {  // block of s', looked up by k_advance
    bc.bx = sx >> 3;
    bc.by = sy >> 3;
    bc.bz = sz >> 3;
    bc.b = sslot;
  }
  // outer directions at s' (is_outer), in ascending order
  uint32_t outer = (sx >= 0 ? 1u : 0u) | (sx <= 0 ? 2u : 0u) | (sy >= 0 ? 4u : 0u) |
                   (sy <= 0 ? 8u : 0u) | (sz >= 0 ? 16u : 0u) | (sz <= 0 ? 32u : 0u);
  while (outer) {
    const int k = __ffs(outer) - 1;
    outer &= outer - 1u;
    int tx = sx, ty = sy, tz = sz;
    step_site(tx, ty, tz, k);
    int sh;
    uint32_t* w = claim_lookup(C, r.grain, tx, ty, tz, sh, bc);
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
    wins |= 1u << k;
  }
  if (wins) {
    float4 gc, r0, r1, r2;
    grain_load(P.gtab, r.grain, gc, r0, r1, r2);
    const Geo& gm = geo_of<BATCH>(P, run_of<BATCH>(gc));
    const float3 sp = site_pos_g(gc, r0, r1, r2, sx, sy, sz);
    for (uint32_t wl = wins; wl; wl &= wl - 1u) {
      const int k = __ffs(wl) - 1;
      if (k != r.dir) ++n_spawn;
      if (inside_np(P, gm, add_dir(sp, r0, r1, r2, k, r.ell))) mask |= 1u << k;
      else ++n_clip;
    }
  }
  return mask;
}

template <bool BATCH, class K>
__device__ __forceinline__ void emit_write(const Params& P, const Rec& r, uint32_t mask,
                                           unsigned long long o, int4* __restrict__ rout,
                                           K* __restrict__ keys,
                                           uint32_t* __restrict__ vals, int64_t cap,
                                           int32_t* __restrict__ parent, int64_t j) {
  float4 gc, r0, r1, r2;
  grain_load(P.gtab, r.grain, gc, r0, r1, r2);
  const Geo& gm = geo_of<BATCH>(P, run_of<BATCH>(gc));
  if (mask & (1u << 6)) {
    if (o < (unsigned long long)cap) {
      Rec w = r;
      w.cross = 0;
      rout[o] = rec_pack(w);
      const float3 p =
          add_dir(site_pos_g(gc, r0, r1, r2, r.sx, r.sy, r.sz), r0, r1, r2, r.dir, r.ell);
      keys[o] = cell_key<K>(P, gm, p);
      vals[o] = (uint32_t)o;
      if (parent) parent[o] = (int32_t)j;
    }
    return;
  }
  int sx = r.sx, sy = r.sy, sz = r.sz;
  step_site(sx, sy, sz, r.dir);
  const float3 sp = site_pos_g(gc, r0, r1, r2, sx, sy, sz);
  for (uint32_t ml = mask & 63u; ml; ml &= ml - 1u) {  // the children, in ascending k
    const int k = __ffs(ml) - 1;
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
      keys[o] = cell_key<K>(P, gm, add_dir(sp, r0, r1, r2, k, r.ell));
      vals[o] = (uint32_t)o;
      if (parent) parent[o] = (int32_t)j;
    }
    ++o;
  }
}

template <bool BATCH, class K, int ITEMS>
__global__ void __launch_bounds__(256, 6) k_emit(Params P, StepArgs S, const int4* __restrict__ rs,
                                              const int32_t* __restrict__ site_slot, int64_t n,
                                              int4* __restrict__ rout,
                                              K* __restrict__ keys,
                                              uint32_t* __restrict__ vals, int64_t cap,
                                              Claims C, Reached R, int32_t* __restrict__ parent,
                                              DevStats* st) {
  __shared__ uint32_t s_warp[8];
  __shared__ unsigned long long s_base;
  __shared__ uint8_t s_mask[ITEMS][256];  // what each record emits
  if constexpr (BATCH) {
    n = (int64_t)st->n_live;
    S.parity = (int)(st->step & 1ull);
  }
  const int tid = threadIdx.x, lane = tid & 31;
  uint32_t n_frozen = 0, n_spawn = 0, n_lost = 0, n_clip = 0;
  for (int64_t base = (int64_t)blockIdx.x * (256 * ITEMS); base < n;
       base += (int64_t)gridDim.x * (256 * ITEMS)) {
    uint32_t cnt = 0;
#pragma unroll 1
    for (int it = 0; it < ITEMS; ++it) {
      const int64_t j = base + it * 256 + tid;
      const bool valid = j < n;
      const Rec r = valid ? rec_unpack(__ldg(rs + j)) : Rec{};
      const int32_t sslot =
          (valid && r.cross && r.state == ST_ACTIVE) ? __ldg(site_slot + j) : -1;
      const uint32_t m =
          emit_decide<BATCH>(P, S, r, valid, sslot, C, R, n_frozen, n_spawn, n_lost, n_clip);
      s_mask[it][tid] = (uint8_t)m;
      cnt += __popc(m);
    }
    uint32_t tot;
    const uint32_t ofs = bscan256(cnt, s_warp, tot);
    if (tid == 0) s_base = tot ? atomicAdd(&st->n_out, (unsigned long long)tot) : 0ull;
    __syncthreads();
    // the warp's outputs start at its lane 0's offset; inside the warp they go in
    // item-major order, so each store instruction writes consecutive slots.  The items
    // are written last to first, from the end of the warp's range: the records the
    // decisions read last are read again first, while L2 still holds more of them.
    unsigned long long o = s_base + __shfl_sync(0xffffffffu, ofs, 0) +
                           __reduce_add_sync(0xffffffffu, cnt);
#pragma unroll 1
    for (int it = ITEMS - 1; it >= 0; --it) {
      const uint32_t m = s_mask[it][tid];
      const uint32_t c = __popc(m);
      uint32_t inc = c;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += t;
      }
      o -= __shfl_sync(0xffffffffu, inc, 31);  // s_base is rewritten only after the next scan
      if (m) {
        const int64_t j = base + it * 256 + tid;
        const Rec r = rec_unpack(__ldg(rs + j));
        emit_write<BATCH, K>(P, r, m, o + inc - c, rout, keys, vals, cap, parent, j);
      }
    }
  }
  warp_add(&st->n_frozen, n_frozen);
  warp_add(&st->spawned, n_spawn);
  warp_add(&st->claims_lost, n_lost);
  warp_add(&st->clipped, n_clip);
}

__global__ void k_emit_check(DevStats* st, int64_t cap) {
  if (st->n_out > (unsigned long long)cap) atomicOr(&st->err, ERR_CAPACITY);
}

// links the reached sites [linked, count) into the per-brick lists; grid-stride
template <bool BATCH>
__global__ void k_link_reached(Params P, Reached R, const unsigned long long* linked) {
  const unsigned long long r0 = *linked;
  const unsigned long long r1 = min(*R.count, R.cap);
  for (unsigned long long r = r0 + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
       r < r1; r += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long key = R.key[r];
    if (key == kDeadSite) continue;  // melted before it was linked: never linked
    int g, sx, sy, sz;
    unpack_site(key, g, sx, sy, sz);
    float4 gc, q0, q1, q2;
    grain_load(P.gtab, g, gc, q0, q1, q2);
    const Geo& gm = geo_of<BATCH>(P, run_of<BATCH>(gc));
    int cx, cy, cz;
    const float3 q = site_pos_g(gc, q0, q1, q2, sx, sy, sz);
    cell_local(gm, P.periodic ? wrap_pos(P, gm, q) : q, cx, cy, cz);
    R.next[r] = atomicExch(R.head + head_index(gm, P.hshift, cx, cy, cz), (uint32_t)r);
  }
}

__global__ void k_link_done(Reached R, unsigned long long* linked) {
  *linked = min(*R.count, R.cap);
}

// ---------------------------------------------------------------------------------
// k_nucleate: one CTA; activation test for every pending site against the state
// after the emit, then activation in registration order.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_nucleate(Params P, StepArgs S1, const float4* npos,
                                                  const float4* ngrain, int* nstate, int m,
                                                  float4* gtab, int max_grains, int4* rout,
                                                  uint32_t* keys, uint32_t* vals, int64_t cap,
                                                  Claims C, Reached R, DevStats* st,
                                                  float* gdtn) {
  __shared__ uint32_t s_warp[8];
  __shared__ uint32_t s_run;
  // phase 1: candidates (nstate: 0 pending, 1 candidate, 2 done)
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    if (nstate[j] != 0) continue;
    const float4 q = npos[j];
    const float3 p = make_float3(q.x, q.y, q.z);
    if (undercooling(P, P.geo, S1, p, P.geo.dT_base1) >= q.w &&
        nearest_reached(P, P.geo, R, p, true) < 0)
      nstate[j] = 1;
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
    const unsigned long long g = g0 + rank;
    const bool made = cand && g < (unsigned long long)max_grains;
    // nucleus site and the six first targets are claimed (all lanes take part)
    {
      BlockCache bc;
      for (int k = -1; k < 6; ++k) {
        int tx = 0, ty = 0, tz = 0;
        if (k >= 0) step_site(tx, ty, tz, k);
        int sh = 0;
        uint32_t* w = warp_claim_word(C, made, (int)g, tx, ty, tz, true, sh, bc);
        if (w) atomicOr(w, 0x80u << sh);
      }
    }
    if (cand) {
      nstate[j] = 2;
      if (!made) {
        atomicOr(&st->err, ERR_GRAINS);
      } else {
        for (int q = 0; q < 4; ++q) gtab[4 * g + q] = ngrain[4 * j + q];
        if (gdtn) gdtn[g] = npos[j].w;  // for a later re-nucleation (melting)
        const float4 cq = ngrain[4 * j];
        const float3 c = make_float3(cq.x, cq.y, cq.z);
        // nucleus site reached
        reached_append(R, (int)g, 0, 0, 0);
        const uint32_t key = cell_key<uint32_t>(P, P.geo, c);
        for (int k = 0; k < 6; ++k) {
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

// ---------------------------------------------------------------------------------
// batched nucleation.  Every registered site j of any run has a grain id reserved
// at registration (nmeta[j] = {grain, run}; its table entry is already written).
// k_nuc_test marks the sites that activate at t_{n+1} against the state after the
// emit; k_nuc_activate then activates them (so no activation of this step can
// suppress another one of the same step, as in the single-run kernel).
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_nuc_test(Params P, StepArgs S1,
                                                  const float4* __restrict__ npos,
                                                  const int2* __restrict__ nmeta, int* nstate,
                                                  int m, Reached R) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    if (nstate[j] != 0) continue;
    const float4 q = npos[j];
    const float3 p = make_float3(q.x, q.y, q.z);
    const Geo& gm = geo_of<true>(P, nmeta[j].y);
    if (undercooling(P, gm, S1, p, gm.dT_base1) >= q.w && nearest_reached(P, gm, R, p, true) < 0)
      nstate[j] = 1;
  }
}

__global__ void __launch_bounds__(256) k_nuc_activate(Params P, const float4* __restrict__ npos,
                                                      const int2* __restrict__ nmeta,
                                                      int* nstate, int m, int4* rout,
                                                      uint64_t* keys, uint32_t* vals,
                                                      int64_t cap, Claims C, Reached R,
                                                      DevStats* st) {
  const int lane = threadIdx.x & 31;
  // warp-uniform trip count: every lane reaches the warp-wide claims
  for (int j0 = blockIdx.x * blockDim.x; j0 < m; j0 += gridDim.x * blockDim.x) {
    const int j = j0 + threadIdx.x;
    const bool cand = j < m && nstate[j] == 1;
    if (!__any_sync(0xffffffffu, cand)) continue;
    const int2 meta = cand ? nmeta[j] : make_int2(0, 0);
    {
      BlockCache bc;
      for (int k = -1; k < 6; ++k) {
        int tx = 0, ty = 0, tz = 0;
        if (k >= 0) step_site(tx, ty, tz, k);
        int sh = 0;
        uint32_t* w = warp_claim_word(C, cand, meta.x, tx, ty, tz, true, sh, bc);
        if (w) atomicOr(w, 0x80u << sh);
      }
    }
    const uint32_t want = __ballot_sync(0xffffffffu, cand);
    unsigned long long ob = 0;
    if (lane == __ffs(want) - 1) ob = atomicAdd(&st->n_out, 6ull * __popc(want));
    ob = __shfl_sync(0xffffffffu, ob, __ffs(want) - 1);
    if (cand) {
      nstate[j] = 2;
      reached_append(R, meta.x, 0, 0, 0);
      const float4 q = npos[j];
      const uint64_t key = cell_key<uint64_t>(P, geo_of<true>(P, meta.y), make_float3(q.x, q.y, q.z));
      const unsigned long long o0 = ob + 6ull * __popc(want & ((1u << lane) - 1u));
      for (int k = 0; k < 6; ++k) {
        const unsigned long long o = o0 + k;
        if (o < (unsigned long long)cap) {
          Rec rr;
          rr.grain = meta.x;
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
    if (lane == 0) atomicAdd(&st->nucleated, (unsigned long long)__popc(want));
  }
}

// per-run step constants of a batch: T_L - T0 - Tdot t at t_n and t_{n+1} for the
// step n held on the device, every product and difference rounded once (the host
// computes a single run's values the same way)
__global__ void k_run_step(Geo* runs, const double2* th, int nruns, const DevStats* st,
                           double dt) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nruns) return;
  const long long n = (long long)st->step;
  const double2 q = th[r];
  const double t0 = __dmul_rn((double)n, dt), t1 = __dmul_rn((double)(n + 1), dt);
  runs[r].dT_base = __double2float_rn(__dsub_rn(q.x, __dmul_rn(q.y, t0)));
  runs[r].dT_base1 = __double2float_rn(__dsub_rn(q.x, __dmul_rn(q.y, t1)));
}

// live and ACTIVE particles of every run (counts: 2 per run)
__global__ void __launch_bounds__(256) k_run_counts(Params P, const int4* __restrict__ rec,
                                                    int64_t n, int nruns,
                                                    unsigned long long* counts) {
  __shared__ unsigned int s_c[2 * kMaxRuns];
  for (int i = threadIdx.x; i < 2 * nruns; i += blockDim.x) s_c[i] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Rec r = rec_unpack(__ldg(rec + i));
    const int run = __float_as_int(__ldg(P.gtab + 4 * (size_t)r.grain).w);
    if (run < 0 || run >= nruns) continue;
    atomicAdd(&s_c[2 * run], 1u);
    if (r.state == ST_ACTIVE) atomicAdd(&s_c[2 * run + 1], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * nruns; i += blockDim.x)
    if (s_c[i]) atomicAdd(counts + i, (unsigned long long)s_c[i]);
}

// ---------------------------------------------------------------------------------
// melting walk-back (Sec. 2.1.3), single-run contexts, at t_n before the hash:
//   k_melt_sites      every reached site: superheated -> melted (list entry dead,
//                     claim byte cleared, appended to the melted list); else its
//                     claim byte gets the "reached and not melted" bit 6
//   k_melt_particles  particles superheated or on a site without bit 6 are removed
//                     and release their (never reached) targets
//   k_walkback        per melted site, the first direction k whose neighbour m - e_k
//                     keeps bit 6 sends a new particle from it to m, which it claims
//   k_compact         drops the removed records from the store
//   k_melt_grains     grains with melted sites and none left become dormant
// gflags per grain: byte 0 = has an unmelted site, byte 1 = lost a site in this pass,
// byte 2 = dormant, byte 3 = re-nucleates this step.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_melt_sites(Params P, StepArgs S, Reached R, Claims C,
                                                    unsigned long long* mlist, int64_t mcap,
                                                    uint8_t* gflags, DevStats* st) {
  const unsigned long long n = min(*R.count, R.cap);
  // warp-uniform trip count: every lane reaches the warp-wide claim lookups
  for (unsigned long long r0 = (unsigned long long)blockIdx.x * blockDim.x; r0 < n;
       r0 += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long r = r0 + threadIdx.x;
    const unsigned long long key = r < n ? R.key[r] : kDeadSite;
    const bool valid = key != kDeadSite;
    int g = 0, sx = 0, sy = 0, sz = 0;
    bool melt = false;
    if (valid) {
      unpack_site(key, g, sx, sy, sz);
      float4 gc, q0, q1, q2;
      grain_load(P.gtab, g, gc, q0, q1, q2);
      const float3 x = wrap_pos(P, P.geo, site_pos_g(gc, q0, q1, q2, sx, sy, sz));
      melt = undercooling(P, P.geo, S, x, P.geo.dT_base) < 0.f;
    }
    BlockCache bc;
    int sh = 0;
    uint32_t* w = warp_claim_word(C, valid, g, sx, sy, sz, true, sh, bc);
    if (w) {
      if (melt) atomicAnd(w, ~(0xffu << sh));
      else atomicOr(w, 0x40u << sh);
    }
    warp_add(&st->melted, melt ? 1u : 0u);
    if (melt) {
      R.key[r] = kDeadSite;
      const unsigned long long i = atomicAdd(&st->n_mlist, 1ull);
      if ((int64_t)i < mcap) mlist[i] = key;
      else atomicOr(&st->err, ERR_CAPACITY);
      gflags[4 * (size_t)g + 1] = 1;
    } else if (valid) {
      gflags[4 * (size_t)g] = 1;
    }
  }
}

// claim byte of site t of grain g (nullptr if its block was never claimed)
__device__ __forceinline__ uint32_t* site_byte(const Claims& C, int g, int tx, int ty, int tz,
                                               int& sh, BlockCache& bc) {
  return claim_lookup(C, g, tx, ty, tz, sh, bc);
}

__global__ void __launch_bounds__(256) k_melt_particles(Params P, StepArgs S, int4* rec,
                                                        int64_t n, Claims C, DevStats* st) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool removed = false;
  if (i < n) {
    Rec r = rec_unpack(rec[i]);
    if (r.state == ST_ACTIVE || r.state == ST_FROZEN) {
      const float3 x =
          wrap_pos(P, P.geo, part_pos(P.gtab, r.grain, r.sx, r.sy, r.sz, r.dir, r.ell));
      BlockCache bc;
      int sh = 0;
      const uint32_t* w = site_byte(C, r.grain, r.sx, r.sy, r.sz, sh, bc);
      const bool alive = w && (((*(volatile const uint32_t*)w) >> sh) & 0x40u);
      if (!alive || undercooling(P, P.geo, S, x, P.geo.dT_base) < 0.f) {
        removed = true;
        r.state = ST_REMOVED;
        rec[i] = rec_pack(r);
        int tx = r.sx, ty = r.sy, tz = r.sz;
        step_site(tx, ty, tz, r.dir);
        uint32_t* wt = site_byte(C, r.grain, tx, ty, tz, sh, bc);
        if (wt && !(((*(volatile uint32_t*)wt) >> sh) & 0x40u)) atomicAnd(wt, ~(0xffu << sh));
      }
    }
  }
  warp_add(&st->removed, removed ? 1u : 0u);
}

__global__ void __launch_bounds__(256) k_walkback(Params P, const unsigned long long* mlist,
                                                  Claims C, int4* rec, int64_t cap,
                                                  DevStats* st) {
  const unsigned long long m = st->n_mlist;
  for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < m;
       q += (unsigned long long)gridDim.x * blockDim.x) {
    int g, mx, my, mz;
    unpack_site(mlist[q], g, mx, my, mz);
    BlockCache bc;
    for (int k = 0; k < 6; ++k) {
      int nx = mx, ny = my, nz = mz;
      step_site(nx, ny, nz, k ^ 1);  // m - e_k
      int sh = 0;
      const uint32_t* w = site_byte(C, g, nx, ny, nz, sh, bc);
      if (!w || !(((*(volatile const uint32_t*)w) >> sh) & 0x40u)) continue;
      const unsigned long long o = atomicAdd(&st->n_live, 1ull);
      if (o < (unsigned long long)cap) {
        Rec r;
        r.grain = g;
        r.sx = nx;
        r.sy = ny;
        r.sz = nz;
        r.dir = k;
        r.state = ST_ACTIVE;
        r.cross = 0;
        r.ell = 0.f;
        rec[o] = rec_pack(r);
      } else {
        atomicOr(&st->err, ERR_CAPACITY);
      }
      int shm = 0;
      uint32_t* wm = site_byte(C, g, mx, my, mz, shm, bc);
      if (wm) atomicOr(wm, 0x80u << shm);
      atomicAdd(&st->walkback, 1ull);
      break;
    }
  }
}

// copies the records of rin[0, n_live) that are not REMOVED to rout (one reservation
// per CTA); n_live becomes their count
__global__ void __launch_bounds__(256) k_compact(const int4* __restrict__ rin, int4* rout,
                                                 const unsigned long long* n_in,
                                                 unsigned long long* n_out) {
  __shared__ uint32_t s_warp[8];
  __shared__ unsigned long long s_base;
  const int64_t n = (int64_t)*n_in;
  for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x; j0 < n;
       j0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = j0 + threadIdx.x;
    int4 v = make_int4(0, 0, 0, 0);
    bool keep = false;
    if (j < n) {
      v = rin[j];
      keep = rec_unpack(v).state != ST_REMOVED;
    }
    uint32_t tot;
    const uint32_t ofs = bscan256(keep ? 1u : 0u, s_warp, tot);
    if (threadIdx.x == 0) s_base = tot ? atomicAdd(n_out, (unsigned long long)tot) : 0ull;
    __syncthreads();
    if (keep) rout[s_base + ofs] = v;  // s_base is rewritten only after the next scan
  }
}

__global__ void k_melt_grains(uint8_t* gflags, int ng, DevStats* st) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
    uint8_t* f = gflags + 4 * (size_t)g;
    if (f[1] && !f[0] && !f[2]) {
      f[2] = 1;
      atomicAdd(&st->n_dormant, 1ull);
    }
    f[0] = 0;
    f[1] = 0;
  }
}

// seeds of dormant grains that nucleate again at t_{n+1}: tested before any
// activation of the step (as the pending sites are)
__global__ void k_dormant_test(Params P, StepArgs S1, Reached R, const float* gdtn,
                               uint8_t* gflags, int ng) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
    uint8_t* f = gflags + 4 * (size_t)g;
    if (!f[2]) continue;
    const float4 c = __ldg(P.gtab + 4 * (size_t)g);
    const float3 p = make_float3(c.x, c.y, c.z);
    if (undercooling(P, P.geo, S1, p, P.geo.dT_base1) >= gdtn[g] &&
        nearest_reached(P, P.geo, R, p, true) < 0)
      f[3] = 1;
  }
}

// re-nucleation of the marked seeds, after the step's new nuclei: six particles at
// the nucleus with the grain's own id, nucleus reached and claimed, targets claimed
__global__ void __launch_bounds__(256) k_renucleate(Params P, uint8_t* gflags, int ng, int4* rout,
                                                    uint32_t* keys, uint32_t* vals, int64_t cap,
                                                    Claims C, Reached R, DevStats* st) {
  for (int g0 = blockIdx.x * blockDim.x; g0 < ng; g0 += gridDim.x * blockDim.x) {
    const int g = g0 + threadIdx.x;
    const bool cand = g < ng && gflags[4 * (size_t)g + 3];
    if (!__any_sync(0xffffffffu, cand)) continue;
    {
      BlockCache bc;
      for (int k = -1; k < 6; ++k) {
        int tx = 0, ty = 0, tz = 0;
        if (k >= 0) step_site(tx, ty, tz, k);
        int sh = 0;
        uint32_t* w = warp_claim_word(C, cand, g, tx, ty, tz, true, sh, bc);
        if (w) atomicOr(w, 0x80u << sh);
      }
    }
    if (!cand) continue;
    gflags[4 * (size_t)g + 2] = 0;
    gflags[4 * (size_t)g + 3] = 0;
    atomicAdd(&st->n_dormant, ~0ull);  // minus one
    atomicAdd(&st->nucleated, 1ull);
    atomicAdd(&st->renucleated, 1ull);
    reached_append(R, g, 0, 0, 0);
    const float4 c = __ldg(P.gtab + 4 * (size_t)g);
    const uint32_t key = cell_key<uint32_t>(P, P.geo, make_float3(c.x, c.y, c.z));
    const unsigned long long o0 = atomicAdd(&st->n_live, 6ull);
    for (int k = 0; k < 6; ++k) {
      const unsigned long long o = o0 + k;
      if (o < (unsigned long long)cap) {
        Rec rr;
        rr.grain = g;
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

// end of a step: live count for the next step; a batch also advances its step and
// cell-table stamp counters on the device
__global__ void k_finalize(DevStats* st, int64_t cap, int counters) {
  unsigned long long nl = st->n_out;
  st->n_live = nl > (unsigned long long)cap ? (unsigned long long)cap : nl;
  if (counters) {
    st->step += 1;
    st->stamp += 1;
  }
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
  const bool ok = i < m;
  const int4 s = ok ? sites[i] : make_int4(0, 0, 0, 0);
  if (claimed) {  // uniform across the launch
    BlockCache bc;
    int sh = 0;
    uint32_t* w = warp_claim_word(C, ok, s.x, s.y, s.z, s.w, true, sh, bc);
    if (w) atomicOr(w, 0x80u << sh);
  }
  if (ok && reached) reached_append(R, s.x, s.y, s.z, s.w);
}

// shell seeding: for every (grain, target offset t with |t|_1 = n0 + 1) one ACTIVE
// particle at the site reached from the lowest axis with t_a != 0.
// re-inserts m claim blocks of a checkpoint into an empty claim table: block key i
// (grain g + 1, block coordinates + 512, 10 bits each) gets a pool slot through the
// same warp-wide insert as every claim, and its kBrickWords words are copied there
__global__ void k_claim_restore(Claims C, const unsigned long long* __restrict__ keys,
                                const uint32_t* __restrict__ words, int64_t m) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = i < m;
  int g = 0, tx = 0, ty = 0, tz = 0;
  if (ok) {
    const unsigned long long k = keys[i];
    g = (int)(k >> 30) - 1;
    // a site inside the block (its last corner: every block of a site in range has one)
    tx = ((int)((k >> 20) & 1023u) - 512) * 8 + 7;
    ty = ((int)((k >> 10) & 1023u) - 512) * 8 + 7;
    tz = ((int)(k & 1023u) - 512) * 8 + 7;
  }
  BlockCache bc;
  int sh = 0;
  const uint32_t* w = warp_claim_word(C, ok, g, tx, ty, tz, true, sh, bc);
  if (!w) return;
  uint32_t* d = C.data + (size_t)bc.b * kBrickWords;
  const uint32_t* src = words + (size_t)i * kBrickWords;
  for (int q = 0; q < kBrickWords; ++q) d[q] = src[q];
}

__global__ void k_seed_shell(Params P, const int32_t* __restrict__ grains, int64_t ng,
                             const short4* __restrict__ toff, int64_t nt, float ell0,
                             int4* __restrict__ rout, int64_t cap, unsigned long long* counter,
                             Claims C, uint32_t* err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool ok = i < ng * nt;
  const int g = ok ? grains[i / nt] : 0;
  const short4 t = ok ? toff[i % nt] : make_short4(1, 0, 0, 0);
  int ts[3] = {t.x, t.y, t.z};
  int a = ts[0] != 0 ? 0 : (ts[1] != 0 ? 1 : 2);
  int sg = ts[a] > 0 ? 1 : -1;
  int s[3] = {ts[0], ts[1], ts[2]};
  s[a] -= sg;
  const int dir = 2 * a + (sg > 0 ? 0 : 1);
  if (ok) ok = inside_np(P, P.geo, part_pos(P.gtab, g, s[0], s[1], s[2], dir, ell0));
  if (ok) {
    unsigned long long o = atomicAdd(counter, 1ull);
    if (o >= (unsigned long long)cap) {
      atomicOr(err, ERR_CAPACITY);
    } else {
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
    }
  }
  BlockCache bc;
  int sh = 0;
  uint32_t* w = warp_claim_word(C, ok, g, ts[0], ts[1], ts[2], true, sh, bc);
  if (w) atomicOr(w, 0x80u << sh);
}

// reached + claimed shell sites |s|_1 = n0 of every listed grain
__global__ void k_seed_shell_sites(Params P, const int32_t* __restrict__ grains, int64_t ng,
                                   const short4* __restrict__ soff, int64_t ns, Claims C,
                                   Reached R) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = i < ng * ns;
  const int g = ok ? grains[i / ns] : 0;
  const short4 s = ok ? soff[i % ns] : make_short4(0, 0, 0, 0);
  BlockCache bc;
  int sh = 0;
  uint32_t* w = warp_claim_word(C, ok, g, s.x, s.y, s.z, true, sh, bc);
  if (w) atomicOr(w, 0x80u << sh);
  if (ok) reached_append(R, g, s.x, s.y, s.z);
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

template <bool BATCH>
__global__ void k_grain_map(Params P, int run, Reached R, double ox, double oy, double oz,
                            double sx, double sy, double sz, int nx, int ny, int nz,
                            int32_t* out, int64_t v0, int64_t nv) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  const int64_t v = v0 + i;
  const int ix = (int)(v % nx);
  const int iy = (int)((v / nx) % ny);
  const int iz = (int)(v / ((int64_t)nx * ny));
  float3 p = make_float3((float)(ox + (ix + 0.5) * sx), (float)(oy + (iy + 0.5) * sy),
                         (float)(oz + (iz + 0.5) * sz));
  out[i] = nearest_reached(P, geo_of<BATCH>(P, run), R, p, false);
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
  uint32_t k = cell_local(P.geo, p, cx, cy, cz);
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
                             const uint32_t* __restrict__ skeys,
                             const uint4* __restrict__ tab, int64_t n,
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
  cell_local(P.geo, p, cx, cy, cz);
  const bool hit =
      pairs ? contact_scan<true, uint32_t, false>(P, P.geo, tab, 1u, skeys, pos4, n, p, g, cx, cy, cz,
                                           ids, idj, pairs, pair_cap, npairs)
            : contact_scan<false, uint32_t, false>(P, P.geo, tab, 1u, skeys, pos4, n, p, g, cx, cy, cz);
  if (freeze) freeze[idj] = (hit && stj == ST_ACTIVE) ? 1 : 0;
}

__global__ void k_build_sa(Params P, const float* __restrict__ x3, const int32_t* __restrict__ grain,
                           const uint8_t* __restrict__ state, const uint32_t* __restrict__ skeys,
                           const uint32_t* __restrict__ svals, int64_t n, float4* pos4,
                           uint8_t* sstate, uint4* tab, uint32_t* err) {
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
  if (key >= ncells_of<false>(P.geo)) return;  // removed points
  seg_build<uint32_t, false>(P.geo, skeys, j, n, key, tab, 1u, err);
}

inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// grid of a device-sized (batch) launch: ctas_total CTAs (the launch configuration's
// CTAs per SM times the SM count), fewer if n_max items need fewer
inline unsigned persistent(int64_t n_max, int per_cta, int ctas_total) {
  const int64_t need = (n_max + per_cta - 1) / per_cta;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, ctas_total));
}

// ---------------------------------------------------------------------------------
// Grouping of a single run's records (in place of the radix sort and the build there).
// Records grouped by key >> kGroupShift (a tile of the cell order) and then ordered by
// cell inside each group are in key order:
//   k_group_count    records per group (one atomic per group present in a warp; the
//                    emit's keys are nearly sorted)
//   k_scan_blocks, k_scan_sums   exclusive scan of the counts (group starts)
//   k_group_scatter  record identities and keys grouped by group (any order inside)
//   k_group_order    one warp per group: cell counts in shared memory, their offsets,
//                    the group's cell-table entries and every record's sorted position
//   k_group_gather   one thread per record: record, position, key and ACTIVE flag to
//                    the sorted position; k_act_list then lists the ACTIVE ones
// On the 4 x 2 x 1 mm weld plate this takes 1.1 + 3.05 ms per step against 5.7 + 2.5 ms
// for the histogram, four onesweep passes and the build.
// ---------------------------------------------------------------------------------

// first sorted position of group t (n past the last group)
__device__ __forceinline__ uint32_t tile_start(const uint32_t* __restrict__ ofs,
                                               const uint32_t* __restrict__ bsum, int64_t t,
                                               int64_t ng, int64_t n) {
  return t >= ng ? (uint32_t)n : ofs[t] + bsum[t >> 8];
}

__global__ void __launch_bounds__(256) k_group_count(const uint32_t* __restrict__ keys, int64_t n,
                                                     uint32_t ng, uint32_t* __restrict__ cnt,
                                                     uint32_t* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t t = __ldg(keys + i) >> kGroupShift;
    const uint32_t m = __activemask();
    const int lane = threadIdx.x & 31;
    const uint32_t peers = __match_any_sync(m, t);  // one atomic per group in the warp
    if (lane == __ffs(peers) - 1) {
      if (t < ng) atomicAdd(cnt + t, (uint32_t)__popc(peers));
      else atomicOr(err, ERR_TIMEOUT);
    }
  }
}

__global__ void __launch_bounds__(256) k_group_scatter(const uint32_t* __restrict__ keys, int64_t n,
                                                       uint32_t ng, const uint32_t* __restrict__ ofs,
                                                       const uint32_t* __restrict__ bsum,
                                                       uint32_t* __restrict__ fill,
                                                       uint32_t* __restrict__ perm,
                                                       uint32_t* __restrict__ gkey, uint32_t* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t key = __ldg(keys + i);
    const uint32_t t = key >> kGroupShift;
    const uint32_t m = __activemask();
    const int lane = threadIdx.x & 31;
    const uint32_t peers = __match_any_sync(m, t);
    const int leader = __ffs(peers) - 1;
    uint32_t b = 0;
    if (lane == leader && t < ng) b = atomicAdd(fill + t, (uint32_t)__popc(peers));
    b = __shfl_sync(m, b, leader);
    if (t < ng) {
      const uint64_t p = (uint64_t)tile_start(ofs, bsum, t, ng, n) + b +
                         __popc(peers & ((1u << lane) - 1u));
      if (p < (uint64_t)n) {
        perm[p] = (uint32_t)i;
        gkey[p] = key;
      } else {
        atomicOr(err, ERR_TIMEOUT);
      }
    }
  }
}

// shared-memory slot of a group's cell: lane l owns cells 32 l .. 32 l + 31 (its two
// segments), stored contiguously in a row of kGroupRow words, so that the lane reads and
// writes them as eight 16-byte vectors; with rows of 36 words the eight lanes of each
// quarter warp fall in different banks
static_assert(kGroupCells == 1024, "one lane per 32 cells of a group");
constexpr int kGroupRow = 36;
__device__ __forceinline__ uint32_t group_slot(uint32_t key) {
  const uint32_t ci = key & (kGroupCells - 1);
  return (ci >> 5) * kGroupRow + (ci & 31u);
}

// One warp per group of kGroupCells cells (groups strided over the warps of the grid).
// The cell-ordered sequence of a single run holds its moving records and its obstacle
// store (the obstacles of a group, okey/opos[ogofs[g] .. ogofs[g+1]), already ordered by
// cell, are copied into it).  s_c holds the group's cell counts, moving records in the low
// 16 bits and obstacles in the high 16 bits of each counter, then the position of each
// cell's next entry in the sequence, which the last pass advances to place every entry
// (dest for the moving records).  Each lane sums its 32 cells, one warp scan gives the
// lanes' first positions, and each lane then writes its cells' offsets and its two
// cell-table entries (counts of both kinds).  msrc[position] (on a flush step only) tells
// the flush what the entry is: an obstacle (bit 31 | obstacle index) or a moving record
// (grouped index; bit 30 if FROZEN, set by the gather).
// With obase != 0 (the index of the obstacle store's first entry in pos4 and skeys, which
// hold the store after the sequence), a group without moving records keeps its obstacles
// where they are: its table entries point into the store, nothing is copied, and on a
// flush step its places in the sequence only carry their msrc, in store order.
__global__ void __launch_bounds__(256, 6) k_group_order(
    const uint32_t* __restrict__ gkey, const uint32_t* __restrict__ ofs,
    const uint32_t* __restrict__ bsum, uint32_t ng, int64_t n, uint64_t seg0,
    uint32_t* __restrict__ dest, uint4* __restrict__ tab, uint32_t stamp, DevStats* st,
    const uint32_t* __restrict__ okey, const float4* __restrict__ opos,
    const uint32_t* __restrict__ ogofs, int64_t no, float4* __restrict__ pos4,
    uint32_t* __restrict__ skeys, uint32_t* __restrict__ msrc, uint32_t obase,
    uint32_t* __restrict__ rbuild, uint32_t build, int reuse) {
  __shared__ uint4 s_c4[8][32 * kGroupRow / 4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t* c = reinterpret_cast<uint32_t*>(s_c4[w]);
  uint4* row = s_c4[w] + lane * (kGroupRow / 4);  // the lane's 32 cells
  for (int64_t g = (int64_t)blockIdx.x * 8 + w; g < (int64_t)ng; g += (int64_t)gridDim.x * 8) {
    const uint32_t s = tile_start(ofs, bsum, g, ng, n);
    const uint32_t e = tile_start(ofs, bsum, g + 1, ng, n);
    const uint32_t os = no ? __ldg(ogofs + g) : 0u, oe = no ? __ldg(ogofs + g + 1) : 0u;
    if (s >= e && os >= oe) continue;  // warp-uniform
    const bool resident = obase != 0u && s >= e;  // obstacles only: read in place
    if (resident && rbuild) {
      // written as resident by the previous build, with the same store (reuse): its
      // entries are the previous build's, given this build's stamp
      if (reuse && rbuild[g] == build - 1u) {  // warp-uniform
        const uint64_t sg = seg0 + ((uint64_t)g << (kGroupShift - kSegShift)) + 2 * lane;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint4 t = tab[sg + h];
          if ((t.y >> 16) == stamp - 1u) {
            t.y = (stamp << 16) | (t.y & 0xffffu);
            tab[sg + h] = t;
          }
        }
        if (msrc)
          for (uint32_t i = os + lane; i < oe; i += 32) msrc[s + i] = 0x80000000u | i;
        __syncwarp();
        if (lane == 0) rbuild[g] = build;
        continue;
      }
      __syncwarp();
      if (lane == 0) rbuild[g] = build;  // written below as resident
    }
#pragma unroll
    for (int q = 0; q < kGroupRow / 4; ++q) s_c4[w][q * 32 + lane] = make_uint4(0, 0, 0, 0);
    __syncwarp();
    // four keys of the lane in flight at a time
    for (uint32_t i0 = s + lane; i0 < e; i0 += 128) {
      uint32_t k[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) k[u] = i0 + 32 * u < e ? __ldg(gkey + i0 + 32 * u) : 0u;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + 32 * u < e) atomicAdd(c + group_slot(k[u]), 1u);
    }
    for (uint32_t i0 = os + lane; i0 < oe; i0 += 128) {
      uint32_t k[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) k[u] = i0 + 32 * u < oe ? __ldg(okey + i0 + 32 * u) : 0u;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + 32 * u < oe) atomicAdd(c + group_slot(k[u]), 1u << 16);
    }
    __syncwarp();
    uint32_t tot = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint4 v = row[q];
      tot += ((v.x & 0xffffu) + (v.x >> 16)) + ((v.y & 0xffffu) + (v.y >> 16)) +
             ((v.z & 0xffffu) + (v.z >> 16)) + ((v.w & 0xffffu) + (v.w >> 16));
    }
    uint32_t inc = tot;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= d) inc += y;
    }
    if (tot) {
      // cells 0-7 / 8-15 of a segment give its z / w word: 4-bit counts saturated at 15
      uint32_t run = (resident ? obase + os : s + os) + inc - tot;
      const uint64_t sg = seg0 + ((uint64_t)g << (kGroupShift - kSegShift)) + 2 * lane;
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const uint32_t start = run;
        uint32_t nb[2], vmax = 0u;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          nb[j] = 0u;
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            // cells 8 j + 4 t .. 8 j + 4 t + 3 of the segment
            const int q = 4 * h + 2 * j + t;
            uint4 v = row[q];
            v.x = (v.x & 0xffffu) + (v.x >> 16);
            v.y = (v.y & 0xffffu) + (v.y >> 16);
            v.z = (v.z & 0xffffu) + (v.z >> 16);
            v.w = (v.w & 0xffffu) + (v.w >> 16);
            uint4 o;
            o.x = run;
            run += v.x;
            o.y = run;
            run += v.y;
            o.z = run;
            run += v.z;
            o.w = run;
            run += v.w;
            row[q] = o;
            nb[j] |= (min(v.x, 15u) | (min(v.y, 15u) << 4) | (min(v.z, 15u) << 8) |
                      (min(v.w, 15u) << 12)) << (16 * t);
            vmax = max(vmax, max(max(v.x, v.y), max(v.z, v.w)));
          }
        }
        const bool sat = vmax >= 15u;
        const uint32_t cnt = run - start;
        if (cnt) {
          if (cnt >= kSegMaxCount) atomicOr(&st->err, ERR_CELL_OVERFLOW);
          const uint32_t cc = cnt < kSegMaxCount ? cnt : kSegMaxCount;
          tab[sg + h] = make_uint4(start, (stamp << 16) | (sat ? 0x8000u : 0u) | cc, nb[0], nb[1]);
        }
      }
    }
    __syncwarp();
    if (resident) {
      // the group's places in the sequence stand for its obstacles, in store order
      if (msrc)
        for (uint32_t i = os + lane; i < oe; i += 32) msrc[s + i] = 0x80000000u | i;
      __syncwarp();
      continue;
    }
    // the obstacles go to their cells' slots, then the moving records (any order inside
    // a cell)
    for (uint32_t i0 = os + lane; i0 < oe; i0 += 128) {
      // keys and positions of four obstacles in flight before their slots are taken
      uint32_t k[4];
      float4 q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool ok = i0 + 32 * u < oe;
        k[u] = ok ? __ldg(okey + i0 + 32 * u) : 0u;
        q[u] = ok ? __ldg(opos + i0 + 32 * u) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      uint32_t d[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        d[u] = i0 + 32 * u < oe ? atomicAdd(c + group_slot(k[u]), 1u) : 0u;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + 32 * u < oe) {
          pos4[d[u]] = q[u];
          skeys[d[u]] = k[u];
          if (msrc) msrc[d[u]] = 0x80000000u | (i0 + 32 * u);
        }
    }
    for (uint32_t i0 = s + lane; i0 < e; i0 += 128) {
      uint32_t k[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) k[u] = i0 + 32 * u < e ? __ldg(gkey + i0 + 32 * u) : 0u;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + 32 * u < e) dest[i0 + 32 * u] = atomicAdd(c + group_slot(k[u]), 1u);
    }
    __syncwarp();
  }
}

// every grouped record i: the record in grouped order (the store the advance and the emit
// walk), its position, key and source in the cell-ordered sequence at dest[i], its store
// index (tape) and its state byte (1 ACTIVE, 3 ACTIVE in the first or last cell of its
// segment, 2 FROZEN, 0 otherwise); one thread per record
__global__ void __launch_bounds__(256) k_group_gather(
    Params P, const uint32_t* __restrict__ gkey, const uint32_t* __restrict__ perm,
    const uint32_t* __restrict__ dest, int64_t n, const int4* __restrict__ rin,
    int4* __restrict__ rout, float4* __restrict__ pos4, uint32_t* __restrict__ skeys,
    uint32_t* __restrict__ svals, uint8_t* __restrict__ sact, uint32_t* __restrict__ msrc,
    int64_t nseq, DevStats* st) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t o = __ldg(perm + i), j = __ldg(dest + i);
  if ((int64_t)o >= n || (int64_t)j >= nseq) {  // only after inconsistent keys
    atomicOr(&st->err, ERR_TIMEOUT);
    return;
  }
  const int4 rv = __ldg(rin + o);
  rout[i] = rv;
  const Rec r = rec_unpack(rv);
  float4 gc, r0, r1, r2;
  grain_load(P.gtab, r.grain, gc, r0, r1, r2);
  const float3 p = add_dir(site_pos_g(gc, r0, r1, r2, r.sx, r.sy, r.sz), r0, r1, r2, r.dir, r.ell);
  const float3 pw = P.periodic ? wrap_pos(P, P.geo, p) : p;
  pos4[j] = make_float4(pw.x, pw.y, pw.z, __int_as_float(r.grain));
  skeys[j] = __ldg(gkey + i);
  if (msrc) msrc[j] = (uint32_t)i | (r.state == ST_FROZEN ? 0x40000000u : 0u);
  if (svals) svals[i] = o;
  // the 3-cell window x-1..x+1 of a cell at either end of its segment reaches into the
  // next segment (tiled keys: x & 15 is the cell's place in its segment)
  const uint32_t xs = (uint32_t)(__ldg(gkey + i) - (uint32_t)P.geo.key0) & (kSegCells - 1);
  sact[i] = r.state == ST_ACTIVE ? (xs == 0 || xs == kSegCells - 1 ? 3 : 1)
                                 : (r.state == ST_FROZEN ? 2 : 0);
}

// List of the ACTIVE grouped indices, in ascending order inside each tile of 1024 records
// (one reservation per tile; each thread takes kActItems consecutive records).  State byte
// 1 goes to the front of act (count in n_act), state byte 3 to the back, from act[n - 1]
// downwards (count in n_actx): the contact search of a particle in the first or last cell
// of a segment reads two segments per neighbour row, and a warp runs the second one
// whenever any of its lanes needs it (one lane in eight; nearly every warp of a mixed
// list).  The advance gives a warp 32 consecutive entries: in record order they are
// neighbours in space (an order that interleaved runs of 32 records 256 apart left the
// advance 4 % slower on the weld plate).
constexpr int kActItems = 4;
__global__ void __launch_bounds__(256) k_act_list(const uint8_t* __restrict__ sact, int64_t n,
                                                  uint32_t* __restrict__ act, DevStats* st) {
  __shared__ uint32_t s_warp[8];
  __shared__ unsigned long long s_base[2];
  for (int64_t j0 = (int64_t)blockIdx.x * (256 * kActItems); j0 < n;
       j0 += (int64_t)gridDim.x * (256 * kActItems)) {
    const int64_t jb = j0 + (int64_t)threadIdx.x * kActItems;
    uint32_t amask = 0, xmask = 0;
#pragma unroll
    for (int it = 0; it < kActItems; ++it) {
      const int64_t j = jb + it;
      const uint8_t v = j < n ? __ldg(sact + j) : (uint8_t)0;
      if (v == 1) amask |= 1u << it;
      if (v == 3) xmask |= 1u << it;
    }
    uint32_t tot, totx;
    const uint32_t ofs = bscan256(__popc(amask), s_warp, tot);
    const uint32_t ofx = bscan256(__popc(xmask), s_warp, totx);
    if (threadIdx.x == 0) {
      s_base[0] = tot ? atomicAdd(&st->n_act, (unsigned long long)tot) : 0ull;
      s_base[1] = totx ? (unsigned long long)atomicAdd(&st->n_actx, totx) : 0ull;
    }
    __syncthreads();
    unsigned long long o = s_base[0] + ofs, ox = s_base[1] + ofx;  // rewritten only after
#pragma unroll                                                    // the next scans
    for (int it = 0; it < kActItems; ++it) {
      if ((amask >> it) & 1u) act[o++] = (uint32_t)(jb + it);
      if ((xmask >> it) & 1u) act[n - 1 - (int64_t)(ox++)] = (uint32_t)(jb + it);
    }
  }
}

// ---------------------------------------------------------------------------------
// obstacle flush (one run).  The cell-ordered sequence of the step holds the obstacle
// store and the moving records in key order; its entries that are obstacles or FROZEN
// moving records (msrc bit 31 or bit 30), taken in sequence order, are the new obstacle
// store, already ordered by key:
//   k_obs_count    joining entries per tile of kObsTile entries, summed into
//                  DevStats::obs_new (the new store's size)
//   k_scan_sums    exclusive scan of the tile counts
//   k_obs_compact  their keys, positions and records into the other copy of the store;
//                  a moving record that joins is marked REMOVED in the grouped store, so
//                  that the emit drops it (the contact search of the step still finds its
//                  position in the sequence)
//   k_obs_groups   the first obstacle of every group of kGroupCells cells (binary search
//                  of the group's first key), which the next steps' ordering reads
// The step after a flush carries no FROZEN record from before it.
// ---------------------------------------------------------------------------------
constexpr int kObsItems = 32;                // sequence entries per thread
constexpr int kObsTile = 256 * kObsItems;    // entries per tile

// source words of the kObsItems entries j0 .. j0 + 31 (0: not joining, past nseq)
__device__ __forceinline__ void obs_words(const uint32_t* __restrict__ msrc, int64_t nseq,
                                          int64_t j0, uint32_t w[kObsItems]) {
  if (j0 + kObsItems <= nseq) {
    const uint4* p = reinterpret_cast<const uint4*>(msrc + j0);  // j0 is a multiple of 32
#pragma unroll
    for (int q = 0; q < kObsItems / 4; ++q) {
      const uint4 v = __ldg(p + q);
      w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < kObsItems; ++q) w[q] = j0 + q < nseq ? __ldg(msrc + j0 + q) : 0u;
  }
}

__device__ __forceinline__ bool joins(uint32_t src) { return (src & 0xC0000000u) != 0u; }

__global__ void __launch_bounds__(256) k_obs_count(const uint32_t* __restrict__ msrc,
                                                   int64_t nseq, uint32_t* __restrict__ tcnt,
                                                   DevStats* st) {
  __shared__ uint32_t s_warp[8];
  const int64_t j0 = (int64_t)blockIdx.x * kObsTile + (int64_t)threadIdx.x * kObsItems;
  uint32_t w[kObsItems], c = 0;
  obs_words(msrc, nseq, j0, w);
#pragma unroll
  for (int q = 0; q < kObsItems; ++q) c += joins(w[q]) ? 1u : 0u;
  uint32_t tot;
  bscan256(c, s_warp, tot);
  if (threadIdx.x == 0) {
    tcnt[blockIdx.x] = tot;
    if (tot) atomicAdd(&st->obs_new, (unsigned long long)tot);
  }
}

// Warp w of the tile takes entries tile * kObsTile + w * 1024 + q * 32 + lane (q = 0..31),
// so that every load and store of a q is coalesced; ranks follow the entries' order (warp
// ballots inside a warp, a block scan of the warps' totals).
__global__ void __launch_bounds__(256) k_obs_compact(
    const uint32_t* __restrict__ msrc, const uint32_t* __restrict__ skeys,
    const float4* __restrict__ pos4, int64_t nseq, const uint32_t* __restrict__ tofs,
    const int4* __restrict__ orec, int4* __restrict__ rs, uint32_t* __restrict__ okey2,
    float4* __restrict__ opos2, int4* __restrict__ orec2, int64_t obase) {
  __shared__ uint32_t s_warp[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t wb = (int64_t)blockIdx.x * kObsTile + (int64_t)w * (32 * kObsItems);
  uint32_t bits = 0, wcnt = 0;
#pragma unroll
  for (int q = 0; q < kObsItems; ++q) {
    const int64_t j = wb + q * 32 + lane;
    const bool f = j < nseq && joins(__ldg(msrc + j));
    bits |= (f ? 1u : 0u) << q;
    wcnt += __popc(__ballot_sync(0xffffffffu, f));
  }
  uint32_t tot;
  const uint32_t wofs = bscan256(lane == 0 ? wcnt : 0u, s_warp, tot);
  uint32_t o = tofs[blockIdx.x] + __shfl_sync(0xffffffffu, wofs, 0);
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll 1
  for (int q = 0; q < kObsItems; ++q) {
    const bool f = (bits >> q) & 1u;
    const uint32_t b = __ballot_sync(0xffffffffu, f);
    if (f) {
      const int64_t j = wb + q * 32 + lane;
      const uint32_t r = o + __popc(b & lt);
      const uint32_t src = __ldg(msrc + j), idx = src & 0x3fffffffu;
      // an obstacle's key and position from the store (entry obase + idx of skeys and
      // pos4: a group read in place has no copy in the sequence), a FROZEN record's from
      // the sequence
      const int64_t from = (src & 0x80000000u) ? obase + idx : j;
      okey2[r] = __ldg(skeys + from);
      opos2[r] = __ldg(pos4 + from);
      if (src & 0x80000000u) {
        orec2[r] = __ldg(orec + idx);
      } else {
        int4 rv = rs[idx];  // FROZEN: it moves to the obstacles, the emit drops it
        orec2[r] = rv;
        rv.z = (int)(((uint32_t)rv.z & ~(3u << 20)) | ((uint32_t)ST_REMOVED << 20));
        rs[idx] = rv;
      }
    }
    o += __popc(b);
  }
}

__global__ void __launch_bounds__(256) k_obs_groups(const uint32_t* __restrict__ okey,
                                                    const DevStats* st, uint32_t ng,
                                                    uint32_t* __restrict__ ogofs) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g > (int64_t)ng) return;
  const int64_t n = (int64_t)st->obs_new;
  const uint64_t key = (uint64_t)g << kGroupShift;
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((uint64_t)__ldg(okey + mid) < key) lo = mid + 1;
    else hi = mid;
  }
  ogofs[g] = (uint32_t)lo;
}

// Runs one bounded wait whose word nothing ever publishes (one thread), with a
// limit of `limit` polls: which = 0 the onesweep look-back of tile 1 on the
// never-published status word of tile 0; which = 1 the claim-slot wait on a
// pending bucket (key set, slot word 0).  The error bits land in *err.
__global__ void k_selftest_wait(int which, uint32_t limit, uint32_t* words, uint32_t* err) {
  if (which == 0) {
    (void)lookback_excl(words, 1, 0, limit, err);
  } else {
    Claims C{};
    C.bucket = reinterpret_cast<ulonglong2*>(words);
    C.err = err;
    (void)claim_wait(C, 0, limit);
  }
}

}  // namespace

// ---------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------
int64_t obs_tiles(int64_t nseq) { return (nseq + kObsTile - 1) / kObsTile; }

void launch_obs_flush(const uint32_t* msrc, const uint32_t* skeys, const float4* pos4,
                      int64_t nseq, uint32_t* tcnt, const int4* orec, int4* rs, uint32_t* okey2,
                      float4* opos2, int4* orec2, uint32_t ng, uint32_t* ogofs2, DevStats* dst,
                      cudaStream_t st, int64_t obase) {
  const int64_t nt = obs_tiles(nseq);
  cudaMemsetAsync(&dst->obs_new, 0, sizeof(unsigned long long), st);
  if (nt > 0) {
    k_obs_count<<<(unsigned)nt, 256, 0, st>>>(msrc, nseq, tcnt, dst);
    k_scan_sums<<<1, 256, 0, st>>>(tcnt, nt);
    k_obs_compact<<<(unsigned)nt, 256, 0, st>>>(msrc, skeys, pos4, nseq, tcnt, orec, rs, okey2,
                                                opos2, orec2, obase);
  }
  k_obs_groups<<<blocks((int64_t)ng + 1), 256, 0, st>>>(okey2, dst, ng, ogofs2);
}

void launch_selftest_wait(int which, uint32_t limit, uint32_t* words, uint32_t* err,
                          cudaStream_t st) {
  k_selftest_wait<<<1, 1, 0, st>>>(which, limit, words, err);
}

// A batch context (batch == true) sorts uint64 keys, a single-run context uint32.
void launch_keys(bool batch, const Params& P, const int4* rec, int64_t n, void* keys,
                 uint32_t* vals, cudaStream_t st) {
  if (n <= 0) return;
  if (batch)
    k_keys<true, uint64_t><<<blocks(n), 256, 0, st>>>(P, rec, n, (uint64_t*)keys, vals);
  else
    k_keys<false, uint32_t><<<blocks(n), 256, 0, st>>>(P, rec, n, (uint32_t*)keys, vals);
}

void launch_build(const Params& P, const uint64_t* skeys, const uint32_t* svals, const int4* rin,
                  int4* rout, float4* pos4, uint4* tab, int64_t n, uint64_t key_end, uint32_t* act,
                  DevStats* dst, cudaStream_t st) {
  if (n <= 0) return;
  k_build<true, uint64_t><<<persistent(n, 256 * kBuildItems, P.launch.build_ctas), 256, 0, st>>>(
      P, skeys, svals, rin, rout, pos4, tab, 0, n, key_end, act, dst);
}

void launch_advance(bool batch, const Params& P, const StepArgs& S, int4* rs, const float4* pos4,
                    const void* skeys, const uint4* tab, uint32_t stamp, int64_t n,
                    const uint32_t* act, const Claims& C, int32_t* site_slot, DevStats* dst,
                    cudaStream_t st, int64_t nrec, const uint32_t* mpos) {
  if (n <= 0) return;
  if (batch)
    k_advance<true, uint64_t><<<persistent(n, 256, P.launch.advance_ctas), 256, 0, st>>>(
        P, S, rs, pos4, (const uint64_t*)skeys, tab, stamp, n, act, C, site_slot, dst, nullptr,
        0);
  else if (P.periodic)
    k_advance<false, uint32_t, true><<<blocks(nrec), 256, 0, st>>>(
        P, S, rs, pos4, (const uint32_t*)skeys, tab, stamp, n, act, C, site_slot, dst, mpos,
        nrec);
  else
    k_advance<false, uint32_t><<<blocks(nrec), 256, 0, st>>>(
        P, S, rs, pos4, (const uint32_t*)skeys, tab, stamp, n, act, C, site_slot, dst, mpos,
        nrec);
}

int64_t emit_tiles(int64_t n, int items) { return (n + 256 * items - 1) / (256 * items); }

void launch_link_reached(bool batch, const Params& P, const Reached& R,
                         unsigned long long* linked, int sms, cudaStream_t st) {
  if (batch) k_link_reached<true><<<sms * 8, 256, 0, st>>>(P, R, linked);
  else k_link_reached<false><<<sms * 8, 256, 0, st>>>(P, R, linked);
  k_link_done<<<1, 1, 0, st>>>(R, linked);
}

void launch_emit(bool batch, const Params& P, const StepArgs& S, const int4* rs,
                 const int32_t* site_slot, int64_t n, int4* rout, void* keys, uint32_t* vals,
                 int64_t cap, const Claims& C, const Reached& R, int32_t* parent, DevStats* dst,
                 cudaStream_t st) {
  if (n <= 0) return;
  // one wave of emit CTAs (P.launch.emit_ctas) sets the tile size of a single run
  const int64_t wave = P.launch.emit_ctas;
  if (batch)
    k_emit<true, uint64_t, kEmitItemsBatch>
        <<<persistent(n, 256 * kEmitItemsBatch, P.launch.emit_ctas), 256, 0, st>>>(
            P, S, rs, site_slot, n, rout, (uint64_t*)keys, vals, cap, C, R, parent, dst);
  else if (emit_tiles(n, kEmitItems) >= wave)
    k_emit<false, uint32_t, kEmitItems><<<(unsigned)emit_tiles(n, kEmitItems), 256, 0, st>>>(
        P, S, rs, site_slot, n, rout, (uint32_t*)keys, vals, cap, C, R, parent, dst);
  else if (emit_tiles(n, kEmitItemsMid) >= wave)
    k_emit<false, uint32_t, kEmitItemsMid>
        <<<(unsigned)emit_tiles(n, kEmitItemsMid), 256, 0, st>>>(
            P, S, rs, site_slot, n, rout, (uint32_t*)keys, vals, cap, C, R, parent, dst);
  else
    k_emit<false, uint32_t, kEmitItemsSmall>
        <<<(unsigned)emit_tiles(n, kEmitItemsSmall), 256, 0, st>>>(
            P, S, rs, site_slot, n, rout, (uint32_t*)keys, vals, cap, C, R, parent, dst);
  k_emit_check<<<1, 1, 0, st>>>(dst, cap);
}

void launch_nucleate_batch(const Params& P, const StepArgs& S1, const float4* npos,
                           const int2* nmeta, int* nstate, int m, int4* rout, uint64_t* keys,
                           uint32_t* vals, int64_t cap, const Claims& C, const Reached& R,
                           DevStats* dst, int sms, cudaStream_t st) {
  if (m <= 0) return;
  const unsigned nb = (unsigned)std::min<int64_t>(blocks(m), (int64_t)sms * 8);
  k_nuc_test<<<nb, 256, 0, st>>>(P, S1, npos, nmeta, nstate, m, R);
  k_nuc_activate<<<nb, 256, 0, st>>>(P, npos, nmeta, nstate, m, rout, keys, vals, cap, C, R,
                                     dst);
}

void launch_nucleate(const Params& P, const StepArgs& S1, const float4* npos, const float4* ngrain,
                     int* nstate, int m, float4* gtab, int max_grains, int4* rout, uint32_t* keys,
                     uint32_t* vals, int64_t cap, const Claims& C, const Reached& R, DevStats* dst,
                     float* gdtn, cudaStream_t st) {
  k_nucleate<<<1, 256, 0, st>>>(P, S1, npos, ngrain, nstate, m, gtab, max_grains, rout, keys,
                                vals, cap, C, R, dst, gdtn);
}

void launch_run_step(Geo* runs, const double2* th, int nruns, const DevStats* dst, double dt,
                     cudaStream_t st) {
  k_run_step<<<(nruns + 255) / 256, 256, 0, st>>>(runs, th, nruns, dst, dt);
}

void launch_run_counts(const Params& P, const int4* rec, int64_t n, int nruns,
                       unsigned long long* counts, cudaStream_t st) {
  if (n <= 0) return;
  const unsigned nb = (unsigned)std::min<int64_t>(blocks(n), 152 * 8);
  k_run_counts<<<nb, 256, 0, st>>>(P, rec, n, nruns, counts);
}

void launch_melt(const Params& P, const StepArgs& S, const Reached& R, const Claims& C,
                 unsigned long long* mlist, int64_t mcap, uint8_t* gflags, int ng, int4* rec,
                 int4* rtmp, int64_t n, int64_t cap, DevStats* dst, int sms, cudaStream_t st) {
  cudaMemsetAsync(&dst->n_mlist, 0, sizeof(unsigned long long), st);
  cudaMemsetAsync(&dst->removed, 0, sizeof(unsigned long long), st);
  k_melt_sites<<<sms * 8, 256, 0, st>>>(P, S, R, C, mlist, mcap, gflags, dst);
  if (n > 0) k_melt_particles<<<blocks(n), 256, 0, st>>>(P, S, rec, n, C, dst);
  k_walkback<<<sms * 4, 256, 0, st>>>(P, mlist, C, rec, cap, dst);
  // the store (walk-back particles appended) is compacted into rtmp
  cudaMemcpyAsync(&dst->n_out, &dst->n_live, sizeof(unsigned long long),
                  cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(&dst->n_live, 0, sizeof(unsigned long long), st);
  k_compact<<<sms * 8, 256, 0, st>>>(rec, rtmp, &dst->n_out, &dst->n_live);
  if (ng > 0) k_melt_grains<<<(ng + 255) / 256, 256, 0, st>>>(gflags, ng, dst);
}

void launch_dormant_test(const Params& P, const StepArgs& S1, const Reached& R, const float* gdtn,
                         uint8_t* gflags, int ng, cudaStream_t st) {
  if (ng > 0) k_dormant_test<<<(ng + 255) / 256, 256, 0, st>>>(P, S1, R, gdtn, gflags, ng);
}

void launch_renucleate(const Params& P, uint8_t* gflags, int ng, int4* rout, uint32_t* keys,
                       uint32_t* vals, int64_t cap, const Claims& C, const Reached& R,
                       DevStats* dst, cudaStream_t st) {
  if (ng > 0)
    k_renucleate<<<(ng + 255) / 256, 256, 0, st>>>(P, gflags, ng, rout, keys, vals, cap, C, R,
                                                   dst);
}

void launch_finalize(DevStats* dst, int64_t cap, bool batch, cudaStream_t st) {
  k_finalize<<<1, 1, 0, st>>>(dst, cap, batch ? 1 : 0);
}

void launch_append(const int4* src, int64_t m, int4* rout, int64_t base, cudaStream_t st) {
  if (m > 0) k_append<<<blocks(m), 256, 0, st>>>(src, m, rout, base);
}

void launch_mark_sites(const Params& P, const int4* sites, int64_t m, int reached, int claimed,
                       const Claims& C, const Reached& R, cudaStream_t st) {
  if (m > 0) k_mark_sites<<<blocks(m), 256, 0, st>>>(P, sites, m, reached, claimed, C, R);
}

void launch_claim_restore(const Claims& C, const unsigned long long* keys, const uint32_t* words,
                          int64_t m, cudaStream_t st) {
  if (m > 0) k_claim_restore<<<blocks(m), 256, 0, st>>>(C, keys, words, m);
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

void launch_grain_map(bool batch, const Params& P, int run, const Reached& R, const double o[3],
                      const double s[3], const int nvox[3], int32_t* out, int64_t v0, int64_t nv,
                      cudaStream_t st) {
  if (nv <= 0) return;
  if (batch)
    k_grain_map<true><<<blocks(nv), 256, 0, st>>>(P, run, R, o[0], o[1], o[2], s[0], s[1], s[2],
                                                  nvox[0], nvox[1], nvox[2], out, v0, nv);
  else
    k_grain_map<false><<<blocks(nv), 256, 0, st>>>(P, 0, R, o[0], o[1], o[2], s[0], s[1], s[2],
                                                   nvox[0], nvox[1], nvox[2], out, v0, nv);
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
                     uint8_t* sstate, uint4* tab, uint32_t* err, cudaStream_t st) {
  if (n > 0)
    k_build_sa<<<blocks(n), 256, 0, st>>>(P, x3, grain, state, skeys, svals, n, pos4, sstate, tab,
                                          err);
}

void launch_contact_sa(const Params& P, const float4* pos4, const uint8_t* sstate,
                       const uint32_t* ids, const uint32_t* skeys, const uint4* tab,
                       int64_t n, uint8_t* freeze, int32_t* pairs, int64_t pair_cap,
                       unsigned long long* npairs, cudaStream_t st) {
  if (n > 0)
    k_contact_sa<<<blocks(n), 256, 0, st>>>(P, pos4, sstate, ids, skeys, tab, n, freeze, pairs,
                                            pair_cap, npairs);
}


void launch_group_build(const Params& P, const uint32_t* keys, int64_t n, uint32_t ng,
                        uint32_t* gcnt, uint32_t* gofs, uint32_t* gbsum, uint32_t* gfill,
                        uint32_t* perm, uint32_t* gkey, uint32_t* gdest, const int4* rin,
                        int4* rout, float4* pos4, uint32_t* skeys, uint32_t* svals,
                        uint8_t* sact, uint4* tab, uint32_t stamp, uint32_t* act, DevStats* dst,
                        int sms, ProfHook* prof, cudaStream_t st, const uint32_t* okey,
                        const float4* opos, const uint32_t* ogofs, int64_t no, uint32_t* msrc,
                        uint32_t obase, uint32_t* rbuild, uint32_t build, int reuse) {
  if (n <= 0) return;
  if (prof) prof->begin(K_GROUP);
  cudaMemsetAsync(gcnt, 0, 4 * (size_t)ng, st);
  cudaMemsetAsync(gfill, 0, 4 * (size_t)ng, st);
  const unsigned g1 = (unsigned)std::min<int64_t>(blocks(n), (int64_t)sms * 16);
  k_group_count<<<g1, 256, 0, st>>>(keys, n, ng, gcnt, &dst->err);
  const int64_t nb = ((int64_t)ng + 255) / 256;
  k_scan_blocks<<<(unsigned)nb, 256, 0, st>>>(gcnt, ng, gofs, gbsum);
  k_scan_sums<<<1, 256, 0, st>>>(gbsum, nb);
  k_group_scatter<<<g1, 256, 0, st>>>(keys, n, ng, gofs, gbsum, gfill, perm, gkey, &dst->err);
  if (prof) prof->end(K_GROUP, (double)n, 4);
  if (prof) prof->begin(K_BUILD);
  // one wave: 32 KB of shared memory per CTA leaves room for six CTAs per SM
  k_group_order<<<(unsigned)(sms * 6), 256, 0, st>>>(gkey, gofs, gbsum, ng, n, P.geo.seg0, gdest,
                                                     tab, stamp, dst, okey, opos, ogofs, no, pos4,
                                                     skeys, msrc, no ? obase : 0u, rbuild,
                                                     build, reuse);
  k_group_gather<<<blocks(n), 256, 0, st>>>(P, gkey, perm, gdest, n, rin, rout, pos4, skeys, svals,
                                            sact, msrc, n + no, dst);
  k_act_list<<<blocks(n, 256 * kActItems), 256, 0, st>>>(sact, n, act, dst);
  if (prof) prof->end(K_BUILD, (double)(n + no), 3);  // entries of the cell-ordered sequence
}

}  // namespace gp
