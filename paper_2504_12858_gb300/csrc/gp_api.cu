// C ABI of the grain-envelope particle library: context, memory, time loop.
// The declarations and the contract of every entry point are in include/gp.h.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/gp.h"
#include "gp_kernels.cuh"

using namespace gp;

namespace {

constexpr size_t kAlign = 256;
// record-steps of carrying a FROZEN record in the dynamic store (ordering, gather,
// emit) that cost about as much as merging one record into the obstacle store
constexpr double kObsCarry = 3.0;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// hash geometry of one run and its place in the context-wide key, cell-table and
// reached-head ranges
struct RunLayout {
  int nc[3];
  int nsx;
  uint64_t ncells, nseg, nheads;
  uint64_t key0, seg0, head0;
};

struct Layout {
  bool batch = false;
  int nruns = 1;
  int hshift = 0;       // reached-site heads per 2^hshift cells along each axis
  std::vector<RunLayout> run;
  uint64_t key_end = 0;  // keys of all runs lie in [0, key_end)
  uint64_t nseg = 0, nheads = 0;
  int nbits = 0, key_bytes = 4;
  int64_t cap = 0, rcap = 0, blocks = 0, buckets = 0;
  int max_grains = 0, max_nuclei = 0;
  int64_t grid_nodes = 0;
  int64_t solute_nodes = 0;
  int64_t tape_steps = 0;
  int64_t tape_every = 1;  // checkpoint interval of the adjoint tape
  // offsets into the arena
  size_t rec0, rec1, pos4, sslot, act, keys0, keys1, vals0, vals1, sstatus, hist, tickets, cells,
      rkey, rnext, rhead, ckeys, cdata, gtab, npos, ngrain, nstate, nmeta, gflags, gdtn, dstats, grid,
      sgrid, runs,
      rtherm, rcount, tape_post, tape_par, tape_code, tape_ckpt, tape_replay, tape_svals,
      tape_grad, gcnt, gofs, gfill,
      gbsum, gkey, gdest, orec[2], opos[2], okey[2], otcnt, ogofs[2], msrc, rbuild, total;
  uint32_t ngroups = 0;  // one run: cell groups of the record grouping
};

bool cells_of(const gp_domain* d, double h, int nc[3], uint64_t* ncells) {
  return hash_cells(d->lo, d->hi, h, nc, ncells);
}

int64_t pow2_at_least(int64_t v) {
  int64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

int bits_for(uint64_t end) {
  uint64_t m = end ? end - 1 : 0;
  int b = 0;
  while (m) {
    ++b;
    m >>= 1;
  }
  return b;
}

bool make_layout(const gp_domain* d, int nruns, bool batch, double h, const gp_memory* m,
                 Layout* L, std::string* why) {
  if (!d || !m || !(h > 0) || nruns < 1 || nruns > kMaxRuns || (!batch && nruns != 1)) {
    *why = "domain, memory, h > 0 and 1..256 runs are required";
    return false;
  }
  L->batch = batch;
  L->nruns = nruns;
  L->hshift = batch ? 2 : 0;
  L->run.assign(nruns, RunLayout{});
  uint64_t key = 0, seg = 0, head = 0;
  for (int r = 0; r < nruns; ++r) {
    RunLayout& R = L->run[r];
    if (!cells_of(d + r, h, R.nc, &R.ncells)) {
      *why = "domain too large for the spatial hash (more than 4096 cells per axis or 2^32 cells)";
      return false;
    }
    double diag = 0;
    for (int a = 0; a < 3; ++a) diag += (d[r].hi[a] - d[r].lo[a]) * (d[r].hi[a] - d[r].lo[a]);
    if (std::sqrt(diag) / h > 4000.0) {
      *why = "domain diagonal exceeds 4000 lattice spacings";
      return false;
    }
    R.nsx = (R.nc[0] + kSegCells - 1) / kSegCells;
    // the particle step orders cells in tiles of 16 x 8 x 8 (x fastest): the key range
    // and the cell table cover whole tiles
    const int ty = (R.nc[1] + (1 << kTileYShift) - 1) >> kTileYShift;
    const int tz = (R.nc[2] + (1 << kTileZShift) - 1) >> kTileZShift;
    const uint64_t tiles = (uint64_t)R.nsx * ty * tz;
    R.nseg = tiles << (kTileYShift + kTileZShift);
    R.ncells = R.nseg << kSegShift;
    if (R.ncells >= (1ull << 32)) {
      *why = "domain too large for the spatial hash (2^32 cells in whole tiles)";
      return false;
    }
    const int hm = (1 << L->hshift) - 1;
    R.nheads = (uint64_t)((R.nc[0] + hm) >> L->hshift) * ((R.nc[1] + hm) >> L->hshift) *
               ((R.nc[2] + hm) >> L->hshift);
    R.key0 = key;
    R.seg0 = seg;
    R.head0 = head;
    key += R.ncells;
    seg += R.nseg;
    head += R.nheads;
  }
  L->key_end = key;
  L->nseg = seg;
  L->nheads = head;
  L->key_bytes = batch ? 8 : 4;
  L->nbits = bits_for(key);
  if (L->nbits > 8 * kSortMaxPasses || (!batch && L->nbits > 32)) {
    *why = "too many hash cells over all runs";
    return false;
  }
  if (m->capacity <= 0 || m->capacity >= (1ll << 30)) {
    *why = "capacity must be in [1, 2^30)";
    return false;
  }
  L->cap = m->capacity;
  L->rcap = m->reached_capacity > 0 ? m->reached_capacity : 2 * m->capacity;
  if (L->rcap >= (1ll << 32) - 1) L->rcap = (1ll << 32) - 2;
  L->blocks = m->claim_blocks > 0 ? m->claim_blocks : std::max<int64_t>(4096, m->capacity / 32);
  L->buckets = pow2_at_least(2 * L->blocks);
  if (L->buckets > (1ll << 31) || L->blocks >= (1ll << 32) - 1) {
    *why = "claim_blocks too large";
    return false;
  }
  L->max_grains = m->max_grains > 0 ? m->max_grains : (1 << 20);
  if (L->max_grains > (1 << kRunShift)) {
    *why = "max_grains must be <= 2^24";
    return false;
  }
  L->max_nuclei = m->max_nuclei > 0 ? m->max_nuclei : 4096;
  L->grid_nodes = m->grid_nodes > 0 ? m->grid_nodes : 0;
  L->solute_nodes = m->solute_nodes > 0 ? m->solute_nodes : 0;
  L->tape_steps = m->tape_steps > 0 ? m->tape_steps : 0;
  L->tape_every = m->tape_checkpoint_every > 0 ? m->tape_checkpoint_every : 1;
  if (batch && (L->grid_nodes || L->tape_steps || L->solute_nodes)) {
    *why = "a batch of runs takes analytic fields only and no adjoint tape";
    return false;
  }
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  const size_t cap = (size_t)L->cap;
  const size_t kb = (size_t)L->key_bytes;
  // one run: the obstacle store's positions and keys (two copies) follow the cell-ordered
  // sequence's own in pos4 and keys1, so that the contact search reads both through one
  // index (entries cap + b * ocap + i of copy b)
  const size_t ocap = batch ? 1 : cap;
  L->rec0 = take(16 * cap);
  L->rec1 = take(16 * cap);
  L->pos4 = take(16 * (cap + 2 * ocap));
  L->sslot = take(4 * cap);
  L->keys0 = take(kb * cap + 16);
  L->keys1 = take(kb * (cap + 2 * ocap) + 16);
  L->vals0 = take(4 * cap + 16);
  L->vals1 = take(4 * cap + 16);
  L->sstatus = take(4 * radix_status_words(L->cap, L->key_bytes));
  L->hist = take(4 * 256 * (size_t)((L->nbits + 7) / 8));  // one histogram per digit
  L->tickets = take(4 * 8);
  L->cells = take(16 * (size_t)L->nseg);
  L->rkey = take(8 * (size_t)L->rcap);
  L->rnext = take(4 * (size_t)L->rcap);
  L->rhead = take(4 * (size_t)L->nheads);
  L->ckeys = take(16 * (size_t)L->buckets);
  L->cdata = take(4 * kBrickWords * (size_t)L->blocks);
  L->gtab = take(64 * (size_t)L->max_grains);
  L->npos = take(16 * (size_t)L->max_nuclei);
  L->ngrain = take(64 * (size_t)L->max_nuclei);
  L->nstate = take(4 * (size_t)L->max_nuclei);
  L->dstats = take(sizeof(DevStats));
  L->grid = take(4 * (size_t)L->grid_nodes);
  // adjoint tape: per step the post-contact states, parents and directions (6 bytes per
  // particle), the store at every tape_every-th step (16 bytes), two stores for the
  // replay and the sorted-to-store map of the step being taped
  const size_t ts = (size_t)L->tape_steps;
  const size_t nck = (ts + (size_t)L->tape_every - 1) / (size_t)L->tape_every;
  L->tape_post = take(cap * ts);
  L->tape_par = take(4 * cap * ts);
  L->tape_code = take(cap * ts);
  L->tape_ckpt = take(16 * cap * nck);
  L->tape_replay = take(ts ? 32 * cap : 16);
  L->tape_svals = take(ts ? 4 * cap : 16);
  L->tape_grad = take(8 * 8);
  L->act = take(4 * cap);
  L->nmeta = take(8 * (size_t)L->max_nuclei);
  L->sgrid = take(4 * (size_t)L->solute_nodes);
  L->gflags = take(4 * (size_t)L->max_grains);
  L->gdtn = take(4 * (size_t)L->max_grains);
  L->runs = take(sizeof(Geo) * (size_t)nruns);
  L->rtherm = take(16 * (size_t)nruns);
  L->rcount = take(16 * (size_t)nruns);
  // one run: counts, offsets and fill cursors of the cell groups
  L->ngroups = batch ? 0u : (uint32_t)(L->run[0].ncells >> kGroupShift);
  L->gcnt = take(4 * (size_t)L->ngroups + 16);
  L->gofs = take(4 * (size_t)L->ngroups + 16);
  L->gfill = take(4 * (size_t)L->ngroups + 16);
  L->gbsum = take(4 * (((size_t)L->ngroups + 255) / 256) + 16);
  L->rbuild = take(4 * (size_t)L->ngroups + 16);  // build that last wrote a group resident
  L->gkey = take(batch ? 16 : 4 * cap + 16);   // one run: cell keys in grouped order
  L->gdest = take(batch ? 16 : 4 * cap + 16);  // and the sorted position of each
  // one run: the obstacle store (FROZEN records ordered by cell key, positions, keys,
  // the first obstacle of every group; two copies, a flush writes one from the other),
  // the source of every entry of the cell-ordered sequence and the flush's tile counts
  for (int b = 0; b < 2; ++b) {
    L->orec[b] = take(16 * ocap);
    L->opos[b] = L->pos4 + 16 * (cap + b * ocap);
    L->okey[b] = L->keys1 + 4 * (cap + b * ocap);
    L->ogofs[b] = take(4 * ((size_t)L->ngroups + 16));
  }
  L->msrc = take(4 * ocap + 16);
  L->otcnt = take(4 * (ocap / 8192 + 16));
  L->total = o;
  return true;
}

// T_L - T0 - Tdot t_n of an analytic field with a = T_L - T0 (every product and
// difference rounded once, as the device-side batch computation does)
float dT_base_at(double a, double Tdot, int64_t n, double dt) {
  volatile double t = (double)n * dt;
  volatile double q = Tdot * t;
  return (float)(a - q);
}

// rotation (crystal -> lab) of a unit quaternion (w, x, y, z)
void quat_rot(const double* qin, double R[9]) {
  double n = std::sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
  double w = qin[0] / n, x = qin[1] / n, y = qin[2] / n, z = qin[3] / n;
  R[0] = 1 - 2 * (y * y + z * z);
  R[1] = 2 * (x * y - w * z);
  R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);
  R[4] = 1 - 2 * (x * x + z * z);
  R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);
  R[7] = 2 * (y * z + w * x);
  R[8] = 1 - 2 * (x * x + y * y);
}

// grain table entry: c (with the run id in w), then the rows of h R
void grain_entry(const double* pos, const double* q, double h, int run, float4 out[4]) {
  double R[9];
  quat_rot(q, R);
  float w;
  std::memcpy(&w, &run, sizeof(w));
  out[0] = make_float4((float)pos[0], (float)pos[1], (float)pos[2], w);
  for (int r = 0; r < 3; ++r)
    out[1 + r] = make_float4((float)(h * R[3 * r]), (float)(h * R[3 * r + 1]),
                             (float)(h * R[3 * r + 2]), 0.f);
}

const char* kKernelNames[K_COUNT] = {"hist",      "onesweep", "keys",     "build",
                                     "advance",   "emit",     "nucleate", "grain_map",
                                     "seed",      "contact",  "cells",    "finalize",
                                     "group",     "obstacle"};
// algorithmic DRAM bytes per processed item:
//   hist      read key (4)
//   onesweep  read key + value, write key + value (16)
//   keys      read record (16), write key + value (8)
//   build     read value + key (8), gather record (16), write record (16), write
//             position + grain (16)
//   advance   per ACTIVE particle: read list index (4), record (16) and own position
//             (16), write record (16); neighbour positions are re-reads of the same
//             cells (cache)
//   emit      read record (16), write record (16) + key + value (8) per output
//   group     read key twice (8), write the grouped identity (4)
//   obstacle  per record of the merged obstacle store: read and write its key,
//             position and record (72)
const double kKernelBytes[K_COUNT] = {4, 16, 24, 56, 52, 40, 0, 0, 0, 0, 0, 0, 12, 72};

struct Prof : ProfHook {
  cudaStream_t st = nullptr;
  bool on = false;
  struct Ev {
    cudaEvent_t a, b;
    int kid;
    double units;
    int kernels;
  };
  std::vector<Ev> pending;
  std::vector<cudaEvent_t> pool;
  int64_t launches[K_COUNT] = {};
  double ms[K_COUNT] = {};
  double units[K_COUNT] = {};
  cudaEvent_t cur = nullptr;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  // every timed segment is also an NVTX range named like its entry (a no-op unless a
  // tracing tool is attached)
  void begin(int kid) override {
    nvtxRangePushA(kKernelNames[kid]);
    if (!on) return;
    cur = get();
    cudaEventRecord(cur, st);
  }
  void end(int kid, double u, int kernels = 1) override {
    nvtxRangePop();
    if (!on || !cur) return;
    cudaEvent_t e = get();
    cudaEventRecord(e, st);
    pending.push_back({cur, e, kid, u, kernels});
    cur = nullptr;
    if (pending.size() > 4096) flush();
  }
  void flush() {
    if (pending.empty()) return;
    cudaStreamSynchronize(st);
    for (auto& p : pending) {
      float t = 0;
      cudaEventElapsedTime(&t, p.a, p.b);
      launches[p.kid] += p.kernels;
      ms[p.kid] += t;
      units[p.kid] += p.units;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  void reset() {
    flush();
    for (int i = 0; i < K_COUNT; ++i) {
      launches[i] = 0;
      ms[i] = 0;
      units[i] = 0;
    }
  }
  ~Prof() override {
    for (auto& p : pending) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

}  // namespace

struct gp_ctx {
  int device = 0;
  cudaStream_t st = nullptr;
  bool own = false;
  char* base = nullptr;
  Layout L{};
  bool batch = false;                // several independent runs (gp_batch_create)
  std::vector<gp_domain> dom;        // per run
  double h = 0, dt = 0;
  gp_growth_law law{};
  Params P{};
  // thermal
  int thermal = 0;                   // 1 analytic (every run), 2 grid (single run)
  std::vector<double> T0, Tdot;      // analytic field per run
  std::vector<char> thermal_set;     // per run
  double gorigin[3] = {0, 0, 0}, gvel[3] = {0, 0, 0};
  float* grid_own = nullptr;  // cudaMalloc'ed grid when the arena has none
  size_t grid_own_bytes = 0;
  // composition field (local liquidus)
  double worigin[3] = {0, 0, 0}, wvel[3] = {0, 0, 0};
  float* wgrid_own = nullptr;
  size_t wgrid_own_bytes = 0;
  // device views
  int4* rec[2] = {nullptr, nullptr};
  int cur = 0;  // rec[cur] is the (unsorted) store
  float4* pos4 = nullptr;
  int32_t* site_slot = nullptr;  // claim-block slot of each crossing particle's reached site
  uint32_t* act = nullptr;       // sorted indices of the ACTIVE particles (built per step)
  SortBufs sb{};
  uint4* cells = nullptr;
  uint32_t stamp = 0;
  Claims C{};
  Reached R{};
  float4* gtab = nullptr;
  float4* npos = nullptr;
  float4* ngrain = nullptr;
  int* nstate = nullptr;
  int2* nmeta = nullptr;             // batch: reserved grain and run of each nucleation site
  Geo* runs = nullptr;               // batch: per-run geometry table
  double2* rtherm = nullptr;         // batch: (T_L - T0, Tdot) per run
  unsigned long long* rcount = nullptr;
  std::vector<Geo> geo;              // host copy of the per-run geometry
  DevStats* dst = nullptr;
  DevStats* hst = nullptr;  // pinned mirror
  // host mirrors
  int64_t n_live = 0, n_grains = 0, step = 0;
  int n_nuclei = 0;
  bool keys_valid = false;
  bool broken = false;
  // adjoint tape: taped steps (sorted count n, count after the step m, step index)
  int periodic = 0;      // periodic axes (bit per axis), single run
  bool melting = false;  // melting walk-back pass at the start of every step
  uint8_t* gflags = nullptr;
  float* gdtn = nullptr;  // nucleation undercooling of each grain's seed
  bool tape_on = false;
  int64_t tape_pos = 0;
  std::vector<int64_t> tape_n, tape_m, tape_t;
  std::string err;
  Prof prof;
  int sms = 152;
  // batch: steps per captured CUDA graph (0: launches issued step by step) and the
  // instantiated graphs by step count
  int graph_steps = 0;
  std::map<int, cudaGraphExec_t> graphs;
  // obstacle store of a single run: n_obs FROZEN records in copy ocur; obs_carry sums
  // the FROZEN records the dynamic store carried since the last flush
  int64_t n_obs = 0;
  int ocur = 0;
  double obs_carry = 0;
  int obs_mode = 1;  // 0 off, 1 flushes when carrying costs as much as merging, 2 every step
  // builds of the single-run ordering (tags in L.rbuild) and whether the next build may keep
  // the table entries of groups that hold only obstacles: not after a flush, a change of
  // the store, a wrap of the table stamp or a build by the inspection
  uint32_t nbuild = 1;
  bool table_reuse = false;
};

namespace {

gp_status fail(gp_ctx* c, gp_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

gp_status cuda_check(gp_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return GP_OK;
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (c) {
    c->err = m;
    c->broken = true;
  }
  return GP_ERR_CUDA;
}

#define GP_CUDA(c, call)                                  \
  do {                                                    \
    gp_status _s = cuda_check((c), (call), #call);        \
    if (_s != GP_OK) return _s;                           \
  } while (0)

template <class T>
T* at(gp_ctx* c, size_t off) {
  return reinterpret_cast<T*>(c->base + off);
}

void refresh_params(gp_ctx* c) {
  Params& P = c->P;
  c->geo.assign(c->L.nruns, Geo{});
  const float inv_c = (float)(1.0 / cell_edge(c->h));
  for (int r = 0; r < c->L.nruns; ++r) {
    Geo& g = c->geo[r];
    const RunLayout& R = c->L.run[r];
    for (int a = 0; a < 3; ++a) {
      g.lo[a] = (float)c->dom[r].lo[a];
      g.hi[a] = (float)c->dom[r].hi[a];
      g.nc[a] = R.nc[a];
      g.inv[a] = inv_c;
      if ((c->periodic >> a) & 1) {  // the period in floor(L / edge) equal cells
        const double L = c->dom[r].hi[a] - c->dom[r].lo[a];
        g.nc[a] = (int)std::floor(L / cell_edge(c->h));
        g.inv[a] = (float)(g.nc[a] / L);
      }
    }
    g.nsx = (g.nc[0] + kSegCells - 1) / kSegCells;
    g.tx = g.nsx;
    g.ty = (g.nc[1] + (1 << kTileYShift) - 1) >> kTileYShift;
    g.key0 = R.key0;
    g.seg0 = R.seg0;
    g.head0 = R.head0;
  }
  P.geo = c->geo[0];
  P.runs = c->batch ? c->runs : nullptr;
  P.periodic = c->periodic;
  for (int a = 0; a < 3; ++a) P.per_L[a] = (float)(c->dom[0].hi[a] - c->dom[0].lo[a]);
  P.hshift = c->L.hshift;
  P.inv_c = (float)(1.0 / cell_edge(c->h));
  float hf = (float)c->h;
  P.rc2 = hf * hf;
  P.dt_over_h = (float)(c->dt / c->h);
  P.nterms = c->law.nterms;
  for (int i = 0; i < 2; ++i) {
    P.a[i] = (float)c->law.a[i];
    P.b[i] = (float)c->law.b[i];
    double bi = c->law.b[i];
    P.bint[i] = (bi == std::floor(bi) && bi >= 1.0 && bi <= 8.0) ? (int)bi : -1;
  }
  P.TL = (float)c->law.T_liquidus;
  P.gtab = c->gtab;
}

StepArgs step_args(const gp_ctx* c, int64_t n) {
  StepArgs S{};
  const double t = (double)n * c->dt;
  for (int a = 0; a < 3; ++a) {
    S.gshift[a] = (float)(c->gorigin[a] + c->gvel[a] * t);
    S.wshift[a] = (float)(c->worigin[a] + c->wvel[a] * t);
  }
  S.parity = (int)(n & 1);
  return S;
}

// kernel constants for step n of a single-run context (analytic field at t_n and
// t_{n+1}); a batch computes its runs' values on the device (launch_run_step)
Params step_params(const gp_ctx* c, int64_t n) {
  Params P = c->P;
  if (!c->batch && c->thermal == 1) {
    const double a = c->law.T_liquidus - c->T0[0];
    P.geo.dT_base = dT_base_at(a, c->Tdot[0], n, c->dt);
    P.geo.dT_base1 = dT_base_at(a, c->Tdot[0], n + 1, c->dt);
  }
  return P;
}

gp_status sync_stats(gp_ctx* c) {
  GP_CUDA(c, cudaMemcpyAsync(c->hst, c->dst, sizeof(DevStats), cudaMemcpyDeviceToHost, c->st));
  GP_CUDA(c, cudaStreamSynchronize(c->st));
  uint32_t e = c->hst->err | *((volatile uint32_t*)&c->hst->err);
  c->n_live = (int64_t)c->hst->n_live;
  c->n_grains = (int64_t)c->hst->n_grains;
  if (e) {
    c->broken = true;
    if (e & ERR_CAPACITY) return fail(c, GP_ERR_CAPACITY, "particle capacity exceeded");
    if (e & ERR_REACHED_CAP) return fail(c, GP_ERR_CAPACITY, "reached-site capacity exceeded");
    if (e & ERR_GRAINS) return fail(c, GP_ERR_CAPACITY, "grain capacity exceeded");
    if (e & ERR_HASH_FULL) return fail(c, GP_ERR_HASH_FULL, "claim table full (raise claim_blocks)");
    if (e & ERR_TIMEOUT) return fail(c, GP_ERR_TIMEOUT, "bounded device wait gave up");
    if (e & ERR_CELL_OVERFLOW) return fail(c, GP_ERR_CAPACITY, "32767 or more particles in a row of 16 hash cells");
    if (e & ERR_SITE_RANGE) return fail(c, GP_ERR_ARG, "lattice site outside [-4095, 4095]");
    return fail(c, GP_ERR_STATE, "device error");
  }
  return GP_OK;
}

// writes the host mirrors of n_live / n_grains into the device counters
gp_status push_counts(gp_ctx* c) {
  c->hst->n_live = (unsigned long long)c->n_live;
  c->hst->n_grains = (unsigned long long)c->n_grains;
  c->hst->step = (unsigned long long)c->step;
  GP_CUDA(c, cudaMemcpyAsync(&c->dst->n_frozen, &c->hst->n_frozen, sizeof(unsigned long long),
                             cudaMemcpyHostToDevice, c->st));
  GP_CUDA(c, cudaMemcpyAsync(&c->dst->step, &c->hst->step, sizeof(unsigned long long),
                             cudaMemcpyHostToDevice, c->st));
  GP_CUDA(c, cudaMemcpyAsync(&c->dst->n_live, &c->hst->n_live, sizeof(unsigned long long),
                             cudaMemcpyHostToDevice, c->st));
  GP_CUDA(c, cudaMemcpyAsync(&c->dst->n_grains, &c->hst->n_grains, sizeof(unsigned long long),
                             cudaMemcpyHostToDevice, c->st));
  GP_CUDA(c, cudaStreamSynchronize(c->st));
  return GP_OK;
}

// The obstacle store serves the plain single-run step.  Periodic axes, melting (which
// removes frozen particles) and the adjoint tape (which follows every particle through
// every step) keep all particles in the dynamic store.
bool obs_usable(const gp_ctx* c) {
  return c->obs_mode != 0 && !c->batch && !c->periodic && !c->melting && !c->tape_on;
}

// empties the obstacle store (its table back to all-empty entries)
gp_status obs_reset(gp_ctx* c) {
  c->n_obs = 0;
  c->obs_carry = 0;
  c->table_reuse = false;
  return GP_OK;
}

// moves the obstacle records back to the end of the dynamic store (its keys are then
// recomputed before the next ordering)
gp_status obs_return(gp_ctx* c) {
  if (c->n_obs == 0) return GP_OK;
  if (c->n_live + c->n_obs > c->L.cap) return fail(c, GP_ERR_CAPACITY, "particle capacity");
  launch_append(at<int4>(c, c->L.orec[c->ocur]), c->n_obs, c->rec[c->cur], c->n_live, c->st);
  GP_CUDA(c, cudaGetLastError());
  c->n_live += c->n_obs;
  c->hst->n_frozen += (unsigned long long)c->n_obs;
  c->keys_valid = false;
  gp_status s = obs_reset(c);
  if (s) return s;
  return push_counts(c);
}

void drop_graphs(gp_ctx* c) {
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.second);
  c->graphs.clear();
}

gp_status check_ctx(gp_ctx* c) {
  if (!c) return GP_ERR_ARG;
  if (c->broken) return fail(c, GP_ERR_STATE, "context is in an error state: " + c->err);
  GP_CUDA(c, cudaSetDevice(c->device));
  return GP_OK;
}

// L1 sphere |t|_1 = m of the integer lattice, as short4 offsets
std::vector<short4> l1_sphere(int m) {
  std::vector<short4> v;
  if (m == 0) {
    v.push_back(make_short4(0, 0, 0, 0));
    return v;
  }
  for (int x = -m; x <= m; ++x)
    for (int y = -(m - std::abs(x)); y <= m - std::abs(x); ++y) {
      int rz = m - std::abs(x) - std::abs(y);
      v.push_back(make_short4((short)x, (short)y, (short)rz, 0));
      if (rz) v.push_back(make_short4((short)x, (short)y, (short)-rz, 0));
    }
  return v;
}

gp_status create_ctx(const gp_domain* domains, int nruns, bool batch, double h, double dt,
                     const gp_growth_law* law, const gp_memory* mem, void* cuda_stream,
                     gp_ctx** out) {
  if (!out || !domains || !law || !mem) return GP_ERR_ARG;
  *out = nullptr;
  if (!(dt > 0) || law->nterms < 1 || law->nterms > 2) return GP_ERR_ARG;
  for (int i = 0; i < law->nterms; ++i)
    if (!std::isfinite(law->a[i]) || !std::isfinite(law->b[i]) || law->b[i] < 0) return GP_ERR_ARG;
  gp_ctx* c = new gp_ctx();
  std::string why;
  if (!make_layout(domains, nruns, batch, h, mem, &c->L, &why)) {
    delete c;
    return GP_ERR_ARG;
  }
  c->batch = batch;
  cudaGetDevice(&c->device);
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  c->st = (cudaStream_t)cuda_stream;
  c->dom.assign(domains, domains + nruns);
  c->T0.assign(nruns, 0.0);
  c->Tdot.assign(nruns, 0.0);
  c->thermal_set.assign(nruns, 0);
  c->h = h;
  c->dt = dt;
  c->law = *law;
  if (c->law.nterms == 1) {
    c->law.a[1] = 0;
    c->law.b[1] = 0;
  }
  if (mem->arena) {
    if (mem->arena_bytes < c->L.total || ((uintptr_t)mem->arena & (kAlign - 1))) {
      delete c;
      return GP_ERR_ARG;
    }
    c->base = (char*)mem->arena;
  } else {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, c->L.total);
    if (e != cudaSuccess) {
      delete c;
      return e == cudaErrorMemoryAllocation ? GP_ERR_CAPACITY : GP_ERR_CUDA;
    }
    c->base = (char*)p;
    c->own = true;
  }
  if (cudaMallocHost((void**)&c->hst, sizeof(DevStats)) != cudaSuccess) {
    if (c->own) cudaFree(c->base);
    delete c;
    return GP_ERR_CUDA;
  }
  std::memset(c->hst, 0, sizeof(DevStats));
  const Layout& L = c->L;
  c->rec[0] = at<int4>(c, L.rec0);
  c->rec[1] = at<int4>(c, L.rec1);
  c->pos4 = at<float4>(c, L.pos4);
  c->site_slot = at<int32_t>(c, L.sslot);
  c->act = at<uint32_t>(c, L.act);
  c->sb.keys[0] = c->base + L.keys0;
  c->sb.keys[1] = c->base + L.keys1;
  c->sb.vals[0] = at<uint32_t>(c, L.vals0);
  c->sb.vals[1] = at<uint32_t>(c, L.vals1);
  c->sb.status = at<uint32_t>(c, L.sstatus);
  c->sb.hist = at<uint32_t>(c, L.hist);
  c->sb.ticket = at<uint32_t>(c, L.tickets);
  c->sb.max_n = L.cap;
  c->sb.sms = c->sms;
  c->sb.prof = &c->prof;
  c->prof.st = c->st;
  c->cells = at<uint4>(c, L.cells);
  c->dst = at<DevStats>(c, L.dstats);
  c->sb.err = &c->dst->err;
  c->R.key = at<unsigned long long>(c, L.rkey);
  c->R.next = at<uint32_t>(c, L.rnext);
  c->R.head = at<uint32_t>(c, L.rhead);
  c->R.count = &c->dst->reached;
  c->R.cap = (unsigned long long)L.rcap;
  c->R.err = &c->dst->err;
  c->C.bucket = at<ulonglong2>(c, L.ckeys);
  c->C.data = at<uint32_t>(c, L.cdata);
  c->C.mask = (uint32_t)(L.buckets - 1);
  c->C.pool_cap = (uint32_t)L.blocks;
  c->C.used = &c->dst->claim_used;
  c->C.err = &c->dst->err;
  c->gtab = at<float4>(c, L.gtab);
  c->npos = at<float4>(c, L.npos);
  c->ngrain = at<float4>(c, L.ngrain);
  c->nstate = at<int>(c, L.nstate);
  c->gflags = at<uint8_t>(c, L.gflags);
  c->gdtn = at<float>(c, L.gdtn);
  c->nmeta = at<int2>(c, L.nmeta);
  c->runs = at<Geo>(c, L.runs);
  c->rtherm = at<double2>(c, L.rtherm);
  c->rcount = at<unsigned long long>(c, L.rcount);
  refresh_params(c);
  c->P.launch.build_ctas = 8 * c->sms;
  c->P.launch.advance_ctas = 8 * c->sms;
  c->P.launch.emit_ctas = 6 * c->sms;
  if (batch) c->sb.n_dev = &c->dst->n_live;  // device-sized sort
  cudaStream_t s = c->st;
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMemsetAsync(c->cells, 0, 16 * L.nseg, s);
  if (L.ngroups) e = e ? e : cudaMemsetAsync(c->base + L.rbuild, 0, 4 * (size_t)L.ngroups, s);
  e = e ? e : cudaMemsetAsync(c->R.head, 0xff, 4 * L.nheads, s);
  e = e ? e : cudaMemsetAsync(c->C.bucket, 0, 16 * (size_t)L.buckets, s);
  e = e ? e : cudaMemsetAsync(c->C.data, 0, 4 * kBrickWords * (size_t)L.blocks, s);
  e = e ? e : cudaMemsetAsync(c->dst, 0, sizeof(DevStats), s);
  e = e ? e : cudaMemsetAsync(c->gtab, 0, 64 * (size_t)L.max_grains, s);
  e = e ? e : cudaMemsetAsync(c->nstate, 0, 4 * (size_t)L.max_nuclei, s);
  e = e ? e : cudaMemsetAsync(c->gflags, 0, 4 * (size_t)L.max_grains, s);
  e = e ? e : cudaMemsetAsync(c->gdtn, 0, 4 * (size_t)L.max_grains, s);
  e = e ? e : cudaMemsetAsync(c->rtherm, 0, 16 * (size_t)L.nruns, s);
  e = e ? e : cudaMemcpyAsync(c->runs, c->geo.data(), sizeof(Geo) * c->geo.size(),
                              cudaMemcpyHostToDevice, s);
  if (batch) {  // a batch's step and stamp counters live on the device
    c->stamp = 1;
    c->hst->stamp = 1;
    e = e ? e : cudaMemcpyAsync(&c->dst->stamp, &c->hst->stamp, sizeof(unsigned long long),
                                cudaMemcpyHostToDevice, s);
  }
  e = e ? e : cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    gp_destroy(c);
    return GP_ERR_CUDA;
  }
  *out = c;
  return GP_OK;
}

}  // namespace

extern "C" {

gp_status gp_arena_bytes(const gp_domain* domain, double h, const gp_memory* mem,
                         size_t* out_bytes) {
  if (!out_bytes) return GP_ERR_ARG;
  Layout L{};
  std::string why;
  if (!make_layout(domain, 1, false, h, mem, &L, &why)) return GP_ERR_ARG;
  *out_bytes = L.total;
  return GP_OK;
}

gp_status gp_batch_arena_bytes(int32_t nruns, const gp_domain* domains, double h,
                               const gp_memory* mem, size_t* out_bytes) {
  if (!out_bytes) return GP_ERR_ARG;
  Layout L{};
  std::string why;
  if (!make_layout(domains, nruns, true, h, mem, &L, &why)) return GP_ERR_ARG;
  *out_bytes = L.total;
  return GP_OK;
}

gp_status gp_create(const gp_domain* domain, double h, double dt, const gp_growth_law* law,
                    const gp_memory* mem, void* cuda_stream, gp_ctx** out) {
  return create_ctx(domain, 1, false, h, dt, law, mem, cuda_stream, out);
}

gp_status gp_batch_create(int32_t nruns, const gp_domain* domains, double h, double dt,
                          const gp_growth_law* law, const gp_memory* mem, void* cuda_stream,
                          gp_ctx** out) {
  return create_ctx(domains, nruns, true, h, dt, law, mem, cuda_stream, out);
}

gp_status gp_destroy(gp_ctx* c) {
  if (!c) return GP_ERR_ARG;
  cudaSetDevice(c->device);
  if (c->st) cudaStreamSynchronize(c->st);
  else cudaDeviceSynchronize();
  c->prof.pending.clear();
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.second);
  if (c->own && c->base) cudaFree(c->base);
  if (c->grid_own) cudaFree(c->grid_own);
  if (c->wgrid_own) cudaFree(c->wgrid_own);
  if (c->hst) cudaFreeHost(c->hst);
  delete c;
  return GP_OK;
}

const char* gp_last_error(const gp_ctx* c) { return c ? c->err.c_str() : "null context"; }

gp_status gp_add_grains(gp_ctx* c, int64_t n, const double* pos3, const double* quat4,
                        int32_t nucleate, int32_t* out_first_id) {
  return gp_run_add_grains(c, 0, n, pos3, quat4, nucleate, out_first_id);
}

gp_status gp_run_add_grains(gp_ctx* c, int32_t run, int64_t n, const double* pos3,
                            const double* quat4, int32_t nucleate, int32_t* out_first_id) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (run < 0 || run >= c->L.nruns) return fail(c, GP_ERR_ARG, "no such run");
  if (n < 0 || (n > 0 && (!pos3 || !quat4))) return fail(c, GP_ERR_ARG, "bad arguments");
  if (c->n_grains + n > c->L.max_grains) return fail(c, GP_ERR_CAPACITY, "grain capacity");
  if (nucleate && c->n_live + c->n_obs + 6 * n > c->L.cap)
    return fail(c, GP_ERR_CAPACITY, "particle capacity");
  for (int64_t i = 0; i < n; ++i) {
    const double* q = quat4 + 4 * i;
    double nq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (!(nq > 0) || !std::isfinite(nq)) return fail(c, GP_ERR_ARG, "quaternion is zero or not finite");
    for (int a = 0; a < 3; ++a)
      if (!(pos3[3 * i + a] >= c->dom[run].lo[a] && pos3[3 * i + a] <= c->dom[run].hi[a]))
        return fail(c, GP_ERR_ARG, "nucleus outside the domain");
  }
  if (out_first_id) *out_first_id = (int32_t)c->n_grains;
  if (n == 0) return GP_OK;
  std::vector<float4> G(4 * (size_t)n);
  for (int64_t i = 0; i < n; ++i)
    grain_entry(pos3 + 3 * i, quat4 + 4 * i, c->h, run, &G[4 * i]);
  GP_CUDA(c, cudaMemcpyAsync(c->gtab + 4 * c->n_grains, G.data(), sizeof(float4) * G.size(),
                             cudaMemcpyHostToDevice, c->st));
  const int64_t g0 = c->n_grains;
  c->n_grains += n;
  if (nucleate) {
    // six nucleation particles per grain, staged through the sorted-record buffer
    // (idle between steps)
    std::vector<int4> recs(6 * (size_t)n);
    std::vector<int4> nuc(n), tgt(6 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
      const int g = (int)(g0 + i);
      nuc[i] = make_int4(g, 0, 0, 0);
      for (int k = 0; k < 6; ++k) {
        Rec r{};
        r.grain = g;
        r.dir = k;
        r.state = ST_ACTIVE;
        recs[6 * i + k] = rec_pack(r);
        int t[3] = {0, 0, 0};
        t[k >> 1] = (k & 1) ? -1 : 1;
        tgt[6 * i + k] = make_int4(g, t[0], t[1], t[2]);
      }
    }
    int4* stg = c->rec[c->cur ^ 1];
    GP_CUDA(c, cudaMemcpyAsync(stg, recs.data(), sizeof(int4) * recs.size(),
                               cudaMemcpyHostToDevice, c->st));
    launch_append(stg, (int64_t)recs.size(), c->rec[c->cur], c->n_live, c->st);
    // nucleus site: reached + claimed; first targets: claimed.  Site lists are
    // staged through the position buffer in chunks of its capacity.
    int4* sstg = reinterpret_cast<int4*>(c->pos4);
    const int64_t chunk = c->L.cap;
    for (int pass = 0; pass < 2; ++pass) {
      const std::vector<int4>& v = pass == 0 ? nuc : tgt;
      for (int64_t b = 0; b < (int64_t)v.size(); b += chunk) {
        const int64_t m = std::min<int64_t>(chunk, (int64_t)v.size() - b);
        GP_CUDA(c, cudaMemcpyAsync(sstg, v.data() + b, sizeof(int4) * m, cudaMemcpyHostToDevice,
                                   c->st));
        launch_mark_sites(c->P, sstg, m, pass == 0 ? 1 : 0, 1, c->C, c->R, c->st);
        GP_CUDA(c, cudaStreamSynchronize(c->st));
      }
    }
    c->n_live += 6 * n;
    c->keys_valid = false;
  }
  GP_CUDA(c, cudaGetLastError());
  s = push_counts(c);
  if (s) return s;
  return sync_stats(c);
}

gp_status gp_seed_shell(gp_ctx* c, int64_t n, const int32_t* grains, int32_t n0, double ell0) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (c->batch) return fail(c, GP_ERR_STATE, "shell seeding is for single-run contexts");
  if (n < 0 || (n > 0 && !grains) || n0 < 0 || n0 > 2000 || !(ell0 >= 0 && ell0 < 1))
    return fail(c, GP_ERR_ARG, "bad arguments");
  for (int64_t i = 0; i < n; ++i)
    if (grains[i] < 0 || grains[i] >= c->n_grains) return fail(c, GP_ERR_ARG, "unknown grain");
  if (n == 0) return GP_OK;
  std::vector<short4> toff = l1_sphere(n0 + 1), soff = l1_sphere(n0);
  // staging: grains + offsets in the key/value buffers (idle between steps)
  size_t need = 4 * (size_t)n + 8 * (toff.size() + soff.size()) + 1024;
  if (need > 16 * (size_t)c->L.cap) return fail(c, GP_ERR_CAPACITY, "staging too small for shell list");
  char* stg = reinterpret_cast<char*>(c->pos4);
  int32_t* dg = reinterpret_cast<int32_t*>(stg);
  short4* dt = reinterpret_cast<short4*>(stg + align_up(4 * (size_t)n));
  short4* ds = dt + toff.size();
  GP_CUDA(c, cudaMemcpyAsync(dg, grains, 4 * (size_t)n, cudaMemcpyHostToDevice, c->st));
  GP_CUDA(c, cudaMemcpyAsync(dt, toff.data(), 8 * toff.size(), cudaMemcpyHostToDevice, c->st));
  GP_CUDA(c, cudaMemcpyAsync(ds, soff.data(), 8 * soff.size(), cudaMemcpyHostToDevice, c->st));
  s = push_counts(c);
  if (s) return s;
  launch_seed_shell(c->P, dg, n, dt, (int64_t)toff.size(), (float)ell0, c->rec[c->cur],
                    c->L.cap - c->n_obs, &c->dst->n_live, c->C, &c->dst->err, c->st);
  launch_seed_shell_sites(c->P, dg, n, ds, (int64_t)soff.size(), c->C, c->R, c->st);
  GP_CUDA(c, cudaGetLastError());
  c->keys_valid = false;
  return sync_stats(c);
}

gp_status gp_set_thermal_analytic(gp_ctx* c, const gp_thermal_analytic* th) {
  return gp_run_set_thermal_analytic(c, 0, th);
}

gp_status gp_run_set_thermal_analytic(gp_ctx* c, int32_t run, const gp_thermal_analytic* th) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (run < 0 || run >= c->L.nruns) return fail(c, GP_ERR_ARG, "no such run");
  if (!th) return fail(c, GP_ERR_ARG, "null field");
  c->thermal = 1;
  c->P.thermal = 1;
  c->T0[run] = th->T0;
  c->Tdot[run] = th->Tdot;
  c->thermal_set[run] = 1;
  Geo& g = c->geo[run];
  for (int a = 0; a < 3; ++a) {
    g.G[a] = (float)th->G[a];
    g.xref[a] = (float)th->x_ref[a];
  }
  if (!c->batch) {
    for (int a = 0; a < 3; ++a) {
      c->P.geo.G[a] = g.G[a];
      c->P.geo.xref[a] = g.xref[a];
    }
    return GP_OK;
  }
  const double2 th2 = make_double2(c->law.T_liquidus - th->T0, th->Tdot);
  GP_CUDA(c, cudaMemcpyAsync(c->runs + run, &g, sizeof(Geo), cudaMemcpyHostToDevice, c->st));
  GP_CUDA(c, cudaMemcpyAsync(c->rtherm + run, &th2, sizeof(double2), cudaMemcpyHostToDevice,
                             c->st));
  GP_CUDA(c, cudaStreamSynchronize(c->st));
  return GP_OK;
}

gp_status gp_set_thermal_grid(gp_ctx* c, const gp_thermal_grid* th) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (c->batch) return fail(c, GP_ERR_STATE, "a batch of runs takes analytic fields only");
  if (!th || !th->T) return fail(c, GP_ERR_ARG, "null grid");
  for (int a = 0; a < 3; ++a)
    if (th->n[a] < 2 || !(th->spacing[a] > 0)) return fail(c, GP_ERR_ARG, "grid needs n >= 2 and spacing > 0");
  const size_t nodes = (size_t)th->n[0] * th->n[1] * th->n[2];
  float* dstp = nullptr;
  if ((int64_t)nodes <= c->L.grid_nodes) {
    dstp = at<float>(c, c->L.grid);
  } else if (c->own) {
    if (c->grid_own_bytes < 4 * nodes) {
      if (c->grid_own) cudaFree(c->grid_own);
      c->grid_own = nullptr;
      c->grid_own_bytes = 0;
      GP_CUDA(c, cudaMalloc((void**)&c->grid_own, 4 * nodes));
      c->grid_own_bytes = 4 * nodes;
    }
    dstp = c->grid_own;
  } else {
    return fail(c, GP_ERR_CAPACITY, "thermal grid larger than gp_memory.grid_nodes");
  }
  GP_CUDA(c, cudaMemcpyAsync(dstp, th->T, 4 * nodes,
                             (th->flags & GP_DEVICE_PTR) ? cudaMemcpyDeviceToDevice
                                                         : cudaMemcpyHostToDevice,
                             c->st));
  c->thermal = 2;
  c->P.thermal = 2;
  c->P.grid = dstp;
  for (int a = 0; a < 3; ++a) {
    c->P.gn[a] = th->n[a];
    c->P.ginv[a] = (float)(1.0 / th->spacing[a]);
    c->gorigin[a] = th->origin[a];
    c->gvel[a] = th->frame_vel[a];
  }
  return GP_OK;
}

gp_status gp_set_periodic(gp_ctx* c, int32_t axes) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (c->batch) return fail(c, GP_ERR_STATE, "periodic axes apply to single-run contexts");
  if (c->tape_on) return fail(c, GP_ERR_STATE, "the adjoint tape is recording");
  if (axes < 0 || axes > 7) return fail(c, GP_ERR_ARG, "axes is a bit mask of x, y, z");
  for (int a = 0; a < 3; ++a)
    if (((axes >> a) & 1) &&
        std::floor((c->dom[0].hi[a] - c->dom[0].lo[a]) / cell_edge(c->h)) < 3)
      return fail(c, GP_ERR_ARG, "a periodic axis needs at least three contact cells");
  if (axes) {  // the periodic contact search reads the dynamic store only
    s = obs_return(c);
    if (s) return s;
  }
  // the thermal constants set so far live in P.geo: keep them across the refresh
  const Geo keep = c->P.geo;
  c->periodic = axes;
  const Params old = c->P;
  refresh_params(c);
  c->P.thermal = old.thermal;
  c->P.grid = old.grid;
  for (int a = 0; a < 3; ++a) {
    c->P.gn[a] = old.gn[a];
    c->P.ginv[a] = old.ginv[a];
    c->P.wn[a] = old.wn[a];
    c->P.winv[a] = old.winv[a];
    c->P.geo.G[a] = keep.G[a];
    c->P.geo.xref[a] = keep.xref[a];
  }
  c->P.solute = old.solute;
  c->P.wgrid = old.wgrid;
  c->P.Tm = old.Tm;
  c->P.mL = old.mL;
  c->P.launch = old.launch;
  // cell geometry changed: keys are recomputed and the reached sites relinked
  c->keys_valid = false;
  c->table_reuse = false;
  GP_CUDA(c, cudaMemsetAsync(c->R.head, 0xff, 4 * c->L.nheads, c->st));
  GP_CUDA(c, cudaMemsetAsync(&c->dst->linked, 0, sizeof(unsigned long long), c->st));
  GP_CUDA(c, cudaStreamSynchronize(c->st));
  return GP_OK;
}

gp_status gp_set_melting(gp_ctx* c, int32_t enable) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (c->batch) return fail(c, GP_ERR_STATE, "melting applies to single-run contexts");
  if (enable && c->tape_on) return fail(c, GP_ERR_STATE, "the adjoint tape is recording");
  if (enable) {  // the melting pass removes frozen particles too: all in the dynamic store
    s = obs_return(c);
    if (s) return s;
  }
  c->melting = enable != 0;
  return GP_OK;
}

gp_status gp_set_obstacle_store(gp_ctx* c, int32_t mode) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (mode < 0 || mode > 2) return fail(c, GP_ERR_ARG, "mode is 0, 1 or 2");
  if (mode == 0) {
    s = obs_return(c);
    if (s) return s;
  }
  c->obs_mode = mode;
  return GP_OK;
}

gp_status gp_inspect_order(gp_ctx* c, int32_t which, int64_t cap, uint32_t* keys_in,
                           uint32_t* keys_sorted, uint32_t* src, int64_t* n_out, uint32_t* table,
                           int64_t table_cap, int64_t* n_seg, uint32_t* stamp) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (c->batch) return fail(c, GP_ERR_STATE, "the inspection is for single-run contexts");
  if ((which != 0 && which != 1) || cap < 0 || table_cap < 0)
    return fail(c, GP_ERR_ARG, "bad arguments");
  const int64_t nd = c->n_live, no = c->n_obs, o = c->ocur;
  if (which == 1) {  // the obstacle store: keys in its order, no table
    if (n_out) *n_out = no;
    if (n_seg) *n_seg = 0;
    if (stamp) *stamp = 0;
    const int64_t m = std::min(no, cap);
    if (m > 0 && keys_sorted)
      GP_CUDA(c, cudaMemcpyAsync(keys_sorted, at<uint32_t>(c, c->L.okey[o]), 4 * m,
                                 cudaMemcpyDeviceToHost, c->st));
    if (src)
      for (int64_t i = 0; i < m; ++i) src[i] = (uint32_t)(nd + i);
    GP_CUDA(c, cudaStreamSynchronize(c->st));
    return GP_OK;
  }
  const int64_t nseq = nd + no;
  if (n_out) *n_out = nseq;
  if (n_seg) *n_seg = (int64_t)c->L.nseg;
  if (nd > 0) {  // the ordering the next step starts with
    const Params P = step_params(c, c->step);
    if (!c->keys_valid) {
      launch_keys(false, P, c->rec[c->cur], nd, c->sb.keys[0], c->sb.vals[0], c->st);
      c->keys_valid = true;
    }
    if (++c->stamp > 0xffffu) {
      GP_CUDA(c, cudaMemsetAsync(c->cells, 0, 16 * c->L.nseg, c->st));
      c->stamp = 1;
    }
    c->table_reuse = false;  // this build copies every obstacle into the sequence
    GP_CUDA(c, cudaMemsetAsync(&c->dst->n_act, 0, sizeof(unsigned long long), c->st));
    GP_CUDA(c, cudaMemsetAsync(&c->dst->n_actx, 0, sizeof(uint32_t), c->st));
    launch_group_build(P, static_cast<const uint32_t*>(c->sb.keys[0]), nd, c->L.ngroups,
                       at<uint32_t>(c, c->L.gcnt), at<uint32_t>(c, c->L.gofs),
                       at<uint32_t>(c, c->L.gbsum), at<uint32_t>(c, c->L.gfill), c->sb.vals[1],
                       at<uint32_t>(c, c->L.gkey), at<uint32_t>(c, c->L.gdest), c->rec[c->cur],
                       c->rec[c->cur ^ 1], c->pos4, static_cast<uint32_t*>(c->sb.keys[1]),
                       nullptr, reinterpret_cast<uint8_t*>(c->site_slot), c->cells, c->stamp,
                       c->act, c->dst, c->sms, nullptr, c->st, at<uint32_t>(c, c->L.okey[o]),
                       at<float4>(c, c->L.opos[o]), at<uint32_t>(c, c->L.ogofs[o]), no,
                       at<uint32_t>(c, c->L.msrc));
    GP_CUDA(c, cudaGetLastError());
  }
  if (stamp) *stamp = c->stamp;
  const int64_t m = std::min(nseq, cap), md = std::min(nd, m);
  if (keys_in) {  // the key of every particle in gp_get_particles order: moving, then obstacles
    if (md > 0)
      GP_CUDA(c, cudaMemcpyAsync(keys_in, c->sb.keys[0], 4 * md, cudaMemcpyDeviceToHost, c->st));
    if (m > md)
      GP_CUDA(c, cudaMemcpyAsync(keys_in + md, at<uint32_t>(c, c->L.okey[o]), 4 * (m - md),
                                 cudaMemcpyDeviceToHost, c->st));
  }
  if (m > 0 && keys_sorted)
    GP_CUDA(c, cudaMemcpyAsync(keys_sorted, c->sb.keys[1], 4 * m, cudaMemcpyDeviceToHost, c->st));
  std::vector<uint32_t> ms, perm;
  if (src && m > 0) {
    ms.resize(m);
    perm.resize(nd);
    GP_CUDA(c, cudaMemcpyAsync(ms.data(), at<uint32_t>(c, c->L.msrc), 4 * m,
                               cudaMemcpyDeviceToHost, c->st));
    if (nd > 0)
      GP_CUDA(c, cudaMemcpyAsync(perm.data(), c->sb.vals[1], 4 * nd, cudaMemcpyDeviceToHost,
                                 c->st));
  }
  const int64_t ts = std::min<int64_t>(table_cap, (int64_t)c->L.nseg);
  if (table && ts > 0)
    GP_CUDA(c, cudaMemcpyAsync(table, c->cells, 16 * ts, cudaMemcpyDeviceToHost, c->st));
  GP_CUDA(c, cudaStreamSynchronize(c->st));
  // the gp_get_particles index of every entry of the sequence
  for (int64_t p = 0; src && p < m; ++p) {
    const uint32_t w = ms[p], idx = w & 0x3fffffffu;
    src[p] = (w & 0x80000000u) ? (uint32_t)(nd + idx) : perm[idx];
  }
  return GP_OK;
}

gp_status gp_set_solute_grid(gp_ctx* c, const gp_solute_grid* sg) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (c->batch) return fail(c, GP_ERR_STATE, "a batch of runs takes the nominal liquidus");
  if (!sg || !sg->w) return fail(c, GP_ERR_ARG, "null composition grid");
  if (!std::isfinite(sg->T_m) || !std::isfinite(sg->m_L))
    return fail(c, GP_ERR_ARG, "T_m and m_L must be finite");
  for (int a = 0; a < 3; ++a)
    if (sg->n[a] < 2 || !(sg->spacing[a] > 0))
      return fail(c, GP_ERR_ARG, "grid needs n >= 2 and spacing > 0");
  const size_t nodes = (size_t)sg->n[0] * sg->n[1] * sg->n[2];
  float* dstp = nullptr;
  if ((int64_t)nodes <= c->L.solute_nodes) {
    dstp = at<float>(c, c->L.sgrid);
  } else if (c->own) {
    if (c->wgrid_own_bytes < 4 * nodes) {
      if (c->wgrid_own) cudaFree(c->wgrid_own);
      c->wgrid_own = nullptr;
      c->wgrid_own_bytes = 0;
      GP_CUDA(c, cudaMalloc((void**)&c->wgrid_own, 4 * nodes));
      c->wgrid_own_bytes = 4 * nodes;
    }
    dstp = c->wgrid_own;
  } else {
    return fail(c, GP_ERR_CAPACITY, "composition grid larger than gp_memory.solute_nodes");
  }
  GP_CUDA(c, cudaMemcpyAsync(dstp, sg->w, 4 * nodes,
                             (sg->flags & GP_DEVICE_PTR) ? cudaMemcpyDeviceToDevice
                                                         : cudaMemcpyHostToDevice,
                             c->st));
  GP_CUDA(c, cudaStreamSynchronize(c->st));
  c->P.solute = 1;
  c->P.wgrid = dstp;
  c->P.Tm = (float)sg->T_m;
  c->P.mL = (float)sg->m_L;
  for (int a = 0; a < 3; ++a) {
    c->P.wn[a] = sg->n[a];
    c->P.winv[a] = (float)(1.0 / sg->spacing[a]);
    c->worigin[a] = sg->origin[a];
    c->wvel[a] = sg->frame_vel[a];
  }
  return GP_OK;
}

gp_status gp_nucleation_sites(gp_ctx* c, int64_t n, const double* pos3, const double* dTn,
                              const double* quat4) {
  return gp_run_nucleation_sites(c, 0, n, pos3, dTn, quat4, nullptr);
}

gp_status gp_run_nucleation_sites(gp_ctx* c, int32_t run, int64_t n, const double* pos3,
                                  const double* dTn, const double* quat4,
                                  int32_t* out_first_grain) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (run < 0 || run >= c->L.nruns) return fail(c, GP_ERR_ARG, "no such run");
  if (n < 0 || (n > 0 && (!pos3 || !dTn || !quat4))) return fail(c, GP_ERR_ARG, "bad arguments");
  if (c->n_nuclei + n > c->L.max_nuclei) return fail(c, GP_ERR_CAPACITY, "nucleus capacity");
  if (c->batch && c->n_grains + n > c->L.max_grains)
    return fail(c, GP_ERR_CAPACITY, "grain capacity");
  for (int64_t i = 0; i < n; ++i) {
    const double* q = quat4 + 4 * i;
    const double nq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (!(nq > 0) || !std::isfinite(nq)) return fail(c, GP_ERR_ARG, "quaternion is zero or not finite");
    if (!std::isfinite(dTn[i])) return fail(c, GP_ERR_ARG, "nucleation undercooling not finite");
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(pos3[3 * i + a])) return fail(c, GP_ERR_ARG, "site position not finite");
  }
  if (out_first_grain) *out_first_grain = c->batch ? (int32_t)c->n_grains : -1;
  if (n == 0) return GP_OK;
  std::vector<float4> P(n), G(4 * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    P[i] = make_float4((float)pos3[3 * i], (float)pos3[3 * i + 1], (float)pos3[3 * i + 2],
                       (float)dTn[i]);
    grain_entry(pos3 + 3 * i, quat4 + 4 * i, c->h, run, &G[4 * i]);
  }
  GP_CUDA(c, cudaMemcpyAsync(c->npos + c->n_nuclei, P.data(), sizeof(float4) * n,
                             cudaMemcpyHostToDevice, c->st));
  if (!c->batch) {
    // grain ids are given at activation, in registration order
    GP_CUDA(c, cudaMemcpyAsync(c->ngrain + 4 * (size_t)c->n_nuclei, G.data(),
                               sizeof(float4) * G.size(), cudaMemcpyHostToDevice, c->st));
    GP_CUDA(c, cudaStreamSynchronize(c->st));
    c->n_nuclei += (int)n;
    return GP_OK;
  }
  // batch: every site reserves its grain id now, so that runs never wait on one
  // another's activations
  std::vector<int2> M(n);
  for (int64_t i = 0; i < n; ++i) M[i] = make_int2((int)(c->n_grains + i), run);
  GP_CUDA(c, cudaMemcpyAsync(c->gtab + 4 * c->n_grains, G.data(), sizeof(float4) * G.size(),
                             cudaMemcpyHostToDevice, c->st));
  GP_CUDA(c, cudaMemcpyAsync(c->nmeta + c->n_nuclei, M.data(), sizeof(int2) * n,
                             cudaMemcpyHostToDevice, c->st));
  c->n_nuclei += (int)n;
  c->n_grains += n;
  drop_graphs(c);  // captured steps launch the nucleation kernels for n_nuclei sites
  return push_counts(c);
}

}  // extern "C"

namespace {

// One step of a batch, every launch sized on the device (counts in DevStats), so
// that a sequence of steps can be captured in a CUDA graph: run constants, sort,
// build, advance, emit, nucleation, counters.
void batch_step_launches(gp_ctx* c) {
  const Params& P = c->P;
  const int64_t cap = c->L.cap;
  const StepArgs S{};  // parity and stamp are read on the device
  cudaStream_t st = c->st;
  const double units = (double)c->n_live;  // timing units (exact when stepped eagerly)
  launch_run_step(c->runs, c->rtherm, c->L.nruns, c->dst, c->dt, st);
  cudaMemsetAsync(&c->dst->n_out, 0, sizeof(unsigned long long), st);
  cudaMemsetAsync(&c->dst->n_frozen, 0, sizeof(unsigned long long), st);
  cudaMemsetAsync(&c->dst->n_act, 0, sizeof(unsigned long long), st);
  const int w = radix_sort<uint64_t>(c->sb, cap, c->L.nbits, st);
  int4* sorted = c->rec[c->cur ^ 1];
  c->prof.begin(K_BUILD);
  launch_build(P, static_cast<const uint64_t*>(c->sb.keys[w]), c->sb.vals[w], c->rec[c->cur], sorted,
               c->pos4, c->cells, cap, c->L.key_end, c->act, c->dst, st);
  c->prof.end(K_BUILD, units);
  c->prof.begin(K_ADVANCE);
  launch_advance(true, P, S, sorted, c->pos4, c->sb.keys[w], c->cells, 0, cap, c->act, c->C,
                 c->site_slot, c->dst, st);
  c->prof.end(K_ADVANCE, units);
  c->prof.begin(K_EMIT);
  launch_emit(true, P, S, sorted, c->site_slot, cap, c->rec[c->cur], c->sb.keys[0],
              c->sb.vals[0], cap, c->C, c->R, nullptr, c->dst, st);
  c->prof.end(K_EMIT, units, 2);  // k_emit, k_emit_check
  if (c->n_nuclei > (int64_t)c->hst->nucleated || (c->graph_steps > 0 && c->n_nuclei > 0)) {
    launch_link_reached(true, P, c->R, &c->dst->linked, c->sms, st);
    c->prof.begin(K_NUCLEATE);
    launch_nucleate_batch(P, StepArgs{}, c->npos, c->nmeta, c->nstate, c->n_nuclei,
                          c->rec[c->cur], static_cast<uint64_t*>(c->sb.keys[0]), c->sb.vals[0],
                          cap, c->C, c->R, c->dst, c->sms, st);
    c->prof.end(K_NUCLEATE, 1.0, 2);  // k_nuc_test, k_nuc_activate
  }
  launch_finalize(c->dst, cap, true, st);
}

// the instantiated graph of k batch steps (captured on first use)
gp_status graph_for(gp_ctx* c, int k, cudaGraphExec_t* out) {
  auto it = c->graphs.find(k);
  if (it != c->graphs.end()) {
    *out = it->second;
    return GP_OK;
  }
  const bool prof = c->prof.on;
  c->prof.on = false;
  GP_CUDA(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < k; ++i) batch_step_launches(c);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->st, &g);
  c->prof.on = prof;
  GP_CUDA(c, e);
  cudaGraphExec_t ge = nullptr;
  const cudaError_t e2 = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  GP_CUDA(c, e2);
  c->graphs[k] = ge;
  *out = ge;
  return GP_OK;
}

gp_status step_batch(gp_ctx* c, int32_t nsteps) {
  for (int r = 0; r < c->L.nruns; ++r)
    if (!c->thermal_set[r]) return fail(c, GP_ERR_STATE, "a run has no thermal field");
  if (c->graph_steps > 0 && c->st == nullptr)
    return fail(c, GP_ERR_STATE, "CUDA graphs need a non-default stream");
  if (c->n_live > 0 && !c->keys_valid) {
    c->prof.begin(K_KEYS);
    launch_keys(true, c->P, c->rec[c->cur], c->n_live, c->sb.keys[0], c->sb.vals[0], c->st);
    c->prof.end(K_KEYS, (double)c->n_live);
  }
  c->keys_valid = true;
  int64_t done = 0;
  while (done < nsteps) {
    const int k = c->graph_steps > 0 ? (int)std::min<int64_t>(c->graph_steps, nsteps - done) : 1;
    if (c->stamp + (uint32_t)k > 0xffffu) {  // stamps are 16 bits in the cell table
      GP_CUDA(c, cudaMemsetAsync(c->cells, 0, 16 * c->L.nseg, c->st));
      c->hst->stamp = 1;
      GP_CUDA(c, cudaMemcpyAsync(&c->dst->stamp, &c->hst->stamp, sizeof(unsigned long long),
                                 cudaMemcpyHostToDevice, c->st));
      c->stamp = 1;
    }
    if (c->graph_steps > 0) {
      cudaGraphExec_t ge = nullptr;
      gp_status s = graph_for(c, k, &ge);
      if (s) return s;
      GP_CUDA(c, cudaGraphLaunch(ge, c->st));
    } else {
      batch_step_launches(c);
    }
    GP_CUDA(c, cudaGetLastError());
    c->step += k;
    c->stamp += (uint32_t)k;
    done += k;
    gp_status s = sync_stats(c);
    if (s) return s;
  }
  return GP_OK;
}

}  // namespace

extern "C" {

gp_status gp_step(gp_ctx* c, int32_t nsteps) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (nsteps < 0) return fail(c, GP_ERR_ARG, "nsteps < 0");
  if (c->batch) return step_batch(c, nsteps);
  if (c->thermal == 0 && c->n_live > 0) return fail(c, GP_ERR_STATE, "no thermal field set");
  const bool batch = false;
  for (int it = 0; it < nsteps; ++it) {
    const StepArgs S = step_args(c, c->step);
    const Params P = step_params(c, c->step);
    if (c->melting) {
      // melting walk-back at t_n (Sec. 2.1.3); the compacted store lands in the other
      // record buffer, which becomes the store
      launch_melt(P, S, c->R, c->C, reinterpret_cast<unsigned long long*>(c->pos4),
                  2 * c->L.cap, c->gflags, (int)c->n_grains, c->rec[c->cur], c->rec[c->cur ^ 1],
                  c->n_live, c->L.cap, c->dst, c->sms, c->st);
      GP_CUDA(c, cudaGetLastError());
      c->cur ^= 1;
      c->keys_valid = false;
      s = sync_stats(c);
      if (s) return s;
    }
    const int64_t n = c->n_live;
    const bool obs = obs_usable(c);
    const bool rec = c->tape_on && c->tape_pos < c->L.tape_steps;
    const size_t tq = (size_t)c->tape_pos, tcap = (size_t)c->L.cap;
    int32_t* tpar = rec ? at<int32_t>(c, c->L.tape_par) + tq * tcap : nullptr;
    uint32_t* tsrc = rec ? at<uint32_t>(c, c->L.tape_svals) : nullptr;
    if (rec) GP_CUDA(c, cudaMemsetAsync(tpar, 0xff, 4 * tcap, c->st));
    if (rec && tq % (size_t)c->L.tape_every == 0 && n > 0)  // checkpoint: the store now
      GP_CUDA(c, cudaMemcpyAsync(at<int4>(c, c->L.tape_ckpt) + (tq / c->L.tape_every) * tcap,
                                 c->rec[c->cur], 16 * n, cudaMemcpyDeviceToDevice, c->st));
    GP_CUDA(c, cudaMemsetAsync(&c->dst->n_out, 0, sizeof(unsigned long long), c->st));
    GP_CUDA(c, cudaMemsetAsync(&c->dst->n_frozen, 0, sizeof(unsigned long long), c->st));
    if (n > 0) {
      if (!c->keys_valid) {
        c->prof.begin(K_KEYS);
        launch_keys(batch, P, c->rec[c->cur], n, c->sb.keys[0], c->sb.vals[0], c->st);
        c->prof.end(K_KEYS, (double)n);
        c->keys_valid = true;
      }
      if (++c->stamp > 0xffffu) {
        GP_CUDA(c, cudaMemsetAsync(c->cells, 0, 16 * c->L.nseg, c->st));
        c->stamp = 1;
        c->table_reuse = false;
      }
      if (++c->nbuild == 0xffffffffu) {  // build tags start again
        GP_CUDA(c, cudaMemsetAsync(at<uint32_t>(c, c->L.rbuild), 0, 4 * (size_t)c->L.ngroups,
                                   c->st));
        c->nbuild = 2;
        c->table_reuse = false;
      }
      int4* sorted = c->rec[c->cur ^ 1];  // the records in grouped order
      GP_CUDA(c, cudaMemsetAsync(&c->dst->n_act, 0, sizeof(unsigned long long), c->st));
      GP_CUDA(c, cudaMemsetAsync(&c->dst->n_actx, 0, sizeof(uint32_t), c->st));
      // records grouped by cell tile (in place of the radix sort): the emit's keys in
      // keys[0], the grouped identities in vals[1]; the cell-ordered sequence of the moving
      // records and the obstacles (positions, keys in keys[1], sources, cell table); the
      // store index of each grouped record for the tape; the state bytes in the
      // claim-slot hand-off (overwritten by the advance before the emit reads it)
      const int o = c->ocur;
      const int64_t nseq = n + (obs ? c->n_obs : 0);
      uint32_t* skeys = static_cast<uint32_t*>(c->sb.keys[1]);
      // obstacle flush: the obstacles and the FROZEN records (hst->n_frozen of them, as the
      // last emit counted) of the cell-ordered sequence become the new obstacle store once
      // carrying the FROZEN records from step to step has cost about as much as rewriting
      // the store, counted as kObsCarry record-steps per obstacle; the first FROZEN records
      // are flushed at once
      bool flush = false;
      if (obs) {
        const double f = (double)c->hst->n_frozen;
        c->obs_carry += f;
        flush = f > 0 && (c->obs_mode == 2 || kObsCarry * c->obs_carry >= (double)c->n_obs + f);
      }
      uint32_t* msrc = flush ? at<uint32_t>(c, c->L.msrc) : nullptr;  // the flush's input
      // index of the current obstacle store in pos4 and skeys (they hold the sequence, then
      // the two copies of the store); groups without moving records are read there in place
      // (0: copy every obstacle, when the three parts exceed 32-bit indices)
      const uint64_t span = 3 * (uint64_t)c->L.cap;
      const uint32_t obase =
          obs && span < (1ull << 32) ? (uint32_t)((uint64_t)c->L.cap * (1 + o)) : 0u;
      launch_group_build(P, static_cast<const uint32_t*>(c->sb.keys[0]), n, c->L.ngroups,
                         at<uint32_t>(c, c->L.gcnt), at<uint32_t>(c, c->L.gofs),
                         at<uint32_t>(c, c->L.gbsum), at<uint32_t>(c, c->L.gfill), c->sb.vals[1],
                         at<uint32_t>(c, c->L.gkey), at<uint32_t>(c, c->L.gdest), c->rec[c->cur],
                         sorted, c->pos4, skeys, tsrc,
                         reinterpret_cast<uint8_t*>(c->site_slot), c->cells, c->stamp, c->act,
                         c->dst, c->sms, &c->prof, c->st, at<uint32_t>(c, c->L.okey[o]),
                         at<float4>(c, c->L.opos[o]), at<uint32_t>(c, c->L.ogofs[o]),
                         obs ? c->n_obs : 0, msrc, obase, at<uint32_t>(c, c->L.rbuild),
                         c->nbuild, c->table_reuse && obase != 0u ? 1 : 0);
      GP_CUDA(c, cudaGetLastError());
      // a flush replaces the store that the entries of resident groups point into
      c->table_reuse = obase != 0u && !flush;
      if (flush) {
        c->prof.begin(K_OBS);
        launch_obs_flush(msrc, skeys, c->pos4, nseq, at<uint32_t>(c, c->L.otcnt),
                         at<int4>(c, c->L.orec[o]), sorted, at<uint32_t>(c, c->L.okey[o ^ 1]),
                         at<float4>(c, c->L.opos[o ^ 1]), at<int4>(c, c->L.orec[o ^ 1]),
                         c->L.ngroups, at<uint32_t>(c, c->L.ogofs[o ^ 1]), c->dst, c->st,
                         (int64_t)c->L.cap * (1 + o));
        GP_CUDA(c, cudaMemcpyAsync(&c->hst->obs_new, &c->dst->obs_new, sizeof(unsigned long long),
                                   cudaMemcpyDeviceToHost, c->st));
        GP_CUDA(c, cudaStreamSynchronize(c->st));
        GP_CUDA(c, cudaGetLastError());
        c->ocur ^= 1;
        c->n_obs = (int64_t)c->hst->obs_new;
        c->obs_carry = 0;
        c->prof.end(K_OBS, (double)c->n_obs, 4);
      }
      c->prof.begin(K_ADVANCE);
      // the table's ranges lie in the sequence or, read in place, in the obstacle store
      launch_advance(batch, P, S, sorted, c->pos4, skeys, c->cells, c->stamp,
                     obase ? (int64_t)span : nseq, c->act, c->C, c->site_slot, c->dst, c->st, n,
                     at<uint32_t>(c, c->L.gdest));
      // units: the ACTIVE particles entering the step (live minus frozen after the last step)
      c->prof.end(K_ADVANCE, (double)(n - std::min<int64_t>(n, (int64_t)c->hst->n_frozen)));
      if (rec) launch_tape_state(sorted, tsrc, n, at<uint8_t>(c, c->L.tape_post) + tq * tcap, c->st);
      c->prof.begin(K_EMIT);
      launch_emit(batch, P, S, sorted, c->site_slot, n, c->rec[c->cur], c->sb.keys[0],
                  c->sb.vals[0], c->L.cap - c->n_obs, c->C, c->R, tpar, c->dst, c->st);
      c->prof.end(K_EMIT, (double)n, 2);  // k_emit, k_emit_check
    }
    // the dynamic store holds what the particle capacity leaves beside the obstacles
    const int64_t dcap = c->L.cap - c->n_obs;
    // pending sites: registered minus activated (re-nucleations of dormant seeds
    // count as nucleations too, so they are subtracted back)
    const int64_t pending =
        c->n_nuclei - ((int64_t)c->hst->nucleated - (int64_t)c->hst->renucleated);
    const int64_t dormant = (int64_t)c->hst->n_dormant;
    const StepArgs S1 = step_args(c, c->step + 1);
    if (pending > 0 || dormant > 0)
      launch_link_reached(batch, P, c->R, &c->dst->linked, c->sms, c->st);
    if (dormant > 0)  // before any activation of the step
      launch_dormant_test(P, S1, c->R, c->gdtn, c->gflags, (int)c->n_grains, c->st);
    if (pending > 0) {
      c->prof.begin(K_NUCLEATE);
      launch_nucleate(P, S1, c->npos, c->ngrain, c->nstate, c->n_nuclei, c->gtab,
                      c->L.max_grains, c->rec[c->cur], static_cast<uint32_t*>(c->sb.keys[0]),
                      c->sb.vals[0], dcap, c->C, c->R, c->dst, c->gdtn, c->st);
      c->prof.end(K_NUCLEATE, 1.0);
    } else {
      c->prof.begin(K_FINALIZE);
      launch_finalize(c->dst, dcap, false, c->st);
      c->prof.end(K_FINALIZE, 1.0);
    }
    if (dormant > 0)
      launch_renucleate(P, c->gflags, (int)c->n_grains, c->rec[c->cur],
                        static_cast<uint32_t*>(c->sb.keys[0]), c->sb.vals[0], dcap, c->C,
                        c->R, c->dst, c->st);
    if (rec)
      launch_tape_out(tpar, tsrc, c->rec[c->cur], at<uint8_t>(c, c->L.tape_code) + tq * tcap,
                      c->L.cap, c->dst, c->sms, c->st);
    GP_CUDA(c, cudaGetLastError());
    const int64_t stepped = c->step;
    ++c->step;
    c->keys_valid = true;
    s = sync_stats(c);
    if (s) return s;
    if (rec) {
      c->tape_n.push_back(n);
      c->tape_m.push_back(c->n_live);
      c->tape_t.push_back(stepped);
      ++c->tape_pos;
    }
  }
  return GP_OK;
}

gp_status gp_tape_begin(gp_ctx* c) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (c->batch) return fail(c, GP_ERR_STATE, "the adjoint is for single-run contexts");
  if (c->melting) return fail(c, GP_ERR_STATE, "the adjoint holds no melting events");
  if (c->periodic) return fail(c, GP_ERR_STATE, "the adjoint takes non-periodic domains");
  if (c->P.solute) return fail(c, GP_ERR_STATE, "the adjoint takes the nominal liquidus");
  if (c->L.tape_steps <= 0) return fail(c, GP_ERR_STATE, "no tape (gp_memory.tape_steps = 0)");
  if (c->thermal != 1) return fail(c, GP_ERR_STATE, "the adjoint needs an analytic field");
  if (c->L.tape_every > 1 &&
      c->n_nuclei - ((int64_t)c->hst->nucleated - (int64_t)c->hst->renucleated) > 0)
    return fail(c, GP_ERR_STATE,
                "a tape with checkpoints replays its steps and cannot replay nucleation: "
                "no pending nucleation sites (or tape_checkpoint_every = 1)");
  s = obs_return(c);  // the tape follows every particle through the dynamic store
  if (s) return s;
  c->tape_on = true;
  c->tape_pos = 0;
  c->tape_n.clear();
  c->tape_m.clear();
  c->tape_t.clear();
  return GP_OK;
}

gp_status gp_adjoint(gp_ctx* c, const float* seed, int64_t n, int32_t flags, double grad[8]) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (!grad || (n > 0 && !seed)) return fail(c, GP_ERR_ARG, "null argument");
  if (!c->tape_on || c->tape_pos == 0) return fail(c, GP_ERR_STATE, "nothing taped");
  if (c->thermal != 1) return fail(c, GP_ERR_STATE, "the adjoint needs an analytic field");
  if (c->tape_t.back() != c->step - 1)
    return fail(c, GP_ERR_STATE, "the taped steps do not end at the current step");
  if (n != c->n_live) return fail(c, GP_ERR_ARG, "seed length differs from the live particles");
  const size_t tcap = (size_t)c->L.cap;
  float* lam_u = static_cast<float*>(c->sb.keys[1]);
  float* lam_s = reinterpret_cast<float*>(c->sb.vals[1]);
  double* gdev = at<double>(c, c->L.tape_grad);
  if (n > 0)
    GP_CUDA(c, cudaMemcpyAsync(lam_u, seed, 4 * n,
                               (flags & GP_DEVICE_PTR) ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyHostToDevice,
                               c->st));
  GP_CUDA(c, cudaMemsetAsync(gdev, 0, 8 * 8, c->st));
  const int64_t every = c->L.tape_every;
  const int4* ckpt = at<int4>(c, c->L.tape_ckpt);
  int4* replay[2] = {at<int4>(c, c->L.tape_replay), at<int4>(c, c->L.tape_replay) + tcap};
  auto post = [&](int64_t q) { return at<uint8_t>(c, c->L.tape_post) + q * tcap; };
  auto par = [&](int64_t q) { return at<int32_t>(c, c->L.tape_par) + q * tcap; };
  auto code = [&](int64_t q) { return at<uint8_t>(c, c->L.tape_code) + q * tcap; };
  for (int64_t q = c->tape_pos - 1; q >= 0; --q) {
    const int64_t nn = c->tape_n[q], m = c->tape_m[q];
    // the store at step q: its checkpoint, replayed forward over the steps since
    const int64_t q0 = (q / every) * every;
    const int4* R = ckpt + (size_t)(q / every) * tcap;
    for (int64_t j = q0; j < q; ++j) {
      int4* out = replay[(j - q0) & 1];
      launch_adj_replay(step_params(c, c->tape_t[j]), step_args(c, c->tape_t[j]), R, post(j),
                        par(j), code(j), c->tape_m[j], out, c->st);
      R = out;
    }
    if (nn > 0) GP_CUDA(c, cudaMemsetAsync(lam_s, 0, 4 * nn, c->st));
    const StepArgs S = step_args(c, c->tape_t[q]);
    const float t = (float)((double)c->tape_t[q] * c->dt);
    launch_adj_step(step_params(c, c->tape_t[q]), S, t, R, post(q), par(q), lam_u, m, lam_s,
                    gdev, c->st);
    std::swap(lam_u, lam_s);  // the adjoint of step q, by store index
  }
  GP_CUDA(c, cudaGetLastError());
  GP_CUDA(c, cudaMemcpyAsync(grad, gdev, 8 * 8, cudaMemcpyDeviceToHost, c->st));
  GP_CUDA(c, cudaStreamSynchronize(c->st));
  return GP_OK;
}

gp_status gp_stats(gp_ctx* c, gp_stats_t* o) {
  if (!c || !o) return GP_ERR_ARG;
  cudaSetDevice(c->device);
  std::memset(o, 0, sizeof(*o));
  if (cudaMemcpyAsync(c->hst, c->dst, sizeof(DevStats), cudaMemcpyDeviceToHost, c->st) ==
      cudaSuccess)
    cudaStreamSynchronize(c->st);
  const DevStats& d = *c->hst;
  o->step = c->step;
  o->n_live = (int64_t)d.n_live + c->n_obs;      // dynamic store + obstacle store
  o->n_frozen = (int64_t)d.n_frozen + c->n_obs;
  o->n_active = o->n_live - o->n_frozen;
  o->n_grains = (int64_t)d.n_grains;
  o->n_reached = (int64_t)std::min<unsigned long long>(d.reached, (unsigned long long)c->L.rcap);
  o->particle_steps = (int64_t)d.particle_steps;
  o->n_frozen_new = (int64_t)d.frozen_new;
  o->n_spawned = (int64_t)d.spawned;
  o->n_claims_lost = (int64_t)d.claims_lost;
  o->n_clipped = (int64_t)d.clipped;
  o->n_clamped = (int64_t)d.clamped;
  o->n_nucleated = (int64_t)d.nucleated;
  o->n_claim_blocks = (int64_t)d.claim_used;
  o->error_flags = (int64_t)d.err;
  o->n_melted = (int64_t)d.melted;
  o->n_walkback = (int64_t)d.walkback;
  return GP_OK;
}

gp_status gp_get_particles(gp_ctx* c, int64_t cap, int32_t* grain, int32_t* site3, int8_t* dir,
                           float* ell, uint8_t* state, float* x3, int64_t* n_out) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (cap < 0) return fail(c, GP_ERR_ARG, "cap < 0");
  // the dynamic store, then the obstacle store
  const int64_t nd = c->n_live, n = nd + c->n_obs;
  if (n_out) *n_out = n;
  const int64_t m = std::min(n, cap), md = std::min(nd, m), mo = m - md;
  if (m == 0) return GP_OK;
  std::vector<int4> recs(m);
  const int4* orec = at<int4>(c, c->L.orec[c->ocur]);
  if (md)
    GP_CUDA(c, cudaMemcpyAsync(recs.data(), c->rec[c->cur], sizeof(int4) * md,
                               cudaMemcpyDeviceToHost, c->st));
  if (mo)
    GP_CUDA(c, cudaMemcpyAsync(recs.data() + md, orec, sizeof(int4) * mo, cudaMemcpyDeviceToHost,
                               c->st));
  if (x3) {
    float* dx = reinterpret_cast<float*>(c->pos4);  // 16 bytes per particle of capacity
    launch_positions(c->P, c->rec[c->cur], md, dx, c->st);
    launch_positions(c->P, orec, mo, dx + 3 * md, c->st);
    GP_CUDA(c, cudaMemcpyAsync(x3, dx, sizeof(float) * 3 * m, cudaMemcpyDeviceToHost, c->st));
  }
  GP_CUDA(c, cudaStreamSynchronize(c->st));
  for (int64_t i = 0; i < m; ++i) {
    Rec r = rec_unpack(recs[i]);
    if (grain) grain[i] = r.grain;
    if (site3) {
      site3[3 * i] = r.sx;
      site3[3 * i + 1] = r.sy;
      site3[3 * i + 2] = r.sz;
    }
    if (dir) dir[i] = (int8_t)r.dir;
    if (ell) ell[i] = r.ell;
    if (state) state[i] = (uint8_t)r.state;
  }
  return GP_OK;
}

gp_status gp_load_particles(gp_ctx* c, int64_t n, const int32_t* grain, const int32_t* site3,
                            const int8_t* dir, const float* ell, const uint8_t* state,
                            int64_t step) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (n < 0 || n > c->L.cap) return fail(c, GP_ERR_CAPACITY, "n exceeds capacity");
  if (n > 0 && (!grain || !site3 || !dir || !ell || !state)) return fail(c, GP_ERR_ARG, "null array");
  std::vector<int4> recs(n);
  for (int64_t i = 0; i < n; ++i) {
    if (grain[i] < 0 || grain[i] >= c->n_grains || dir[i] < 0 || dir[i] > 5 || state[i] > 1 ||
        !(ell[i] >= 0.f && ell[i] < 1.f))
      return fail(c, GP_ERR_ARG, "invalid particle");
    for (int a = 0; a < 3; ++a)
      if (site3[3 * i + a] < -kSiteMax || site3[3 * i + a] > kSiteMax)
        return fail(c, GP_ERR_ARG, "site out of range");
    Rec r{};
    r.grain = grain[i];
    r.sx = site3[3 * i];
    r.sy = site3[3 * i + 1];
    r.sz = site3[3 * i + 2];
    r.dir = dir[i];
    r.state = state[i];
    r.ell = ell[i];
    recs[i] = rec_pack(r);
  }
  if (n > 0)
    GP_CUDA(c, cudaMemcpyAsync(c->rec[c->cur], recs.data(), sizeof(int4) * n,
                               cudaMemcpyHostToDevice, c->st));
  c->n_live = n;
  c->step = step;
  c->keys_valid = false;
  int64_t nfz = 0;
  for (int64_t i = 0; i < n; ++i) nfz += state[i] == ST_FROZEN;
  c->hst->n_frozen = (unsigned long long)nfz;
  s = obs_reset(c);  // every particle is in the dynamic store now
  if (s) return s;
  return push_counts(c);
}

gp_status gp_add_sites(gp_ctx* c, int64_t n, const int32_t* grain, const int32_t* site3,
                       int32_t reached, int32_t claimed) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (n < 0 || (n > 0 && (!grain || !site3))) return fail(c, GP_ERR_ARG, "bad arguments");
  const int64_t chunk = c->L.cap;  // int4 entries that fit in the position buffer
  std::vector<int4> v;
  for (int64_t b = 0; b < n; b += chunk) {
    const int64_t m = std::min(chunk, n - b);
    v.resize(m);
    for (int64_t i = 0; i < m; ++i) {
      const int64_t j = b + i;
      if (grain[j] < 0 || grain[j] >= c->n_grains) return fail(c, GP_ERR_ARG, "unknown grain");
      v[i] = make_int4(grain[j], site3[3 * j], site3[3 * j + 1], site3[3 * j + 2]);
    }
    int4* stg = reinterpret_cast<int4*>(c->pos4);
    GP_CUDA(c, cudaMemcpyAsync(stg, v.data(), sizeof(int4) * m, cudaMemcpyHostToDevice, c->st));
    launch_mark_sites(c->P, stg, m, reached ? 1 : 0, claimed ? 1 : 0, c->C, c->R, c->st);
    GP_CUDA(c, cudaStreamSynchronize(c->st));
  }
  GP_CUDA(c, cudaGetLastError());
  return sync_stats(c);
}

gp_status gp_get_reached(gp_ctx* c, int64_t cap, int32_t* grain, int32_t* site3, int64_t* n_out) {
  gp_status s = check_ctx(c);
  if (s) return s;
  s = sync_stats(c);
  if (s) return s;
  const int64_t n = (int64_t)std::min<unsigned long long>(c->hst->reached, c->L.rcap);
  std::vector<unsigned long long> k(n);
  if (n > 0) GP_CUDA(c, cudaMemcpy(k.data(), c->R.key, 8 * n, cudaMemcpyDeviceToHost));
  k.erase(std::remove(k.begin(), k.end(), kDeadSite), k.end());  // melted sites
  if (n_out) *n_out = (int64_t)k.size();
  const int64_t m = std::min((int64_t)k.size(), cap);
  for (int64_t i = 0; i < m; ++i) {
    int g, x, y, z;
    unpack_site(k[i], g, x, y, z);
    if (grain) grain[i] = g;
    if (site3) {
      site3[3 * i] = x;
      site3[3 * i + 1] = y;
      site3[3 * i + 2] = z;
    }
  }
  return GP_OK;
}

// ---------------------------------------------------------------------------------
// checkpoints of a single-run context
// ---------------------------------------------------------------------------------
namespace {

constexpr char kCkptMagic[8] = {'G', 'P', 'C', 'K', 'P', 'T', '\0', '\1'};
constexpr uint32_t kCkptVersion = 1;

// The fixed part of a checkpoint.  The sections follow it, each on a 16-byte boundary
// (CkptSections); multi-byte values are in the byte order of the machine that wrote it.
struct CkptHeader {
  char magic[8];
  uint32_t version, header_bytes;
  uint64_t total_bytes;
  uint64_t checksum;  // 64-bit FNV-1a of the whole checkpoint with this field zero
  gp_domain dom;
  double h, dt;
  gp_growth_law law;
  int64_t step, n_rec, n_grains, n_nuclei, n_reached, n_blocks;
  int32_t thermal, periodic, melting, obs_mode;
  double T0, Tdot;          // analytic field (thermal == 1) as the context holds it
  float G[3], xref[3];
  DevStats stats;           // device counters between steps
};

struct CkptSections {
  size_t rec, gtab, gflags, gdtn, npos, ngrain, nstate, rkey, bkey, bdata, total;
};

size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// byte offsets of the sections for the counts in h; false for a count out of range
bool ckpt_sections(const CkptHeader& h, CkptSections* o) {
  const int64_t lim = (int64_t)1 << 40;
  const int64_t cnt[5] = {h.n_rec, h.n_grains, h.n_nuclei, h.n_reached, h.n_blocks};
  for (int64_t v : cnt)
    if (v < 0 || v > lim) return false;
  size_t p = align16(sizeof(CkptHeader));
  auto take = [&](size_t bytes) {
    const size_t q = p;
    p = align16(p + bytes);
    return q;
  };
  o->rec = take(16 * (size_t)h.n_rec);            // particle records (int4)
  o->gtab = take(64 * (size_t)h.n_grains);        // grain frames (4 float4)
  o->gflags = take(4 * (size_t)h.n_grains);       // melting flags (four bytes per grain)
  o->gdtn = take(4 * (size_t)h.n_grains);         // nucleation undercooling of each seed
  o->npos = take(16 * (size_t)h.n_nuclei);        // nucleation sites (position, dTn)
  o->ngrain = take(64 * (size_t)h.n_nuclei);      // frames of the grains they nucleate
  o->nstate = take(4 * (size_t)h.n_nuclei);       // their activation state
  o->rkey = take(8 * (size_t)h.n_reached);        // reached-site list (melted entries too)
  o->bkey = take(8 * (size_t)h.n_blocks);         // claim block keys, by pool slot
  o->bdata = take(4 * (size_t)kBrickWords * (size_t)h.n_blocks);  // their claim bytes
  o->total = p;
  return true;
}

uint64_t fnv1a(const unsigned char* p, size_t n, uint64_t h) {
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

// 64-bit FNV-1a of the checkpoint with eight zero bytes in place of the checksum field
uint64_t ckpt_checksum(const unsigned char* b, size_t bytes) {
  const size_t off = offsetof(CkptHeader, checksum);
  const unsigned char zero[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  uint64_t h = fnv1a(b, off, 14695981039346656037ull);
  h = fnv1a(zero, 8, h);
  return fnv1a(b + off + 8, bytes - off - 8, h);
}

// why buf is not a checkpoint of this format (nullptr if it is one)
const char* ckpt_invalid(const void* buf, size_t bytes, CkptHeader* h, CkptSections* sec) {
  if (!buf) return "null checkpoint";
  if (bytes < sizeof(CkptHeader)) return "checkpoint truncated";
  std::memcpy(h, buf, sizeof(CkptHeader));
  if (std::memcmp(h->magic, kCkptMagic, sizeof kCkptMagic) != 0) return "not a checkpoint";
  if (h->version != kCkptVersion || h->header_bytes != (uint32_t)sizeof(CkptHeader))
    return "checkpoint of another format version";
  if (h->total_bytes != (uint64_t)bytes) return "checkpoint truncated or padded";
  if (!ckpt_sections(*h, sec) || sec->total != bytes) return "checkpoint sections do not add up";
  if (ckpt_checksum(static_cast<const unsigned char*>(buf), bytes) != h->checksum)
    return "checkpoint checksum mismatch (corrupt)";
  return nullptr;
}

bool same_law(const gp_growth_law& a, const gp_growth_law& b) {
  if (a.nterms != b.nterms || a.T_liquidus != b.T_liquidus) return false;
  for (int i = 0; i < a.nterms && i < 2; ++i)
    if (a.a[i] != b.a[i] || a.b[i] != b.b[i]) return false;
  return true;
}

}  // namespace

gp_status gp_checkpoint_check(const void* buf, size_t bytes, int64_t* step,
                              int64_t* n_particles) {
  CkptHeader h;
  CkptSections sec;
  if (ckpt_invalid(buf, bytes, &h, &sec)) return GP_ERR_ARG;
  if (step) *step = h.step;
  if (n_particles) *n_particles = h.n_rec;
  return GP_OK;
}

gp_status gp_save(gp_ctx* c, void* buf, size_t cap, size_t* bytes) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (c->batch) return fail(c, GP_ERR_STATE, "checkpoints are of single-run contexts");
  if (c->tape_on) return fail(c, GP_ERR_STATE, "the adjoint tape is recording");
  if (!bytes) return fail(c, GP_ERR_ARG, "null size");
  s = sync_stats(c);
  if (s) return s;
  const DevStats d = *c->hst;
  CkptHeader h;
  std::memset(&h, 0, sizeof h);
  std::memcpy(h.magic, kCkptMagic, sizeof kCkptMagic);
  h.version = kCkptVersion;
  h.header_bytes = (uint32_t)sizeof(CkptHeader);
  h.dom = c->dom[0];
  h.h = c->h;
  h.dt = c->dt;
  h.law = c->law;
  h.step = c->step;
  h.n_rec = c->n_live + c->n_obs;
  h.n_grains = c->n_grains;
  h.n_nuclei = c->n_nuclei;
  h.n_reached = (int64_t)std::min<unsigned long long>(d.reached, (unsigned long long)c->L.rcap);
  h.n_blocks = (int64_t)d.claim_used;
  if (h.n_blocks > c->L.blocks) return fail(c, GP_ERR_STATE, "claim pool overflowed");
  h.thermal = c->thermal;
  h.periodic = c->periodic;
  h.melting = c->melting ? 1 : 0;
  h.obs_mode = c->obs_mode;
  if (c->thermal == 1) {
    h.T0 = c->T0[0];
    h.Tdot = c->Tdot[0];
    for (int a = 0; a < 3; ++a) {
      h.G[a] = c->P.geo.G[a];
      h.xref[a] = c->P.geo.xref[a];
    }
  }
  h.stats = d;
  CkptSections sec;
  ckpt_sections(h, &sec);
  h.total_bytes = sec.total;
  *bytes = sec.total;
  if (!buf) return GP_OK;
  if (cap < sec.total) return fail(c, GP_ERR_CAPACITY, "checkpoint buffer too small");
  unsigned char* b = static_cast<unsigned char*>(buf);
  std::memset(b, 0, sec.total);  // the padding between sections
  auto d2h = [&](size_t off, const void* src, size_t n) -> gp_status {
    if (n) GP_CUDA(c, cudaMemcpyAsync(b + off, src, n, cudaMemcpyDeviceToHost, c->st));
    return GP_OK;
  };
  const int64_t nd = c->n_live;
  gp_status e = GP_OK;
  // the dynamic store, then the obstacle store
  e = e ? e : d2h(sec.rec, c->rec[c->cur], 16 * (size_t)nd);
  e = e ? e : d2h(sec.rec + 16 * (size_t)nd, at<int4>(c, c->L.orec[c->ocur]), 16 * (size_t)c->n_obs);
  e = e ? e : d2h(sec.gtab, c->gtab, 64 * (size_t)h.n_grains);
  e = e ? e : d2h(sec.gflags, c->gflags, 4 * (size_t)h.n_grains);
  e = e ? e : d2h(sec.gdtn, c->gdtn, 4 * (size_t)h.n_grains);
  e = e ? e : d2h(sec.npos, c->npos, 16 * (size_t)h.n_nuclei);
  e = e ? e : d2h(sec.ngrain, c->ngrain, 64 * (size_t)h.n_nuclei);
  e = e ? e : d2h(sec.nstate, c->nstate, 4 * (size_t)h.n_nuclei);
  e = e ? e : d2h(sec.rkey, c->R.key, 8 * (size_t)h.n_reached);
  // pool slots 0 .. n_blocks - 1 are the handed-out blocks
  e = e ? e : d2h(sec.bdata, c->C.data, 4 * (size_t)kBrickWords * (size_t)h.n_blocks);
  if (e) return e;
  std::vector<ulonglong2> bk((size_t)c->L.buckets);
  GP_CUDA(c, cudaMemcpyAsync(bk.data(), c->C.bucket, 16 * bk.size(), cudaMemcpyDeviceToHost,
                             c->st));
  GP_CUDA(c, cudaStreamSynchronize(c->st));
  // the key of every pool slot, from the buckets {key, slot + 1}
  std::vector<unsigned long long> keys((size_t)h.n_blocks, 0ull);
  int64_t found = 0;
  for (const ulonglong2& q : bk) {
    if (q.x == 0ull) continue;
    if (q.y == 0ull || q.y == kSlotFull || q.y - 1 >= (unsigned long long)h.n_blocks ||
        keys[q.y - 1] != 0ull)
      return fail(c, GP_ERR_STATE, "claim table inconsistent");
    keys[q.y - 1] = q.x;
    ++found;
  }
  if (found != h.n_blocks) return fail(c, GP_ERR_STATE, "claim table inconsistent");
  if (h.n_blocks) std::memcpy(b + sec.bkey, keys.data(), 8 * keys.size());
  std::memcpy(b, &h, sizeof h);
  h.checksum = ckpt_checksum(b, sec.total);
  std::memcpy(b + offsetof(CkptHeader, checksum), &h.checksum, sizeof h.checksum);
  return GP_OK;
}

gp_status gp_load(gp_ctx* c, const void* buf, size_t bytes) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (c->batch) return fail(c, GP_ERR_STATE, "checkpoints are of single-run contexts");
  if (c->tape_on) return fail(c, GP_ERR_STATE, "the adjoint tape is recording");
  s = sync_stats(c);
  if (s) return s;
  if (c->n_grains || c->n_live || c->n_obs || c->n_nuclei || c->step || c->hst->reached ||
      c->hst->claim_used)
    return fail(c, GP_ERR_STATE, "a checkpoint loads into a new context (no grains, "
                                 "particles, sites or steps yet)");
  CkptHeader h;
  CkptSections sec;
  if (const char* why = ckpt_invalid(buf, bytes, &h, &sec)) return fail(c, GP_ERR_ARG, why);
  if (std::memcmp(&h.dom, &c->dom[0], sizeof(gp_domain)) != 0 || h.h != c->h || h.dt != c->dt ||
      !same_law(h.law, c->law))
    return fail(c, GP_ERR_ARG, "checkpoint of another domain, h, dt or growth law");
  if (h.n_rec > c->L.cap) return fail(c, GP_ERR_CAPACITY, "particle capacity");
  if (h.n_grains > c->L.max_grains) return fail(c, GP_ERR_CAPACITY, "grain capacity");
  if (h.n_nuclei > c->L.max_nuclei) return fail(c, GP_ERR_CAPACITY, "nucleus capacity");
  if (h.n_reached > c->L.rcap) return fail(c, GP_ERR_CAPACITY, "reached-site capacity");
  if (h.n_blocks > c->L.blocks) return fail(c, GP_ERR_CAPACITY, "claim block capacity");
  if (h.thermal < 0 || h.thermal > 2 || h.periodic < 0 || h.periodic > 7 || h.obs_mode < 0 ||
      h.obs_mode > 2 || h.melting < 0 || h.melting > 1 || h.step < 0)
    return fail(c, GP_ERR_ARG, "checkpoint settings out of range");
  const unsigned char* b = static_cast<const unsigned char*>(buf);
  // the claim blocks are staged through the position buffer (16 bytes per particle of
  // capacity, idle between steps), a chunk at a time
  const int64_t per = (16 * c->L.cap - 16) / (8 + 4 * kBrickWords);
  if (h.n_blocks > 0 && per < 1)
    return fail(c, GP_ERR_CAPACITY, "particle capacity too small to stage the claim blocks");
  int64_t nfz = 0;
  for (int64_t i = 0; i < h.n_rec; ++i) {
    int4 v;
    std::memcpy(&v, b + sec.rec + 16 * (size_t)i, sizeof v);
    const Rec r = rec_unpack(v);
    bool ok = r.grain >= 0 && r.grain < h.n_grains && r.dir >= 0 && r.dir <= 5 &&
              (r.state == ST_ACTIVE || r.state == ST_FROZEN) && r.ell >= 0.f && r.ell < 1.f;
    for (int a = 0; a < 3; ++a) {
      const int sa = a == 0 ? r.sx : (a == 1 ? r.sy : r.sz);
      ok = ok && sa >= -kSiteMax && sa <= kSiteMax;
    }
    if (!ok) return fail(c, GP_ERR_ARG, "invalid particle in the checkpoint");
    nfz += r.state == ST_FROZEN;
  }
  // settings first: periodic axes refresh the cell geometry
  if (h.periodic) {
    s = gp_set_periodic(c, h.periodic);
    if (s) return s;
  }
  if (h.melting) {
    s = gp_set_melting(c, 1);
    if (s) return s;
  }
  c->obs_mode = h.obs_mode;
  if (h.thermal == 1) {  // a thermal grid is an input: the caller sets it again
    c->thermal = 1;
    c->P.thermal = 1;
    c->T0[0] = h.T0;
    c->Tdot[0] = h.Tdot;
    c->thermal_set[0] = 1;
    for (int a = 0; a < 3; ++a) {
      c->geo[0].G[a] = c->P.geo.G[a] = h.G[a];
      c->geo[0].xref[a] = c->P.geo.xref[a] = h.xref[a];
    }
  }
  auto h2d = [&](void* dst, size_t off, size_t n) -> gp_status {
    if (n) GP_CUDA(c, cudaMemcpyAsync(dst, b + off, n, cudaMemcpyHostToDevice, c->st));
    return GP_OK;
  };
  gp_status e = GP_OK;
  e = e ? e : h2d(c->rec[c->cur], sec.rec, 16 * (size_t)h.n_rec);
  e = e ? e : h2d(c->gtab, sec.gtab, 64 * (size_t)h.n_grains);
  e = e ? e : h2d(c->gflags, sec.gflags, 4 * (size_t)h.n_grains);
  e = e ? e : h2d(c->gdtn, sec.gdtn, 4 * (size_t)h.n_grains);
  e = e ? e : h2d(c->npos, sec.npos, 16 * (size_t)h.n_nuclei);
  e = e ? e : h2d(c->ngrain, sec.ngrain, 64 * (size_t)h.n_nuclei);
  e = e ? e : h2d(c->nstate, sec.nstate, 4 * (size_t)h.n_nuclei);
  e = e ? e : h2d(c->R.key, sec.rkey, 8 * (size_t)h.n_reached);
  if (e) return e;
  char* stg = reinterpret_cast<char*>(c->pos4);
  for (int64_t b0 = 0; b0 < h.n_blocks; b0 += per) {
    const int64_t m = std::min(per, h.n_blocks - b0);
    unsigned long long* dk = reinterpret_cast<unsigned long long*>(stg);
    uint32_t* dw = reinterpret_cast<uint32_t*>(stg + align16(8 * (size_t)m));
    e = e ? e : h2d(dk, sec.bkey + 8 * (size_t)b0, 8 * (size_t)m);
    e = e ? e : h2d(dw, sec.bdata + 4 * (size_t)kBrickWords * (size_t)b0,
                    4 * (size_t)kBrickWords * (size_t)m);
    if (e) return e;
    launch_claim_restore(c->C, dk, dw, m, c->st);
    GP_CUDA(c, cudaGetLastError());
    GP_CUDA(c, cudaStreamSynchronize(c->st));  // before the staging buffer is reused
  }
  // the counters as saved, but for what the load itself sets: every particle is in the
  // dynamic store, the reached sites are linked again before their next query, and the
  // claim pool holds the blocks just inserted
  GP_CUDA(c, cudaMemcpyAsync(c->hst, c->dst, sizeof(DevStats), cudaMemcpyDeviceToHost, c->st));
  GP_CUDA(c, cudaStreamSynchronize(c->st));
  DevStats nd = h.stats;
  nd.claim_used = c->hst->claim_used;
  nd.err = c->hst->err;
  nd.n_live = (unsigned long long)h.n_rec;
  nd.n_frozen = (unsigned long long)nfz;
  nd.n_grains = (unsigned long long)h.n_grains;
  nd.reached = (unsigned long long)h.n_reached;
  nd.linked = 0ull;
  nd.step = (unsigned long long)h.step;
  nd.stamp = c->hst->stamp;
  *c->hst = nd;
  GP_CUDA(c, cudaMemcpyAsync(c->dst, c->hst, sizeof(DevStats), cudaMemcpyHostToDevice, c->st));
  GP_CUDA(c, cudaStreamSynchronize(c->st));
  c->n_live = h.n_rec;
  c->n_grains = h.n_grains;
  c->n_nuclei = (int)h.n_nuclei;
  c->step = h.step;
  c->keys_valid = false;
  s = obs_reset(c);
  if (s) return s;
  return sync_stats(c);
}

gp_status gp_grain_map(gp_ctx* c, const gp_voxel_grid* g, int32_t* out, int32_t flags) {
  return gp_run_grain_map(c, 0, g, out, flags);
}

gp_status gp_run_grain_map(gp_ctx* c, int32_t run, const gp_voxel_grid* g, int32_t* out,
                           int32_t flags) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (run < 0 || run >= c->L.nruns) return fail(c, GP_ERR_ARG, "no such run");
  if (!g || !out) return fail(c, GP_ERR_ARG, "null argument");
  for (int a = 0; a < 3; ++a)
    if (g->n[a] < 0) return fail(c, GP_ERR_ARG, "negative voxel count");
  const int64_t nv = (int64_t)g->n[0] * g->n[1] * g->n[2];
  if (nv == 0) return GP_OK;
  const int nvox[3] = {g->n[0], g->n[1], g->n[2]};
  launch_link_reached(c->batch, c->P, c->R, &c->dst->linked, c->sms, c->st);
  c->prof.begin(K_GRAIN_MAP);
  if (flags & GP_DEVICE_PTR) {
    launch_grain_map(c->batch, c->P, run, c->R, g->origin, g->spacing, nvox, out, 0, nv, c->st);
  } else {
    int32_t* stg = reinterpret_cast<int32_t*>(c->pos4);
    const int64_t chunk = 4 * c->L.cap;
    for (int64_t v0 = 0; v0 < nv; v0 += chunk) {
      const int64_t m = std::min(chunk, nv - v0);
      launch_grain_map(c->batch, c->P, run, c->R, g->origin, g->spacing, nvox, stg, v0, m,
                       c->st);
      GP_CUDA(c, cudaMemcpyAsync(out + v0, stg, 4 * m, cudaMemcpyDeviceToHost, c->st));
      GP_CUDA(c, cudaStreamSynchronize(c->st));
    }
  }
  c->prof.end(K_GRAIN_MAP, (double)nv);
  GP_CUDA(c, cudaGetLastError());
  GP_CUDA(c, cudaStreamSynchronize(c->st));
  return GP_OK;
}

gp_status gp_run_counts(gp_ctx* c, int32_t nruns, int64_t* live, int64_t* active) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (nruns != c->L.nruns) return fail(c, GP_ERR_ARG, "nruns differs from the context's runs");
  std::vector<unsigned long long> h(2 * (size_t)nruns);
  GP_CUDA(c, cudaMemsetAsync(c->rcount, 0, 16 * (size_t)nruns, c->st));
  launch_run_counts(c->P, c->rec[c->cur], c->n_live, nruns, c->rcount, c->st);
  GP_CUDA(c, cudaMemcpyAsync(h.data(), c->rcount, 16 * (size_t)nruns, cudaMemcpyDeviceToHost,
                             c->st));
  GP_CUDA(c, cudaStreamSynchronize(c->st));
  GP_CUDA(c, cudaGetLastError());
  for (int r = 0; r < nruns; ++r) {
    if (live) live[r] = (int64_t)h[2 * r];
    if (active) active[r] = (int64_t)h[2 * r + 1];
  }
  return GP_OK;
}

gp_status gp_get_launch_config(gp_ctx* c, gp_launch_config* out) {
  if (!c || !out) return GP_ERR_ARG;
  out->build_ctas_per_sm = c->P.launch.build_ctas / c->sms;
  out->advance_ctas_per_sm = c->P.launch.advance_ctas / c->sms;
  out->emit_ctas_per_sm = c->P.launch.emit_ctas / c->sms;
  out->graph_steps = c->graph_steps;
  return GP_OK;
}

gp_status gp_set_launch_config(gp_ctx* c, const gp_launch_config* cfg) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (!cfg) return fail(c, GP_ERR_ARG, "null configuration");
  if (!c->batch) return fail(c, GP_ERR_STATE, "launch configurations apply to batch contexts");
  auto ok = [](int v, int hi) { return v >= 1 && v <= hi; };
  // resident CTAs per SM: 8 for the build and the advance (32 registers a thread), 6
  // for the emit (40); a larger grid only queues CTAs
  if (!ok(cfg->build_ctas_per_sm, 8) || !ok(cfg->advance_ctas_per_sm, 8) ||
      !ok(cfg->emit_ctas_per_sm, 8) || cfg->graph_steps < 0 || cfg->graph_steps > 1000)
    return fail(c, GP_ERR_ARG, "launch configuration out of range");
  c->P.launch.build_ctas = cfg->build_ctas_per_sm * c->sms;
  c->P.launch.advance_ctas = cfg->advance_ctas_per_sm * c->sms;
  c->P.launch.emit_ctas = cfg->emit_ctas_per_sm * c->sms;
  c->graph_steps = cfg->graph_steps;
  drop_graphs(c);
  return GP_OK;
}

gp_status gp_autotune(gp_ctx* c, int32_t trial_steps, gp_launch_config* best) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (!c->batch) return fail(c, GP_ERR_STATE, "the autotuner applies to batch contexts");
  if (trial_steps < 1) return fail(c, GP_ERR_ARG, "trial_steps < 1");
  gp_launch_config cur{};
  gp_get_launch_config(c, &cur);
  const int builds[] = {4, 8}, advances[] = {4, 8}, emits[] = {4, 6};
  cudaEvent_t ev[2];
  GP_CUDA(c, cudaEventCreate(&ev[0]));
  GP_CUDA(c, cudaEventCreate(&ev[1]));
  double best_cost = 1e300;
  gp_launch_config pick = cur;
  for (int b : builds)
    for (int a : advances)
      for (int e : emits) {
        if (s) break;
        gp_launch_config t = cur;
        t.build_ctas_per_sm = b;
        t.advance_ctas_per_sm = a;
        t.emit_ctas_per_sm = e;
        t.graph_steps = 0;
        s = gp_set_launch_config(c, &t);
        // cost of a configuration: device time per particle record of its trial steps
        // (the steps are real steps: every configuration gives the same results)
        double records = 0, ms = 0;
        for (int i = 0; i < trial_steps && !s; ++i) {
          records += (double)c->n_live;
          cudaEventRecord(ev[0], c->st);
          s = gp_step(c, 1);
          cudaEventRecord(ev[1], c->st);
          cudaEventSynchronize(ev[1]);
          float t_ms = 0;
          cudaEventElapsedTime(&t_ms, ev[0], ev[1]);
          ms += t_ms;
        }
        const double cost = ms / std::max(records, 1.0);
        if (!s && cost < best_cost) {
          best_cost = cost;
          pick = t;
        }
      }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (s) return s;
  pick.graph_steps = cur.graph_steps;
  s = gp_set_launch_config(c, &pick);
  if (s) return s;
  if (best) *best = pick;
  return GP_OK;
}

gp_status gp_grain_table(gp_ctx* c, int64_t cap, float* c3, int32_t* run, int64_t* n_out) {
  gp_status s = check_ctx(c);
  if (s) return s;
  if (cap < 0) return fail(c, GP_ERR_ARG, "cap < 0");
  s = sync_stats(c);
  if (s) return s;
  if (n_out) *n_out = c->n_grains;
  const int64_t m = std::min(cap, c->n_grains);
  if (m <= 0) return GP_OK;
  std::vector<float4> G(4 * (size_t)m);
  GP_CUDA(c, cudaMemcpyAsync(G.data(), c->gtab, sizeof(float4) * G.size(), cudaMemcpyDeviceToHost,
                             c->st));
  GP_CUDA(c, cudaStreamSynchronize(c->st));
  for (int64_t i = 0; i < m; ++i) {
    const float4 q = G[4 * i];
    if (c3) {
      c3[3 * i] = q.x;
      c3[3 * i + 1] = q.y;
      c3[3 * i + 2] = q.z;
    }
    if (run) std::memcpy(run + i, &q.w, sizeof(int32_t));
  }
  return GP_OK;
}

gp_status gp_profile(gp_ctx* c, int32_t enable) {
  if (!c) return GP_ERR_ARG;
  c->prof.reset();
  c->prof.on = enable != 0;
  return GP_OK;
}

gp_status gp_profile_read(gp_ctx* c, int32_t max, gp_kernel_prof* out, int32_t* n_out) {
  if (!c) return GP_ERR_ARG;
  c->prof.flush();
  int k = 0;
  for (int i = 0; i < K_COUNT; ++i) {
    if (c->prof.launches[i] == 0) continue;
    if (out && k < max) {
      std::memset(&out[k], 0, sizeof(gp_kernel_prof));
      std::snprintf(out[k].name, sizeof(out[k].name), "%s", kKernelNames[i]);
      out[k].launches = c->prof.launches[i];
      out[k].total_ms = c->prof.ms[i];
      out[k].units = c->prof.units[i];
      out[k].bytes_per_unit = kKernelBytes[i];
    }
    ++k;
  }
  if (n_out) *n_out = k;
  return GP_OK;
}

// ---------------------------------------------------------------------------------
// stand-alone hash / contact
// ---------------------------------------------------------------------------------
namespace {
// status of the sticky device error bits of a stand-alone call
gp_status sa_status(uint32_t err) {
  if (err & ERR_CELL_OVERFLOW) return GP_ERR_CAPACITY;
  if (err & ERR_TIMEOUT) return GP_ERR_TIMEOUT;
  return err ? GP_ERR_STATE : GP_OK;
}

struct SaLayout {
  size_t keys0, keys1, vals0, vals1, status, hist, tickets, err, flags, ofs, bsum, ncell, pos4,
      sstate, cells, total;
};
uint64_t sa_segments(const int nc[3]) {
  return (uint64_t)((nc[0] + kSegCells - 1) / kSegCells) * nc[1] * nc[2];
}
bool sa_layout(int64_t n, uint64_t nseg, SaLayout* L) {
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t a = o;
    o = align_up(o + b);
    return a;
  };
  const size_t m = (size_t)std::max<int64_t>(n, 1);
  L->keys0 = take(4 * m + 16);
  L->keys1 = take(4 * m + 16);
  L->vals0 = take(4 * m + 16);
  L->vals1 = take(4 * m + 16);
  L->status = take(4 * radix_status_words(n, 4));
  L->hist = take(4 * kSortMaxPasses * 256);
  L->tickets = take(64);
  L->err = take(64);
  L->flags = take(4 * m);
  L->ofs = take(4 * m);
  L->bsum = take(4 * ((m + 255) / 256) + 16);
  L->ncell = take(64);
  L->pos4 = take(16 * m);
  L->sstate = take(m);
  L->cells = take(16 * (size_t)nseg);
  L->total = o;
  return true;
}
Params sa_params(const gp_domain* d, double h, const int nc[3]) {
  Params P{};
  for (int a = 0; a < 3; ++a) {
    P.geo.lo[a] = (float)d->lo[a];
    P.geo.hi[a] = (float)d->hi[a];
    P.geo.nc[a] = nc[a];
  }
  P.geo.nsx = (nc[0] + kSegCells - 1) / kSegCells;
  P.inv_c = (float)(1.0 / cell_edge(h));
  for (int a = 0; a < 3; ++a) P.geo.inv[a] = P.inv_c;
  float hf = (float)h;
  P.rc2 = hf * hf;
  return P;
}
}  // namespace

gp_status gp_hash_workspace_bytes(int64_t n, const gp_domain* domain, double h,
                                  size_t* out_bytes) {
  if (!domain || !out_bytes || n < 0 || !(h > 0) || n >= (1ll << 30)) return GP_ERR_ARG;
  int nc[3];
  uint64_t ncells;
  if (!cells_of(domain, h, nc, &ncells)) return GP_ERR_ARG;
  SaLayout L;
  sa_layout(n, sa_segments(nc), &L);
  *out_bytes = L.total;
  return GP_OK;
}

static gp_status sa_sort(const float* x3, const uint8_t* state, int64_t n, const gp_domain* domain,
                         double h, void* ws, size_t wsb, cudaStream_t st, SaLayout* L,
                         Params* P, uint64_t* ncells, int* w, SortBufs* sb) {
  int nc[3];
  if (!cells_of(domain, h, nc, ncells)) return GP_ERR_ARG;
  sa_layout(n, sa_segments(nc), L);
  if (!ws || wsb < L->total || ((uintptr_t)ws & (kAlign - 1))) return GP_ERR_ARG;
  char* b = (char*)ws;
  *P = sa_params(domain, h, nc);
  sb->keys[0] = (uint32_t*)(b + L->keys0);
  sb->keys[1] = (uint32_t*)(b + L->keys1);
  sb->vals[0] = (uint32_t*)(b + L->vals0);
  sb->vals[1] = (uint32_t*)(b + L->vals1);
  sb->status = (uint32_t*)(b + L->status);
  sb->hist = (uint32_t*)(b + L->hist);
  sb->ticket = (uint32_t*)(b + L->tickets);
  sb->err = (uint32_t*)(b + L->err);
  sb->max_n = n;
  int dev = 0;
  cudaGetDevice(&dev);
  sb->sms = 152;
  cudaDeviceGetAttribute(&sb->sms, cudaDevAttrMultiProcessorCount, dev);
  sb->prof = nullptr;
  if (cudaMemsetAsync(sb->err, 0, 64, st) != cudaSuccess) return GP_ERR_CUDA;
  launch_keys_pos(*P, x3, state, n, (uint32_t*)sb->keys[0], sb->vals[0], st);
  uint64_t nm1 = *ncells - 1;
  int nbits = 0;
  while (nm1) {
    ++nbits;
    nm1 >>= 1;
  }
  if (state) nbits = 32;  // removed points carry key 0xffffffff and sort last
  *w = radix_sort<uint32_t>(*sb, n, nbits, st);
  return *w < 0 ? GP_ERR_ARG : GP_OK;
}

gp_status gp_hash_build(const float* x3, int64_t n, const gp_domain* domain, double h,
                        uint32_t* keys_sorted, int32_t* ids_sorted, uint32_t* cell_keys,
                        int32_t* cell_start, int64_t* n_cells, void* workspace,
                        size_t workspace_bytes, void* cuda_stream) {
  if (!domain || n < 0 || n >= (1ll << 30) || !(h > 0)) return GP_ERR_ARG;
  if (n > 0 && (!x3 || !keys_sorted || !ids_sorted || !cell_keys || !cell_start))
    return GP_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (n == 0) {
    if (n_cells) *n_cells = 0;
    return GP_OK;
  }
  SaLayout L;
  Params P;
  uint64_t ncells;
  int w;
  SortBufs sb{};
  gp_status s = sa_sort(x3, nullptr, n, domain, h, workspace, workspace_bytes, st, &L, &P,
                        &ncells, &w, &sb);
  if (s) return s;
  char* b = (char*)workspace;
  const uint32_t* skeys = (const uint32_t*)sb.keys[w];
  if (cudaMemcpyAsync(keys_sorted, skeys, 4 * n, cudaMemcpyDeviceToDevice, st) ||
      cudaMemcpyAsync(ids_sorted, sb.vals[w], 4 * n, cudaMemcpyDeviceToDevice, st) ||
      cudaMemsetAsync(b + L.ncell, 0, 8, st))
    return GP_ERR_CUDA;
  launch_cells(skeys, n, (uint32_t)ncells, (uint32_t*)(b + L.flags), (uint32_t*)(b + L.ofs),
               (uint32_t*)(b + L.bsum), cell_keys, cell_start,
               (unsigned long long*)(b + L.ncell), st);
  unsigned long long nc = 0;
  uint32_t err = 0;
  if (cudaMemcpyAsync(&nc, b + L.ncell, 8, cudaMemcpyDeviceToHost, st) ||
      cudaMemcpyAsync(&err, sb.err, 4, cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st) ||
      cudaGetLastError())
    return GP_ERR_CUDA;
  if (err) return sa_status(err);
  if (n_cells) *n_cells = (int64_t)nc;
  return GP_OK;
}

gp_status gp_contact(const float* x3, const int32_t* grain, const uint8_t* state, int64_t n,
                     const gp_domain* domain, double h, uint8_t* freeze, int32_t* pairs,
                     int64_t pair_cap, int64_t* n_pairs, void* workspace, size_t workspace_bytes,
                     void* cuda_stream) {
  if (!domain || n < 0 || n >= (1ll << 30) || !(h > 0) || pair_cap < 0) return GP_ERR_ARG;
  if (n > 0 && (!x3 || !grain || !state)) return GP_ERR_ARG;
  if (pairs && !n_pairs) return GP_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (n == 0) {
    if (n_pairs) *n_pairs = 0;
    return GP_OK;
  }
  SaLayout L;
  Params P;
  uint64_t ncells;
  int w;
  SortBufs sb{};
  gp_status s = sa_sort(x3, state, n, domain, h, workspace, workspace_bytes, st, &L, &P, &ncells,
                        &w, &sb);
  if (s) return s;
  char* b = (char*)workspace;
  const uint32_t* skeys = (const uint32_t*)sb.keys[w];
  if (cudaMemsetAsync(b + L.cells, 0, 16 * sa_segments(P.geo.nc), st) ||
      cudaMemsetAsync(b + L.ncell, 0, 8, st))
    return GP_ERR_CUDA;
  if (freeze && cudaMemsetAsync(freeze, 0, n, st)) return GP_ERR_CUDA;
  launch_build_sa(P, x3, grain, state, skeys, sb.vals[w], n, (float4*)(b + L.pos4),
                  (uint8_t*)(b + L.sstate), (uint4*)(b + L.cells), sb.err, st);
  launch_contact_sa(P, (const float4*)(b + L.pos4), (const uint8_t*)(b + L.sstate), sb.vals[w],
                    skeys, (const uint4*)(b + L.cells), n, freeze, pairs,
                    pair_cap, (unsigned long long*)(b + L.ncell), st);
  unsigned long long np = 0;
  uint32_t err = 0;
  if (cudaMemcpyAsync(&np, b + L.ncell, 8, cudaMemcpyDeviceToHost, st) ||
      cudaMemcpyAsync(&err, sb.err, 4, cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st) ||
      cudaGetLastError())
    return GP_ERR_CUDA;
  if (err) return sa_status(err);
  if (n_pairs) *n_pairs = (int64_t)np;
  return GP_OK;
}

gp_status gp_selftest_wait(int32_t which, uint32_t spin_limit, void* cuda_stream) {
  if (which < 0 || which > 1 || spin_limit < 1 || spin_limit > kSpinLimit) return GP_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  uint32_t* words = nullptr;
  if (cudaMalloc((void**)&words, 4 * 513) != cudaSuccess) return GP_ERR_CUDA;
  uint32_t err = 0;
  cudaError_t e = cudaMemsetAsync(words, 0, 4 * 513, st);
  if (e == cudaSuccess && which == 1) {  // bucket 0: key set, slot never published
    const unsigned long long key = 1ull;
    e = cudaMemcpyAsync(words, &key, sizeof(key), cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) {
    launch_selftest_wait(which, spin_limit, words, words + 512, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, words + 512, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(words);
  if (e != cudaSuccess) return GP_ERR_CUDA;
  return err & ERR_TIMEOUT ? GP_ERR_TIMEOUT : (err ? GP_ERR_STATE : GP_OK);
}

}  // extern "C"
