/*
 * gp.h - C ABI of the GB300 (sm_103a) grain-envelope particle library.
 *
 * The library implements the per-timestep update of the particle-based grain
 * envelope tracking method of Mosbah et al., "A particle-based approach for the
 * prediction of grain microstructures in solidification processes"
 * (arXiv 2504.12858), Sec. 2.1 and 2.3:
 *   nucleation activation (Sec. 2.1.1), growth of tracking points along the
 *   rotated <100> directions with a power-law tip velocity (Sec. 2.1.2, Eq. 1 and
 *   Eq. 2), generation of outer tracking points every lambda_0 (Sec. 2.1.2,
 *   Fig. 2), impingement of grains by a cell-list contact search (Sec. 2.1.2 and
 *   Sec. 2.3) and grain-id voxelisation by nearest tracking information
 *   (Sec. 2.3).
 *
 * Conventions for every call:
 *  - Units are SI.  Scalars and host arrays at the boundary are double precision;
 *    the device state is binary32.
 *  - Every call returns a gp_status.  On failure gp_last_error(ctx) returns a
 *    message.  A status other than GP_OK from gp_step leaves the context in an
 *    error state: only gp_stats, gp_last_error and gp_destroy remain valid.
 *  - Host input arrays are read during the call and not retained: the caller
 *    keeps ownership.  Output arrays are caller-allocated.
 *  - A context is bound to the CUDA device current at gp_create and to one CUDA
 *    stream; all its work is ordered on that stream.  A context is not
 *    thread-safe.  Calls that return data to host memory synchronise the stream.
 *  - Lattice sites are integer coordinates in the crystal frame of a grain,
 *    relative to its nucleus, |s_a| <= 4095 (gp_create rejects domains whose
 *    diagonal exceeds 4000 lattice spacings).
 *  - Directions k = 0..5 are +x, -x, +y, -y, +z, -z of the crystal frame.
 *  - Particle states: 0 ACTIVE, 1 FROZEN (stopped by another grain), 2 REMOVED.
 */
#ifndef GP_H
#define GP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GP_OK = 0,
  GP_ERR_ARG = 1,       /* invalid argument (null pointer, bad size, bad value)  */
  GP_ERR_CAPACITY = 2,  /* a particle, site, grain or nucleus capacity exceeded  */
  GP_ERR_HASH_FULL = 3, /* the lattice-site claim table is full                  */
  GP_ERR_CUDA = 4,      /* a CUDA runtime call failed                            */
  GP_ERR_STATE = 5,     /* call not valid in the current state                   */
  GP_ERR_TIMEOUT = 6    /* a bounded device-side wait gave up                    */
} gp_status;

typedef struct gp_ctx gp_ctx;

/* Axis-aligned simulation box [lo, hi] (m).  Particles leaving it are removed. */
typedef struct {
  double lo[3], hi[3];
} gp_domain;

/* Tip-velocity law v(dT) for dT = T_L - T > 0, zero otherwise.
 * nterms = 1: v = a[0] dT^b[0]                       (Eq. 1)
 * nterms = 2: v = a[0] dT^b[0] + a[1] dT^b[1]        (Eq. 2)
 * T_liquidus is T_L of the alloy at its nominal composition (Sec. 2.1.2). */
typedef struct {
  int32_t nterms;
  double a[2], b[2];
  double T_liquidus;
} gp_growth_law;

/* Imposed temperature T(x, t) = T0 + G . (x - x_ref) + Tdot t
 * (frozen-temperature approximation, Sec. 3.3 / 3.4). */
typedef struct {
  double T0, G[3], x_ref[3], Tdot;
} gp_thermal_analytic;

/* Imposed temperature tabulated on a node-centred grid that moves with velocity
 * frame_vel: node (i,j,k) sits at origin + frame_vel t + (i,j,k) * spacing; T is
 * n[0]*n[1]*n[2] binary32 values, x fastest.  Sampled trilinearly after clamping
 * to the table (this replaces the cellPointFace interpolation of Sec. 2.3).
 * flags & GP_DEVICE_PTR: T is a device pointer (copied device-to-device),
 * otherwise a host pointer.  Each n[a] >= 2. */
typedef struct {
  const float* T;
  int32_t n[3];
  double origin[3], spacing[3], frame_vel[3];
  int32_t flags;
} gp_thermal_grid;

/* Composition field for a local liquidus T_L(w) = T_m + m_L w(x, t): ΔT then is
 * T_L(w(x, t)) - T(x, t) instead of taking T_L at the nominal composition.
 * Sec. 2.1.2 states that the velocity may depend on T and w; Sec. 2.1.3 notes the
 * extension of the nominal liquidus to the local composition; Sec. 3.3 / 3.4 take
 * the undercooling with respect to the local solute concentration.  w is tabulated
 * like gp_thermal_grid (node-centred, x fastest, moving with frame_vel, trilinear
 * after clamping); m_L is the liquidus slope in K per unit of w. */
typedef struct {
  const float* w;
  int32_t n[3];
  double origin[3], spacing[3], frame_vel[3];
  double T_m, m_L;
  int32_t flags;
} gp_solute_grid;

/* Voxel grid for gp_grain_map: voxel centres origin + (i + 1/2) spacing. */
typedef struct {
  double origin[3], spacing[3];
  int32_t n[3];
} gp_voxel_grid;

/* Capacities and memory.  Zero fields take defaults (given per field).  If arena
 * is non-NULL it must be device memory of arena_bytes >= gp_arena_bytes(...),
 * 256-byte aligned; the library then allocates no device memory of its own and
 * the caller keeps the arena alive until gp_destroy.  If arena is NULL the
 * library allocates (and frees) its memory with cudaMalloc. */
typedef struct {
  int64_t capacity;         /* live (ACTIVE + FROZEN) particles; required > 0     */
  int64_t reached_capacity; /* reached lattice sites; default 2 * capacity        */
  int64_t claim_blocks;     /* 8^3-site blocks of lattice-site claims (512 bytes
                               each, allocated on first claim); default
                               capacity / 32                                      */
  int32_t max_grains;       /* default 1 << 20                                    */
  int32_t max_nuclei;       /* pending nucleation sites; default 4096             */
  int64_t grid_nodes;       /* thermal-grid nodes reserved in the arena; default 0 */
  int64_t tape_steps;       /* steps the adjoint tape holds; default 0 (none).  Per
                               particle of capacity: 6 bytes per step, 16 bytes per
                               checkpoint, 36 bytes of scratch                      */
  void* arena;
  size_t arena_bytes;
  int64_t solute_nodes;     /* composition-grid nodes reserved in the arena; default 0 */
  int64_t tape_checkpoint_every; /* the tape keeps the particle records of every k-th
                               step only and rebuilds the others in the reverse sweep
                               (k replays per taped step at most); default 1        */
} gp_memory;

typedef struct {
  int64_t step;           /* timesteps taken (t = step * dt)                      */
  int64_t n_live;         /* ACTIVE + FROZEN particles                            */
  int64_t n_active;
  int64_t n_frozen;
  int64_t n_grains;
  int64_t n_reached;      /* reached lattice sites recorded                        */
  int64_t particle_steps; /* sum over steps of the ACTIVE particles at step start  */
  int64_t n_frozen_new;   /* particles frozen by contact (cumulative)              */
  int64_t n_spawned;      /* new particles from outer directions (cumulative)      */
  int64_t n_claims_lost;  /* spawn candidates refused by the claim rule            */
  int64_t n_clipped;      /* particles removed at the domain boundary              */
  int64_t n_clamped;      /* advances capped at one lattice spacing per step       */
  int64_t n_nucleated;
  int64_t n_claim_blocks; /* claim blocks in use (at most gp_memory.claim_blocks)   */
  int64_t error_flags;    /* sticky device error bits (0 when healthy)             */
  int64_t n_melted;       /* reached sites melted (cumulative, gp_set_melting)     */
  int64_t n_walkback;     /* particles re-activated by the walk-back (cumulative)  */
  int64_t reserved[3];
} gp_stats_t;

/* Per-kernel timing collected with CUDA events when profiling is enabled. */
typedef struct {
  char name[32];
  int64_t launches;       /* kernel launches (some entries time several kernels)  */
  double total_ms;
  double units;           /* items processed (particles, keys, voxels) summed     */
  double bytes_per_unit;  /* algorithmic DRAM bytes per item                      */
} gp_kernel_prof;

#define GP_DEVICE_PTR 1

/* ---- context ------------------------------------------------------------------ */

/* Device bytes gp_create needs for this domain, spacing h and capacities. */
gp_status gp_arena_bytes(const gp_domain* domain, double h, const gp_memory* mem,
                         size_t* out_bytes);

/* Creates a simulation with lattice spacing h = lambda_0 (Sec. 2.1.2; also the
 * contact radius; the spatial hash uses cells of edge h (1 + 2^-9)) and
 * timestep dt.  Returns GP_ERR_ARG if the domain spans more than 4000 lattice
 * spacings along its diagonal or more than 2^32 hash cells.
 * cuda_stream is a cudaStream_t (NULL: the legacy default stream). */
gp_status gp_create(const gp_domain* domain, double h, double dt, const gp_growth_law* law,
                    const gp_memory* mem, void* cuda_stream, gp_ctx** out);

gp_status gp_destroy(gp_ctx* ctx);

const char* gp_last_error(const gp_ctx* ctx);

/* ---- set-up ------------------------------------------------------------------ */

/* Adds n grains with nuclei at pos3 (n x 3) and crystal->lab orientations given
 * as unit quaternions quat4 (n x 4, w x y z; normalised here).  If nucleate != 0
 * each grain starts with its six tracking points at the nucleus (Sec. 2.1.2,
 * Fig. 2 Step 0).  *out_first_id (optional) receives the id of the first grain;
 * ids are consecutive. */
gp_status gp_add_grains(gp_ctx* ctx, int64_t n, const double* pos3, const double* quat4,
                        int32_t nucleate, int32_t* out_first_id);

/* Seeds each listed grain with the envelope a nucleus reaches after n0 complete
 * lattice shells in a uniform melt: one ACTIVE particle per site t with
 * |t|_1 = n0 + 1, placed at the site reached from the lowest axis a with
 * t_a != 0, heading to t, with progress ell0 in [0,1).  Sites with |s|_1 = n0
 * are recorded as reached; they and the targets are claimed.  Particles outside
 * the domain are not seeded. */
gp_status gp_seed_shell(gp_ctx* ctx, int64_t n, const int32_t* grains, int32_t n0,
                        double ell0);

gp_status gp_set_thermal_analytic(gp_ctx* ctx, const gp_thermal_analytic* th);
gp_status gp_set_thermal_grid(gp_ctx* ctx, const gp_thermal_grid* th);

/* Periodic axes of a single-run context (Sec. 3.4 applies periodic conditions on
 * the faces normal to x and y): axes is a bit mask (1 = x, 2 = y, 4 = z).  Along a
 * periodic axis a point is identified with its images x + m L (L = hi - lo):
 * positions wrap into [lo, hi) for the hash, the fields and the grain map, distances
 * take the nearest image, and nothing is clipped.  A grain's lattice is unbounded,
 * so a grain crossing a periodic face continues on the other side.  The contact
 * cells divide each period into floor(L / edge) equal cells, at least three
 * (GP_ERR_ARG otherwise).  GP_ERR_STATE on a batch context or while the adjoint tape
 * records; the adjoint refuses periodic contexts. */
gp_status gp_set_periodic(gp_ctx* ctx, int32_t axes);

/* Melting (Sec. 2.1.3).  With enable != 0 every step of a single-run context starts,
 * at t_n, with a melting pass in which:
 *   - every reached lattice site whose position has Delta T < 0 melts: it is no
 *     longer reached nor claimed (gp_get_reached and the grain map skip it);
 *   - every particle whose position has Delta T < 0, or whose site has melted, is
 *     removed, and its target is released;
 *   - walk-back: each melted site m gets one new ACTIVE particle (ell = 0), from
 *     its neighbour m - e_k for the first direction k = 0..5 whose neighbour is
 *     still reached, heading to m, which it claims (the two sites straddle the
 *     Delta T = 0 surface, within the paper's search distance of 2 lambda_0);
 *   - a grain left without reached sites keeps its seed, which nucleates again,
 *     with the same grain id and six particles, once its nucleation undercooling is
 *     reached (0 for grains from gp_add_grains) and no reached site lies within h.
 * The pass visits every reached site, so it costs about the reached-site list per
 * step.  Grains seeded with gp_seed_shell record only their outer shell, so their
 * interior counts as liquid.  GP_ERR_STATE on a batch context or while the adjoint
 * tape records. */
gp_status gp_set_melting(gp_ctx* ctx, int32_t enable);

/* Obstacle store of a single-run context.  A particle stopped by another grain
 * (FROZEN) never moves again: the points where two grains meet stop for good and
 * form the grain boundary (Sec. 2.1.2, impingement).  Instead of carrying FROZEN
 * particles through the per-step ordering, gather and compaction, the library moves
 * them, in batches, into an obstacle store ordered by cell, with their positions.  Each
 * step's ordering lays out the moving particles and the obstacles in one cell-ordered
 * sequence with one cell table, which the contact search reads; a tile of 16 x 8 x 8
 * cells that holds no moving particle is read in place from the store instead of being
 * copied.  Results do not depend on the mode; only the cost does.
 *   mode 0: off, every particle stays in the per-step store (obstacles already
 *           moved go back to it);
 *   mode 1 (default): a batch is moved once carrying the FROZEN particles from step
 *           to step has cost about as much as merging them into the store;
 *   mode 2: every step that starts with FROZEN particles in the per-step store.
 * The store is not used by a batch context, with periodic axes, with melting (which
 * removes frozen particles) or while the adjoint tape records; turning any of these on
 * moves the obstacles back.  gp_get_particles lists the per-step store first, then
 * the obstacle store; gp_stats counts both.  GP_ERR_ARG for another mode. */
gp_status gp_set_obstacle_store(gp_ctx* ctx, int32_t mode);

/* Inspection of the ordering of the particle step (used by the tests; the paper has
 * no counterpart).  which = 0: runs on the current state the ordering the next gp_step
 * starts with, without advancing the state: the cell key of every particle, and the
 * cell-ordered sequence that the contact search reads, which holds the particles of
 * the per-step store (grouped by tile of 1024 cells, ordered by cell inside each tile)
 * and those of the obstacle store; it copies to host arrays (any may be NULL):
 *   keys_in     the cell key of every particle, in the order of gp_get_particles;
 *   keys_sorted the keys of the sequence (*n_out entries, all particles);
 *   src         the gp_get_particles index of each entry of the sequence;
 *   table       4 words per segment of 16 cells (table_cap segments at most): index
 *               of its first entry, stamp << 16 | saturation flag << 15 | count, then the
 *               4-bit counts (saturated at 15) of cells 0-7 and 8-15; an entry whose
 *               stamp differs from *stamp is an empty segment.
 * Particles of one cell may come in any order (the ordering places them by atomic
 * counters); keys, cells and counts are exact.  The inspection copies every obstacle
 * into the sequence; the step reads those of tiles without moving particles in place.
 * which = 1: the obstacle store: its
 * *n_out keys in its order in keys_sorted, src the gp_get_particles index of each (the
 * obstacles are the last particles that gp_get_particles lists), no table (*n_seg = 0).
 * GP_ERR_STATE on a batch context. */
gp_status gp_inspect_order(gp_ctx* ctx, int32_t which, int64_t cap, uint32_t* keys_in,
                           uint32_t* keys_sorted, uint32_t* src, int64_t* n_out,
                           uint32_t* table, int64_t table_cap, int64_t* n_seg,
                           uint32_t* stamp);

/* Sets (or replaces) the composition field of a single-run context; the grid is
 * copied into the arena (gp_memory.solute_nodes) or, for a library-allocated
 * context, into memory the library allocates.  GP_ERR_STATE on a batch context;
 * gp_tape_begin refuses a context with a composition field. */
gp_status gp_set_solute_grid(gp_ctx* ctx, const gp_solute_grid* sg);

/* Registers n pending nucleation sites (Sec. 2.1.1): position pos3 (n x 3),
 * nucleation undercooling dTn (n) and orientation quat4 (n x 4).  A site becomes
 * a grain at the end of the first step after which its undercooling is >= dTn,
 * unless a reached site of an existing grain lies within h of it.  Grain ids of
 * sites activating in the same step follow registration order. */
gp_status gp_nucleation_sites(gp_ctx* ctx, int64_t n, const double* pos3, const double* dTn,
                              const double* quat4);

/* ---- time stepping ----------------------------------------------------------- */

/* Advances nsteps timesteps.  Each step: spatial hash of all live particles,
 * contact freeze, thermal sample and growth law at (x_n, t_n), explicit Euler
 * advance capped at one lattice spacing, spawning of outer points at reached
 * sites with the once-per-site claim rule, domain clip, nucleation at t_{n+1}. */
gp_status gp_step(gp_ctx* ctx, int32_t nsteps);

/* Grain id of every voxel centre: the grain of the nearest reached lattice site
 * closer than h (ties: smaller grain id), else -1 (Sec. 2.3 Voronoi
 * interpolation).  out has n[0]*n[1]*n[2] int32 values, x fastest; it is a device
 * pointer if flags & GP_DEVICE_PTR, else host memory. */
gp_status gp_grain_map(gp_ctx* ctx, const gp_voxel_grid* grid, int32_t* out, int32_t flags);

/* ---- state access -------------------------------------------------------------- */

gp_status gp_stats(gp_ctx* ctx, gp_stats_t* out);

/* Copies up to cap live particles to host arrays (any may be NULL): grain,
 * site3 (cap x 3), dir, ell, state, x3 (cap x 3, binary32 positions).  *n_out
 * receives the number of live particles.  Order is the library's store order. */
gp_status gp_get_particles(gp_ctx* ctx, int64_t cap, int32_t* grain, int32_t* site3,
                           int8_t* dir, float* ell, uint8_t* state, float* x3,
                           int64_t* n_out);

/* Replaces the particle set with n particles given on the host and sets the step
 * counter (state import, e.g. from a checkpoint). */
gp_status gp_load_particles(gp_ctx* ctx, int64_t n, const int32_t* grain,
                            const int32_t* site3, const int8_t* dir, const float* ell,
                            const uint8_t* state, int64_t step);

/* Marks n lattice sites (grain, site3) as reached (reached != 0) and/or claimed
 * (claimed != 0). */
gp_status gp_add_sites(gp_ctx* ctx, int64_t n, const int32_t* grain, const int32_t* site3,
                       int32_t reached, int32_t claimed);

/* Copies up to cap reached sites (grain, site3) to the host; *n_out = count. */
gp_status gp_get_reached(gp_ctx* ctx, int64_t cap, int32_t* grain, int32_t* site3,
                         int64_t* n_out);

/* ---- checkpoints (not in the paper, which keeps no run state on disk) --------- */

/* Checkpoint of a single-run context between steps, written to the caller's host
 * buffer buf of cap bytes; *bytes receives its size (buf == NULL: the size only, nothing
 * written).  It holds every particle record (dynamic and obstacle store), the grain
 * frames and melted-grain flags, the nucleation sites and their activation state, the
 * reached-site list, the claim blocks (key and claim bytes of each), the step counter,
 * the device counters, the periodic axes, the melting and obstacle-store settings and an
 * analytic thermal field.  A thermal grid or a solute grid is an input of the caller and
 * is not saved.  A 64-bit FNV-1a checksum covers the whole buffer.  The buffer stays the
 * caller's.  GP_ERR_STATE for a batch context or while the adjoint tape records;
 * GP_ERR_CAPACITY if cap is smaller than the checkpoint (nothing written). */
gp_status gp_save(gp_ctx* ctx, void* buf, size_t cap, size_t* bytes);

/* Loads a checkpoint of gp_save (host buffer of bytes bytes, read during the call) into
 * a new single-run context: no grains, particles, nucleation sites, reached sites or
 * steps yet, created with the same domain, h, dt and growth law; its capacities may
 * differ as long as the saved state fits.  Every particle starts in the dynamic store.
 * Stepping on gives the particles, reached sites, grain maps and counters that the
 * saved run gives.  A thermal grid or a solute grid is set again by the caller (before
 * or after the load).  GP_ERR_ARG for a buffer that is not an intact checkpoint (magic,
 * format version, size, checksum), holds an invalid particle, or is of another domain,
 * h, dt or growth law; GP_ERR_CAPACITY if the saved state does not fit; GP_ERR_STATE for
 * a batch context, a context that is not new, or while the adjoint tape records. */
gp_status gp_load(gp_ctx* ctx, const void* buf, size_t bytes);

/* Host-only check of a checkpoint buffer (no context, no device call): GP_OK if buf
 * holds an intact checkpoint of this format, with its step counter and particle count
 * in *step and *n_particles (each optional); GP_ERR_ARG otherwise. */
gp_status gp_checkpoint_check(const void* buf, size_t bytes, int64_t* step,
                              int64_t* n_particles);

/* Enables (1) / disables (0) per-kernel CUDA-event timing and resets it. */
gp_status gp_profile(gp_ctx* ctx, int32_t enable);
/* Copies up to max entries of per-kernel timing; *n_out = number of kernels. */
gp_status gp_profile_read(gp_ctx* ctx, int32_t max, gp_kernel_prof* out, int32_t* n_out);

/* ---- adjoint of the advance ---------------------------------------------------- */

/* Starts recording the adjoint tape: the next steps (at most gp_memory.tape_steps)
 * store the state of every particle after the contact search, the parent and the
 * direction of every particle of the following step, and, every
 * gp_memory.tape_checkpoint_every steps, the particle records before the step.  The
 * reverse sweep rebuilds the records of the steps between checkpoints by replaying
 * these events with the forward's arithmetic.  Recording restarts at every call.
 * Needs an analytic field; with checkpoints every k > 1 steps, GP_ERR_STATE while
 * nucleation sites are pending (a nucleation is not replayed). */
gp_status gp_tape_begin(gp_ctx* ctx);

/* Reverse sweep over the taped steps, with the discrete events of the forward run
 * (contacts, spawns, clips, the one-spacing cap) held fixed.  Each particle's
 * progress obeys ell' = ell + dl (minus one at a spawn, for every child), with
 * dl = v(dT(x(ell), t)) dt / h (Eq. 1/2, Sec. 2.1.2), so
 *   d ell'/d ell = 1 + d dl/d ell   and   d ell'/d theta = d dl/d theta.
 * seed: dL/d ell of every live particle after the last taped step, in store order
 * (the order of gp_get_particles), n of them; device pointer if flags &
 * GP_DEVICE_PTR, else host.  grad[8] receives dL/d(a[0], b[0], a[1], b[1], G[0],
 * G[1], G[2], Tdot) of the growth law and the analytic field.  The taped steps
 * must end at the current step. */
gp_status gp_adjoint(gp_ctx* ctx, const float* seed, int64_t n, int32_t flags, double grad[8]);

/* ---- batches of independent runs ----------------------------------------------- */

/* A batch context advances nruns (1..256) independent simulations together, for
 * ensembles of seeds, orientations and thermal histories such as a
 * columnar-to-equiaxed transition map (Sec. 3.5).  Each run r has its own domain
 * domains[r], analytic field, grains and nucleation sites; all runs share h, dt,
 * the growth law and the capacities of mem (the particle, reached-site, claim,
 * grain and nucleus pools are shared).  A run never sees another run's particles:
 * the spatial hash, the contact search, the clip and the nucleation test of a
 * particle use its own run's domain and cells only, so every run evolves exactly
 * as it would alone in a single-run context (same binary32 arithmetic).  Every
 * kernel of a step covers all runs in one launch.  The hash tables of all runs
 * are dense and laid out one after the other: the arena grows by about 1.5 bytes
 * per hash cell of every run.  The single-run calls (gp_add_grains, gp_step,
 * gp_stats, gp_get_particles, ...) apply to a batch context too and act on run 0
 * where they take no run; gp_step advances all runs.  A batch takes analytic
 * fields only (no gp_set_thermal_grid, gp_seed_shell or adjoint tape). */
gp_status gp_batch_arena_bytes(int32_t nruns, const gp_domain* domains, double h,
                               const gp_memory* mem, size_t* out_bytes);
gp_status gp_batch_create(int32_t nruns, const gp_domain* domains, double h, double dt,
                          const gp_growth_law* law, const gp_memory* mem, void* cuda_stream,
                          gp_ctx** out);

/* The calls of the same name without "run_", for run `run` of a context (a
 * single-run context has run 0 only).  Grain ids are global to the context. */
gp_status gp_run_set_thermal_analytic(gp_ctx* ctx, int32_t run, const gp_thermal_analytic* th);
gp_status gp_run_add_grains(gp_ctx* ctx, int32_t run, int64_t n, const double* pos3,
                            const double* quat4, int32_t nucleate, int32_t* out_first_id);
/* In a batch context every site reserves its grain id at registration: the sites
 * of one call get consecutive ids from *out_first_grain on (a single-run context
 * numbers grains at activation and writes -1). */
gp_status gp_run_nucleation_sites(gp_ctx* ctx, int32_t run, int64_t n, const double* pos3,
                                  const double* dTn, const double* quat4,
                                  int32_t* out_first_grain);
gp_status gp_run_grain_map(gp_ctx* ctx, int32_t run, const gp_voxel_grid* grid, int32_t* out,
                           int32_t flags);

/* Live (live[r]) and ACTIVE (active[r]) particles of each of the nruns runs
 * (host arrays, either may be NULL); nruns must equal the context's run count. */
gp_status gp_run_counts(gp_ctx* ctx, int32_t nruns, int64_t* live, int64_t* active);

/* Launches of a batch step.  Every kernel of a batch step sizes itself on the
 * device: the counts live in device memory and the grids are persistent
 * (*_ctas_per_sm CTAs per SM over the whole GPU: build 1..8, advance 1..8, emit
 * 1..8; eight, eight and six are resident at once).  graph_steps > 0 captures graph_steps consecutive steps in a CUDA
 * graph on first use and replays it (no host round trip inside a graph; the
 * context's stream must not be the legacy default stream); 0 issues the launches
 * step by step.  Results do not depend on the configuration. */
typedef struct {
  int32_t build_ctas_per_sm, advance_ctas_per_sm, emit_ctas_per_sm;
  int32_t graph_steps;
} gp_launch_config;
gp_status gp_get_launch_config(gp_ctx* ctx, gp_launch_config* out);
gp_status gp_set_launch_config(gp_ctx* ctx, const gp_launch_config* cfg);

/* Autotuner of the batch launches: runs trial_steps real steps of the simulation
 * with each candidate configuration (build 4/8, advance 2/5, emit 4/8 CTAs per SM),
 * times them with CUDA events, keeps the configuration with the least device time
 * per particle record (graph_steps unchanged) and writes it to *best (optional). */
gp_status gp_autotune(gp_ctx* ctx, int32_t trial_steps, gp_launch_config* best);

/* Nucleus position (binary32, c3: cap x 3) and run of up to cap grains, by grain
 * id; *n_out receives the number of grains (including reserved ones). */
gp_status gp_grain_table(gp_ctx* ctx, int64_t cap, float* c3, int32_t* run, int64_t* n_out);

/* ---- stand-alone steps on caller device buffers ------------------------------ */

/* Device workspace bytes for gp_hash_build / gp_contact on n points. */
gp_status gp_hash_workspace_bytes(int64_t n, const gp_domain* domain, double h,
                                  size_t* out_bytes);

/* Spatial hash (Sec. 2.3 point partitioning): for n binary32 points x3 (device,
 * n x 3), cell key = (cz*ny + cy)*nx + cx with c_a = clamp(floor((x_a - lo_a) *
 * inv), 0, n_a - 1), lo_a = (float)domain.lo[a], cell edge e = h (1 + 2^-9),
 * inv = (float)(1/e), n_a = max(1, ceil((hi_a - lo_a)/e)), in binary32 without
 * contraction.  The edge margin makes any two points closer than h fall in
 * neighbouring cells despite binary32 rounding (up to 4096 cells per axis).
 * Writes the keys sorted stably (keys_sorted, n), the point ids in that order
 * (ids_sorted, n), the occupied cells (cell_keys) and the index of their first
 * point (cell_start); *n_cells (host) receives the number of occupied cells
 * (cell_keys and cell_start need n entries).  All arrays are device memory; the
 * call synchronises the stream to return *n_cells. */
gp_status gp_hash_build(const float* x3, int64_t n, const gp_domain* domain, double h,
                        uint32_t* keys_sorted, int32_t* ids_sorted, uint32_t* cell_keys,
                        int32_t* cell_start, int64_t* n_cells, void* workspace,
                        size_t workspace_bytes, void* cuda_stream);

/* Contact search (Sec. 2.1.2 impingement): freeze[i] = 1 iff state[i] == 0
 * (ACTIVE) and a point j with state[j] != 2 and grain[j] != grain[i] satisfies
 * ((dx*dx + dy*dy) + dz*dz) < hf*hf in binary32, hf = (float)h, d = x_i - x_j.
 * If pairs != NULL, the unordered pairs (i < j) of non-removed points of
 * different grains within that distance are written (2 int32 each, up to
 * pair_cap, in no particular order) and *n_pairs (host) receives their total
 * count.  Device arrays; synchronises the stream when pairs != NULL. */
gp_status gp_contact(const float* x3, const int32_t* grain, const uint8_t* state, int64_t n,
                     const gp_domain* domain, double h, uint8_t* freeze, int32_t* pairs,
                     int64_t pair_cap, int64_t* n_pairs, void* workspace,
                     size_t workspace_bytes, void* cuda_stream);

/* ---- failure detection --------------------------------------------------------- */

/* Self-test of the library's bounded device waits.  Every wait of the library gives
 * up after a limit of polls, sets a sticky device error bit and lets the kernel
 * return, so that a stalled producer shows up as GP_ERR_TIMEOUT on the host instead
 * of a hung GPU.  which = 0: the decoupled look-back of a radix-sort pass, waiting
 * for a preceding tile's status word; which = 1: a claim-table insert, waiting for
 * another warp to publish a block's pool slot.  The call allocates a 2 KB device
 * buffer, prepares in it a word that nothing ever publishes, runs that wait in one
 * thread with a limit of spin_limit polls (1 .. 4194304, the limit of the production
 * waits) and frees the buffer.  It returns GP_ERR_TIMEOUT when the wait gave up, as
 * it must; the device stays usable.  GP_ERR_ARG for other which or spin_limit.
 * The paper has no counterpart of this call (it describes no software). */
gp_status gp_selftest_wait(int32_t which, uint32_t spin_limit, void* cuda_stream);

/* ---- stand-alone hash without allocation ------------------------------------- */

/* Largest point count gp_hash_build_static accepts. */
#define GP_STATIC_SCRATCH_MAX_POINTS 262144

/* The spatial hash of gp_hash_build (same keys, order, cells and arguments, with
 * x3, keys_sorted, ids_sorted, cell_keys and cell_start in device memory), for
 * callers that can neither pass a workspace nor let the library allocate one:
 * for example a solver embedded in a host code whose device memory is owned and
 * budgeted by that code's own allocator, or a caller that must not pay the
 * device synchronisation of cudaMalloc.  The paper has no counterpart of this
 * call; it exists for such callers only.
 * Scratch comes from one static device array of the library (6,390,784 bytes,
 * about 6.4 MB), which every GPU that loads the library keeps until the process
 * exits.  The call allocates no device memory.
 *  - n > GP_STATIC_SCRATCH_MAX_POINTS returns GP_ERR_CAPACITY (nothing runs).
 *  - All calls on a device share the array and find what the previous call left
 *    there; the call clears the counters that must start at zero.  Calls whose
 *    device work can overlap (other streams, unordered host threads) race on the
 *    array and must be ordered by the caller.
 *  - The first call on a device looks up the array's device address with that
 *    device current and caches it; make that first call before any stream
 *    capture on the device.
 * Synchronises cuda_stream to return *n_cells. */
gp_status gp_hash_build_static(const float* x3, int64_t n, const gp_domain* domain, double h,
                               uint32_t* keys_sorted, int32_t* ids_sorted, uint32_t* cell_keys,
                               int32_t* cell_start, int64_t* n_cells, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GP_H */
