// Host launchers of the step kernels (defined in gp_kernels.cu).
#pragma once

#include "gp_internal.cuh"

namespace gp {

// batch == true: a context of several runs (uint64 cell keys); false: one run
// (uint32 cell keys)
void launch_keys(bool batch, const Params& P, const int4* rec, int64_t n, void* keys,
                 uint32_t* vals, cudaStream_t st);
// batch: the build after the radix sort; it lists the sorted indices of the ACTIVE
// particles in act (count in dst->n_act, which must be zero before the build), reads its
// counts and stamp from dst and uses a persistent grid.  The advance runs over that list.
void launch_build(const Params& P, const uint64_t* skeys, const uint32_t* svals, const int4* rin,
                  int4* rout, float4* pos4, uint4* tab, int64_t n, uint64_t key_end, uint32_t* act,
                  DevStats* dst, cudaStream_t st);
// one run: the records grouped by cell tile in place of the radix sort and build (keys:
// the emit's cell keys of the n records of rin).  rout receives the records in grouped
// order (gdest[i]: the position of grouped record i in the cell-ordered sequence; svals,
// if given, its store index; sact its state byte; act the ACTIVE ones, dst->n_act at the
// front and dst->n_actx at the back, both zero before the build); the sequence holds the
// moving records and the no obstacles of (okey, opos, group offsets ogofs): positions
// pos4, keys skeys, sources msrc, cell table tab.  obase != 0: okey and opos are entries
// obase.. of skeys and pos4, and a group without moving records is read there in place
// (its table entries point into the store; its places in the sequence hold no copy).
// rbuild (one tag per group), build and reuse: such a group that the previous build (tag
// build - 1) also wrote as resident keeps its table entries, restamped, when reuse says
// that the store and the table are those of the previous build
void launch_group_build(const Params& P, const uint32_t* keys, int64_t n, uint32_t ng,
                        uint32_t* gcnt, uint32_t* gofs, uint32_t* gbsum, uint32_t* gfill,
                        uint32_t* perm, uint32_t* gkey, uint32_t* gdest, const int4* rin,
                        int4* rout, float4* pos4, uint32_t* skeys, uint32_t* svals,
                        uint8_t* sact, uint4* tab, uint32_t stamp, uint32_t* act, DevStats* dst,
                        int sms, ProfHook* prof, cudaStream_t st, const uint32_t* okey = nullptr,
                        const float4* opos = nullptr, const uint32_t* ogofs = nullptr,
                        int64_t no = 0, uint32_t* msrc = nullptr, uint32_t obase = 0,
                        uint32_t* rbuild = nullptr, uint32_t build = 0, int reuse = 0);
// a batch: n records, sorted like pos4.  A single run: pos4, skeys and tab hold the n
// entries of the cell-ordered sequence (moving particles and obstacles), rs the nrec
// records in grouped order, mpos[j] the position of record j in the sequence.
void launch_advance(bool batch, const Params& P, const StepArgs& S, int4* rs, const float4* pos4,
                    const void* skeys, const uint4* tab, uint32_t stamp, int64_t n,
                    const uint32_t* act, const Claims& C, int32_t* site_slot, DevStats* dst,
                    cudaStream_t st, int64_t nrec = 0, const uint32_t* mpos = nullptr);
int64_t emit_tiles(int64_t n, int items);
void launch_link_reached(bool batch, const Params& P, const Reached& R,
                         unsigned long long* linked, int sms, cudaStream_t st);
void launch_emit(bool batch, const Params& P, const StepArgs& S, const int4* rs,
                 const int32_t* site_slot, int64_t n, int4* rout, void* keys, uint32_t* vals,
                 int64_t cap, const Claims& C, const Reached& R, int32_t* parent, DevStats* dst,
                 cudaStream_t st);
void launch_nucleate_batch(const Params& P, const StepArgs& S1, const float4* npos,
                           const int2* nmeta, int* nstate, int m, int4* rout, uint64_t* keys,
                           uint32_t* vals, int64_t cap, const Claims& C, const Reached& R,
                           DevStats* dst, int sms, cudaStream_t st);
// adjoint tape and reverse sweep (gp_adjoint.cu), in store order.  tape_state: the
// post-contact state of sorted particle j at its store index src[j]; tape_out (after
// the step): the emit's sorted parent indices to store indices and the direction of
// every particle of the new store; adj_replay: the store of step n+1 from that of
// step n and the taped events; adj_step: one reverse step
void launch_tape_state(const int4* rs, const uint32_t* src, int64_t n, uint8_t* out,
                       cudaStream_t st);
void launch_tape_out(int32_t* par, const uint32_t* src, const int4* rec, uint8_t* code,
                     int64_t cap, const DevStats* dst, int sms, cudaStream_t st);
void launch_adj_replay(const Params& P, const StepArgs& S, const int4* rec, const uint8_t* post,
                       const int32_t* par, const uint8_t* code, int64_t m, int4* out,
                       cudaStream_t st);
void launch_adj_step(const Params& P, const StepArgs& S, float t, const int4* rec,
                     const uint8_t* post, const int32_t* par, const float* lam_u, int64_t m,
                     float* lam_s, double* grad, cudaStream_t st);
void launch_nucleate(const Params& P, const StepArgs& S1, const float4* npos, const float4* ngrain,
                     int* nstate, int m, float4* gtab, int max_grains, int4* rout, uint32_t* keys,
                     uint32_t* vals, int64_t cap, const Claims& C, const Reached& R, DevStats* dst,
                     float* gdtn, cudaStream_t st);
// melting walk-back pass at t_n (single run): melts superheated reached sites,
// removes particles in the melt, re-activates the walk-back particles, compacts the
// store from rec into rtmp (the caller swaps them), marks fully melted grains
void launch_melt(const Params& P, const StepArgs& S, const Reached& R, const Claims& C,
                 unsigned long long* mlist, int64_t mcap, uint8_t* gflags, int ng, int4* rec,
                 int4* rtmp, int64_t n, int64_t cap, DevStats* dst, int sms, cudaStream_t st);
void launch_dormant_test(const Params& P, const StepArgs& S1, const Reached& R, const float* gdtn,
                         uint8_t* gflags, int ng, cudaStream_t st);
void launch_renucleate(const Params& P, uint8_t* gflags, int ng, int4* rout, uint32_t* keys,
                       uint32_t* vals, int64_t cap, const Claims& C, const Reached& R,
                       DevStats* dst, cudaStream_t st);
void launch_finalize(DevStats* dst, int64_t cap, bool batch, cudaStream_t st);
void launch_run_step(Geo* runs, const double2* th, int nruns, const DevStats* dst, double dt,
                     cudaStream_t st);
void launch_run_counts(const Params& P, const int4* rec, int64_t n, int nruns,
                       unsigned long long* counts, cudaStream_t st);
void launch_append(const int4* src, int64_t m, int4* rout, int64_t base, cudaStream_t st);
void launch_mark_sites(const Params& P, const int4* sites, int64_t m, int reached, int claimed,
                       const Claims& C, const Reached& R, cudaStream_t st);
// inserts m claim blocks (keys, kBrickWords words each) into an empty claim table
void launch_claim_restore(const Claims& C, const unsigned long long* keys, const uint32_t* words,
                          int64_t m, cudaStream_t st);
void launch_seed_shell(const Params& P, const int32_t* grains, int64_t ng, const short4* toff,
                       int64_t nt, float ell0, int4* rout, int64_t cap,
                       unsigned long long* counter, const Claims& C, uint32_t* err,
                       cudaStream_t st);
void launch_seed_shell_sites(const Params& P, const int32_t* grains, int64_t ng,
                             const short4* soff, int64_t ns, const Claims& C, const Reached& R,
                             cudaStream_t st);
void launch_positions(const Params& P, const int4* rec, int64_t n, float* x3, cudaStream_t st);
void launch_grain_map(bool batch, const Params& P, int run, const Reached& R, const double o[3],
                      const double s[3], const int nvox[3], int32_t* out, int64_t v0, int64_t nv,
                      cudaStream_t st);
void launch_keys_pos(const Params& P, const float* x3, const uint8_t* state, int64_t n,
                     uint32_t* keys, uint32_t* vals, cudaStream_t st);
void launch_cells(const uint32_t* skeys, int64_t n, uint32_t nvalid_key, uint32_t* flags,
                  uint32_t* ofs, uint32_t* bsum, uint32_t* cell_keys, int32_t* cell_start,
                  unsigned long long* ncell, cudaStream_t st);
void launch_build_sa(const Params& P, const float* x3, const int32_t* grain, const uint8_t* state,
                     const uint32_t* skeys, const uint32_t* svals, int64_t n, float4* pos4,
                     uint8_t* sstate, uint4* tab, uint32_t* err, cudaStream_t st);
void launch_contact_sa(const Params& P, const float4* pos4, const uint8_t* sstate,
                       const uint32_t* ids, const uint32_t* skeys, const uint4* tab,
                       int64_t n, uint8_t* freeze, int32_t* pairs, int64_t pair_cap,
                       unsigned long long* npairs, cudaStream_t st);

// obstacle flush of a single run (see gp_kernels.cu): the entries of the cell-ordered
// sequence (nseq of them: keys skeys, positions pos4, sources msrc) that are obstacles or
// FROZEN moving records become the new obstacle store (okey2, opos2, orec2; records from
// orec and from the grouped store rs, whose joining records are marked REMOVED); an
// obstacle's key and position come from the current store, entries obase.. of skeys and
// pos4; its size lands in dst->obs_new and the first obstacle of every group in
// ogofs2[0 .. ng].  tcnt holds obs_tiles(nseq) words.
int64_t obs_tiles(int64_t nseq);
void launch_obs_flush(const uint32_t* msrc, const uint32_t* skeys, const float4* pos4,
                      int64_t nseq, uint32_t* tcnt, const int4* orec, int4* rs, uint32_t* okey2,
                      float4* opos2, int4* orec2, uint32_t ng, uint32_t* ogofs2, DevStats* dst,
                      cudaStream_t st, int64_t obase);

// bounded-wait self-test: words holds 512 zeroed uint32 (a status array of two
// tiles, or one claim bucket), err one zeroed word
void launch_selftest_wait(int which, uint32_t limit, uint32_t* words, uint32_t* err,
                          cudaStream_t st);

}  // namespace gp
