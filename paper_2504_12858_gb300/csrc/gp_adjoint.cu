// Adjoint of the particle advance over a recorded tape (reverse sweep).
//
// Forward, per particle and step (Sec. 2.1.2, Eq. 1/2, explicit Euler):
//   dl    = v(dT) dt / h,  v = a0 dT^b0 (+ a1 dT^b1),  dT = dT_base(t) - G . (x - x_ref)
//   ell'  = ell + dl  (minus one in every child at a spawn)
//   x     = c + h R (s + ell e_k)
// with the discrete events (contact freeze, spawn, clip, the one-spacing cap, no
// growth for dT <= 0) held at their forward values.  Backward, for each particle
// of step n+1 with adjoint lambda and parent p at step n:
//   lambda_p += lambda (1 + d dl_p / d ell_p),   grad += lambda d dl_p / d theta
// where d dl / d ell = (dt/h) v'(dT) (-G . d x / d ell) and d x / d ell = sigma_k h R e_a.
#include <algorithm>

#include "gp_kernels.cuh"

namespace gp {

namespace {

// The tape holds, for every taped step n, in the order of the particle store
// (the order of gp_get_particles) at the start of that step:
//   post[i]  the state of particle i after the contact search of step n;
//   par[o]   for every particle o of step n+1, the store index at step n of the
//            particle it came from (itself, or the parent whose target it started
//            from; -1 for a particle from nucleation);
//   code[o]  its direction;
// and the records of the store at every checkpoint step.  The records at the other
// steps are rebuilt by replaying these events from the last checkpoint before them
// (k_adj_replay), with the forward's own arithmetic for the progress.

// post-contact state of every sorted particle j, stored at its store index src[j]
__global__ void k_tape_state(const int4* __restrict__ rs, const uint32_t* __restrict__ src,
                             int64_t n, uint8_t* __restrict__ out) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[__ldg(src + j)] = (uint8_t)rec_unpack(__ldg(rs + j)).state;
}

// after the step: parents by store index (the emit wrote sorted indices) and the
// direction of every particle of the new store (its count read on the device)
__global__ void k_tape_out(int32_t* __restrict__ par, const uint32_t* __restrict__ src,
                           const int4* __restrict__ rec, uint8_t* __restrict__ code,
                           const DevStats* st) {
  const int64_t m = (int64_t)st->n_live;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < m;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = par[o];
    if (p >= 0) par[o] = (int32_t)__ldg(src + p);
    code[o] = (uint8_t)rec_unpack(__ldg(rec + o)).dir;
  }
}

// Rebuilds the store of step n+1 (m particles) from that of step n and the taped
// events of step n: a particle that the contact search froze keeps its record with
// state FROZEN; an ACTIVE one advances by the forward's Euler step (euler_ell), and
// where it reached its target every particle it left starts at the reached site in its
// taped direction with the carried progress; a FROZEN one is unchanged.
__global__ void __launch_bounds__(256) k_adj_replay(Params P, StepArgs S,
                                                    const int4* __restrict__ rec,
                                                    const uint8_t* __restrict__ post,
                                                    const int32_t* __restrict__ par,
                                                    const uint8_t* __restrict__ code, int64_t m,
                                                    int4* __restrict__ out) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= m) return;
  const int32_t p = __ldg(par + o);
  if (p < 0) return;  // nucleated: not replayed (the tape refuses pending nuclei)
  Rec r = rec_unpack(__ldg(rec + p));
  if (r.state == ST_ACTIVE) {
    if (__ldg(post + p) != ST_ACTIVE) {
      r.state = ST_FROZEN;
    } else {
      float4 gc, r0, r1, r2;
      grain_load(P.gtab, r.grain, gc, r0, r1, r2);
      const float3 x =
          add_dir(site_pos_g(gc, r0, r1, r2, r.sx, r.sy, r.sz), r0, r1, r2, r.dir, r.ell);
      bool capped;
      const float e = euler_ell(P, P.geo, S, x, r.ell, capped);
      if (reaches_target(e)) {
        step_site(r.sx, r.sy, r.sz, r.dir);
        r.dir = __ldg(code + o);
        r.ell = fmaxf(__fsub_rn(e, 1.f), 0.f);
      } else {
        r.ell = e;
      }
    }
  }
  r.cross = 0;
  out[o] = rec_pack(r);
}

// One reverse step.  lam_u: adjoint of the particles of step n+1 by store index
// (m of them); par: their parent's store index at step n (-1: nucleated).
// rec / post: the store before the advance and the states after the contact search
// at step n, by store index.  Accumulates lam_s (store order, step n) and grad[8].
__global__ void __launch_bounds__(256) k_adj_step(Params P, StepArgs S, float t,
                                                  const int4* __restrict__ rec,
                                                  const uint8_t* __restrict__ post,
                                                  const int32_t* __restrict__ par,
                                                  const float* __restrict__ lam_u, int64_t m,
                                                  float* lam_s, double* grad) {
  __shared__ double s_g[8][8];
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float g8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (o < m) {
    const int32_t p = par[o];
    const float lam = lam_u[o];
    if (p >= 0 && lam != 0.f) {
      const Rec r = rec_unpack(__ldg(rec + p));
      float dldl = 0.f;
      if (r.state == ST_ACTIVE && post[p] == ST_ACTIVE) {
        float4 gc, r0, r1, r2;
        grain_load(P.gtab, r.grain, gc, r0, r1, r2);
        const float3 x =
            add_dir(site_pos_g(gc, r0, r1, r2, r.sx, r.sy, r.sz), r0, r1, r2, r.dir, r.ell);
        const float dT = undercooling(P, P.geo, S, x, P.geo.dT_base);
        if (dT > 0.f) {
          float v = 0.f, dv = 0.f;  // v(dT) and dv/d dT
          float pw[2] = {0.f, 0.f}, lg = logf(dT);
          for (int i = 0; i < P.nterms; ++i) {
            pw[i] = P.bint[i] > 0 ? ipow(dT, P.bint[i]) : powf(dT, P.b[i]);
            v += P.a[i] * pw[i];
            dv += P.a[i] * P.b[i] * pw[i] / dT;
          }
          const float k = P.dt_over_h;
          if (v * k <= 1.f) {  // not capped at one spacing
            // d x / d ell: sigma * column a of h R
            const int a = r.dir >> 1;
            const float sg = (r.dir & 1) ? -1.f : 1.f;
            const float cxl = sg * (a == 0 ? r0.x : (a == 1 ? r0.y : r0.z));
            const float cyl = sg * (a == 0 ? r1.x : (a == 1 ? r1.y : r1.z));
            const float czl = sg * (a == 0 ? r2.x : (a == 1 ? r2.y : r2.z));
            const float gdx = P.geo.G[0] * cxl + P.geo.G[1] * cyl + P.geo.G[2] * czl;
            dldl = -k * dv * gdx;
            for (int i = 0; i < P.nterms; ++i) {
              g8[2 * i] = lam * k * pw[i];                   // d/d a_i
              g8[2 * i + 1] = lam * k * P.a[i] * pw[i] * lg;  // d/d b_i
            }
            g8[4] = -lam * k * dv * (x.x - P.geo.xref[0]);       // d/d G
            g8[5] = -lam * k * dv * (x.y - P.geo.xref[1]);
            g8[6] = -lam * k * dv * (x.z - P.geo.xref[2]);
            g8[7] = -lam * k * dv * t;                      // d/d Tdot
          }
        }
      }
      atomicAdd(lam_s + p, lam * (1.f + dldl));
    }
  }
  // block reduction of the eight gradient terms in double
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    double v = g8[q];
#pragma unroll
    for (int of = 16; of > 0; of >>= 1) v += __shfl_xor_sync(0xffffffffu, v, of);
    if (lane == 0) s_g[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += s_g[w][threadIdx.x];
    if (v != 0.0) atomicAdd(grad + threadIdx.x, v);
  }
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

void launch_tape_state(const int4* rs, const uint32_t* src, int64_t n, uint8_t* out,
                       cudaStream_t st) {
  if (n > 0) k_tape_state<<<nblk(n), 256, 0, st>>>(rs, src, n, out);
}

void launch_tape_out(int32_t* par, const uint32_t* src, const int4* rec, uint8_t* code,
                     int64_t cap, const DevStats* dst, int sms, cudaStream_t st) {
  if (cap > 0)
    k_tape_out<<<(unsigned)std::min<int64_t>(nblk(cap), (int64_t)sms * 8), 256, 0, st>>>(
        par, src, rec, code, dst);
}

void launch_adj_replay(const Params& P, const StepArgs& S, const int4* rec, const uint8_t* post,
                       const int32_t* par, const uint8_t* code, int64_t m, int4* out,
                       cudaStream_t st) {
  if (m > 0) k_adj_replay<<<nblk(m), 256, 0, st>>>(P, S, rec, post, par, code, m, out);
}

void launch_adj_step(const Params& P, const StepArgs& S, float t, const int4* rec,
                     const uint8_t* post, const int32_t* par, const float* lam_u, int64_t m,
                     float* lam_s, double* grad, cudaStream_t st) {
  if (m > 0)
    k_adj_step<<<nblk(m), 256, 0, st>>>(P, S, t, rec, post, par, lam_u, m, lam_s, grad);
}

}  // namespace gp
