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
#include "gp_kernels.cuh"

namespace gp {

namespace {

// post-contact state of every sorted particle (byte per particle)
__global__ void k_tape_state(const int4* __restrict__ rs, int64_t n, uint8_t* __restrict__ out) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = (uint8_t)rec_unpack(__ldg(rs + j)).state;
}

// One reverse step.  lam_u: adjoint of the particles of step n+1 by store index
// (m of them); par: their parent's sorted index at step n (-1: nucleated).
// rec / post: sorted records before the advance and states after the contact
// search at step n.  Accumulates lam_s (sorted, step n) and grad[8].
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

// lam_u[vals[j]] = lam_s[j]: adjoint by store index from adjoint by sorted index
__global__ void k_adj_unsort(const float* __restrict__ lam_s, const uint32_t* __restrict__ vals,
                             int64_t n, float* __restrict__ lam_u) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) lam_u[vals[j]] = lam_s[j];
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

void launch_tape_state(const int4* rs, int64_t n, uint8_t* out, cudaStream_t st) {
  if (n > 0) k_tape_state<<<nblk(n), 256, 0, st>>>(rs, n, out);
}

void launch_adj_step(const Params& P, const StepArgs& S, float t, const int4* rec,
                     const uint8_t* post, const int32_t* par, const float* lam_u, int64_t m,
                     float* lam_s, double* grad, cudaStream_t st) {
  if (m > 0)
    k_adj_step<<<nblk(m), 256, 0, st>>>(P, S, t, rec, post, par, lam_u, m, lam_s, grad);
}

void launch_adj_unsort(const float* lam_s, const uint32_t* vals, int64_t n, float* lam_u,
                       cudaStream_t st) {
  if (n > 0) k_adj_unsort<<<nblk(n), 256, 0, st>>>(lam_s, vals, n, lam_u);
}

}  // namespace gp
