// Plain FP64 CPU oracle of the Lagrangian grain-envelope particle step
// (Mosbah et al., "A particle-based approach for the prediction of grain
// microstructures in solidification processes", arXiv 2504.12858).
//
// TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
// CUDA library.  Only the test suite, the smoke check and the CPU-baseline leg
// of the benchmark load it; the product path never does.  It shares no code,
// header, table or constant with the CUDA sources.
//
// It is written for a reader checking it against the paper: slow, sequential,
// standard containers, no blocking or fusion.  Each function names the passage
// it follows.  Where the paper is silent, the reading taken is stated in the
// comment beside the code that implements it.
//
// Notation (paper Sec. 2.1.2): a grain g has a nucleus c_g and a crystal->lab
// rotation R_g; its six <100> growth directions are d_k = R_g e_k with
// k = 0..5 for +x,-x,+y,-y,+z,-z.  Tracking points ("particles") sit on the
// grain's cubic lattice of spacing lambda_0 = h: a particle carries its last
// reached lattice site s (integer, crystal frame), its direction k and its
// progress ell in [0,1) towards the target site s + e_k, so that its position is
// x = c_g + h R_g (s + ell e_k).
//
// Parity mode: positions, cell keys and contact distances are FP64 in the
// dynamics.  The stand-alone hash / contact functions (go_hash_build_f32,
// go_contact_f32) evaluate the binning and contact predicates in IEEE binary32
// exactly as written (this file is compiled with -ffp-contract=off), because
// there a floating-point value decides an integer and both implementations
// must take that decision in the precision of the kernel.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

enum State : int { ACTIVE = 0, FROZEN = 1, REMOVED = 2 };

// progress tolerance of the reached-target test (reading r6): 2^-20 by default,
// settable (go_set_reach_tol) so that a pin can show it changes nothing on steps
// that are not commensurate with h
constexpr double kReachTolDefault = 1.0 / 1048576.0;

inline int axis_of(int k) { return k >> 1; }
inline int sign_of(int k) { return (k & 1) ? -1 : +1; }

struct Grain {
  double c[3];
  double R[9];      // row-major, crystal -> lab
  double dTn = 0;   // nucleation undercooling of its seed (0 for grains placed directly)
  int dormant = 0;  // melted entirely; its seed waits to nucleate again (reading r17)
};

struct Particle {
  int32_t grain;
  int32_t s[3];
  int32_t k;
  double ell;
  int32_t state;
};

struct SiteKey {
  int32_t g, x, y, z;
  bool operator==(const SiteKey& o) const {
    return g == o.g && x == o.x && y == o.y && z == o.z;
  }
  bool operator<(const SiteKey& o) const {
    if (g != o.g) return g < o.g;
    if (x != o.x) return x < o.x;
    if (y != o.y) return y < o.y;
    return z < o.z;
  }
};
struct SiteKeyHash {
  size_t operator()(const SiteKey& k) const {
    uint64_t a = (uint64_t)(uint32_t)k.g * 0x9E3779B97F4A7C15ull;
    a ^= (uint64_t)(uint32_t)k.x * 0xC2B2AE3D27D4EB4Full;
    a ^= (uint64_t)(uint32_t)k.y * 0x165667B19E3779F9ull;
    a ^= (uint64_t)(uint32_t)k.z * 0x27D4EB2F165667C5ull;
    return (size_t)(a ^ (a >> 29));
  }
};

struct Nucleus {
  double p[3];
  double dTn;
  double q[4];
  int done;
};

struct Stats {
  int64_t steps, particle_steps, n_frozen_new, n_spawned, n_claims_lost,
      n_clipped, n_clamped, n_nucleated, n_reached, n_melted, n_walkback;
};

// Unit quaternion (w,x,y,z) -> rotation matrix (crystal -> lab).  The paper gives
// orientations as Euler angles without a convention (Sec. 3.1, 3.3); the
// library interface takes quaternions (reading r10).
void quat_to_R(const double qin[4], double R[9]) {
  double n = std::sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] +
                       qin[3] * qin[3]);
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

// Sec. 2.1.2, Fig. 2: only "outer" points are generated, i.e. directions that
// increase the grain volume.  Reading r4: at lattice site s (relative to the
// nucleus) the direction sigma*e_a is outer iff s_a == 0 or sign(s_a) == sigma,
// i.e. iff it increases |s|_1.  This gives 6 directions at the nucleus, 5 at a
// vertex site, 4 at an edge site and 3 at a face site.
bool is_outer(const int32_t s[3], int k) {
  int a = axis_of(k), sg = sign_of(k);
  return s[a] == 0 || (s[a] > 0) == (sg > 0);
}

struct Sim {
  double lo[3], hi[3], h, dt;
  int nterms;
  double a[2], b[2], TL;
  int thermal_mode = 0;  // 0 none (T = TL), 1 analytic, 2 grid
  double T0 = 0, G[3] = {0, 0, 0}, xref[3] = {0, 0, 0}, Tdot = 0;
  std::vector<float> grid;
  int gn[3] = {0, 0, 0};
  double gorigin[3] = {0, 0, 0}, gspacing[3] = {1, 1, 1}, gvel[3] = {0, 0, 0};
  int64_t step = 0;
  double reach_tol = kReachTolDefault;
  bool melting = false;  // melting walk-back (Sec. 2.1.3), reading r17
  std::vector<Grain> grains;
  std::vector<Particle> parts;
  std::unordered_map<SiteKey, uint8_t, SiteKeyHash> claimed;
  std::vector<SiteKey> reached;
  std::vector<Nucleus> nuclei;
  Stats st{};

  void site_pos(int g, const int32_t s[3], double ell, int k, double x[3]) const {
    // x = c_g + h R_g (s + ell e_k)   (Sec. 2.1.2, tracking-point position)
    double u[3] = {(double)s[0], (double)s[1], (double)s[2]};
    if (ell != 0.0) u[axis_of(k)] += ell * sign_of(k);
    const Grain& G_ = grains[g];
    for (int r = 0; r < 3; ++r)
      x[r] = G_.c[r] + h * (G_.R[3 * r + 0] * u[0] + G_.R[3 * r + 1] * u[1] +
                            G_.R[3 * r + 2] * u[2]);
  }
  void part_pos(const Particle& p, double x[3]) const {
    site_pos(p.grain, p.s, p.ell, p.k, x);
  }

  // Composition-dependent liquidus T_L(w) = T_m + m_L w(x, t) with w trilinear on its
  // own moving grid (Sec. 2.1.3 notes that the nominal liquidus extends to a local
  // composition; Sec. 3.3/3.4 take the undercooling with respect to the local
  // solute concentration).  Unset: the nominal T_L of the growth law.
  bool solute = false;
  std::vector<float> wgrid;
  int wn[3] = {0, 0, 0};
  double worigin[3] = {0, 0, 0}, wspacing[3] = {1, 1, 1}, wvel[3] = {0, 0, 0};
  double Tm = 0, mL = 0;

  // Trilinear sample of a node-centred grid moving with velocity vel
  // (reading r14: replaces OpenFOAM's cellPointFace interpolation of Sec. 2.3).
  static double trilinear(const std::vector<float>& g, const int n[3], const double origin[3],
                          const double spacing[3], const double vel[3], const double x[3],
                          double t) {
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
      double u = (x[a] - vel[a] * t - origin[a]) / spacing[a];
      double umax = (double)(n[a] - 1);
      if (u < 0) u = 0;
      if (u > umax) u = umax;
      int i = (int)std::floor(u);
      if (i > n[a] - 2) i = n[a] - 2;
      i0[a] = i;
      f[a] = u - i;
    }
    auto at = [&](int i, int j, int k) {
      return (double)g[((size_t)k * n[1] + j) * n[0] + i];
    };
    double c[2][2];
    for (int dk = 0; dk < 2; ++dk)
      for (int dj = 0; dj < 2; ++dj) {
        double v0 = at(i0[0], i0[1] + dj, i0[2] + dk);
        double v1 = at(i0[0] + 1, i0[1] + dj, i0[2] + dk);
        c[dk][dj] = v0 + f[0] * (v1 - v0);
      }
    double e0 = c[0][0] + f[1] * (c[0][1] - c[0][0]);
    double e1 = c[1][0] + f[1] * (c[1][1] - c[1][0]);
    return e0 + f[2] * (e1 - e0);
  }
  double grid_T(const double x[3], double t) const {
    return trilinear(grid, gn, gorigin, gspacing, gvel, x, t);
  }
  double liquidus(const double x[3], double t) const {
    if (!solute) return TL;
    return Tm + mL * trilinear(wgrid, wn, worigin, wspacing, wvel, x, t);
  }

  // Total undercooling Delta T = T_L - T(x, t)  (Sec. 2.1.2, before Eq. 1), with the
  // local liquidus when a composition field is set.
  double undercooling(const double xin[3], double t) const {
    double x[3] = {xin[0], xin[1], xin[2]};
    wrap(x);  // fields are sampled at the position inside the domain
    const double tl = liquidus(x, t);
    if (thermal_mode == 1) {
      double T = T0 + G[0] * (x[0] - xref[0]) + G[1] * (x[1] - xref[1]) +
                 G[2] * (x[2] - xref[2]) + Tdot * t;
      return tl - T;
    }
    if (thermal_mode == 2) return tl - grid_T(x, t);
    return 0.0;
  }

  // Growth law, Eq. (1) (nterms = 1) or Eq. (2) (nterms = 2); zero velocity when
  // the melt is not undercooled (reading r9: no melting in the growth step).
  double velocity(double dT) const {
    if (!(dT > 0)) return 0.0;
    double v = 0;
    for (int i = 0; i < nterms; ++i) v += a[i] * std::pow(dT, b[i]);
    return v;
  }

  // Periodic axes (Sec. 3.4 applies periodic conditions on the faces normal to x
  // and y), reading r18: along a periodic axis a point is identified with its images
  // x + m L (L = hi - lo); positions are wrapped into [lo, hi), distances take the
  // nearest image, and nothing is clipped.  The lattice of a grain is unbounded, so
  // a grain crossing the face continues on the other side.
  int periodic = 0;  // bit a set: axis a is periodic
  bool per(int a_) const { return (periodic >> a_) & 1; }
  void wrap(double x[3]) const {
    for (int a_ = 0; a_ < 3; ++a_) {
      if (!per(a_)) continue;
      const double L = hi[a_] - lo[a_];
      double u = x[a_] - lo[a_];
      u -= L * std::floor(u / L);
      x[a_] = lo[a_] + u;
    }
  }
  double dist2(const double a[3], const double b[3]) const {
    double d2 = 0;
    for (int a_ = 0; a_ < 3; ++a_) {
      double d = a[a_] - b[a_];
      if (per(a_)) {
        const double L = hi[a_] - lo[a_];
        d -= L * std::round(d / L);
      }
      d2 += d * d;
    }
    return d2;
  }

  bool inside(const double x[3]) const {
    for (int a_ = 0; a_ < 3; ++a_)
      if (!per(a_) && !(x[a_] >= lo[a_] && x[a_] <= hi[a_])) return false;
    return true;
  }

  // Cell list in FP64.  The cell edge is the contact radius h enlarged by 2^-9
  // (reading r3), so two points closer than h always lie in neighbouring cells.
  // Along a periodic axis the period is divided into floor(L / edge) equal cells
  // (at least 3), each no narrower than that edge, and neighbours wrap around.
  // Returns the cell index triple, clamped to the domain grid.
  double cell_edge() const { return h * (1.0 + 1.0 / 512.0); }
  double edge(int a_, const int n[3]) const {
    return per(a_) ? (hi[a_] - lo[a_]) / n[a_] : cell_edge();
  }
  void cell_of(const double xin[3], int c[3], const int n[3]) const {
    double x[3] = {xin[0], xin[1], xin[2]};
    wrap(x);
    for (int a_ = 0; a_ < 3; ++a_) {
      int v = (int)std::floor((x[a_] - lo[a_]) / edge(a_, n));
      if (v < 0) v = 0;
      if (v > n[a_] - 1) v = n[a_] - 1;
      c[a_] = v;
    }
  }
  void ncells(int n[3]) const {
    for (int a_ = 0; a_ < 3; ++a_) {
      const double L = hi[a_] - lo[a_];
      int v = per(a_) ? (int)std::floor(L / cell_edge()) : (int)std::ceil(L / cell_edge());
      n[a_] = v < 1 ? 1 : v;
    }
  }
  // cell c + d along axis a: wrapped on a periodic axis, else -1 outside the grid
  int nb_cell(int c, int d, int a_, const int n[3]) const {
    int v = c + d;
    if (per(a_)) return (v + n[a_]) % n[a_];
    return (v < 0 || v >= n[a_]) ? -1 : v;
  }

  // Sec. 2.1.2 (impingement): "the advance of particles is naturally stopped when
  // two particles from different grains meet".  Reading r7: an ACTIVE particle
  // freezes when a live particle (ACTIVE or FROZEN) of another grain lies at a
  // distance < h.  Evaluated on the positions at t_n for all particles at once.
  std::vector<uint8_t> contact_f64(const std::vector<std::array<double, 3>>& X) const {
    int n[3];
    ncells(n);
    std::unordered_map<int64_t, std::vector<int64_t>> cells;
    std::vector<int64_t> keyv(parts.size());
    for (size_t i = 0; i < parts.size(); ++i) {
      if (parts[i].state == REMOVED) continue;
      int c[3];
      cell_of(X[i].data(), c, n);
      int64_t key = ((int64_t)c[2] * n[1] + c[1]) * n[0] + c[0];
      cells[key].push_back((int64_t)i);
    }
    std::vector<uint8_t> fr(parts.size(), 0);
    double rc2 = h * h;
    for (size_t i = 0; i < parts.size(); ++i) {
      if (parts[i].state != ACTIVE) continue;
      int c[3];
      cell_of(X[i].data(), c, n);
      bool hit = false;
      for (int dz = -1; dz <= 1 && !hit; ++dz)
        for (int dy = -1; dy <= 1 && !hit; ++dy)
          for (int dx = -1; dx <= 1 && !hit; ++dx) {
            int cx = nb_cell(c[0], dx, 0, n), cy = nb_cell(c[1], dy, 1, n),
                cz = nb_cell(c[2], dz, 2, n);
            if (cx < 0 || cy < 0 || cz < 0) continue;
            auto it = cells.find(((int64_t)cz * n[1] + cy) * n[0] + cx);
            if (it == cells.end()) continue;
            for (int64_t j : it->second) {
              if (parts[j].grain == parts[i].grain) continue;
              if (dist2(X[i].data(), X[j].data()) < rc2) {
                hit = true;
                break;
              }
            }
          }
      fr[i] = hit ? 1 : 0;
    }
    return fr;
  }

  bool is_claimed(const SiteKey& k) const { return claimed.count(k) != 0; }

  // Reading r12: a pending nucleation site is suppressed when a reached lattice
  // site of any grain lies within h of it (the site is inside a grain envelope).
  bool suppressed(const double p[3]) const {
    double rc2 = h * h;
    for (const SiteKey& r : reached) {
      int32_t s[3] = {r.x, r.y, r.z};
      double q[3];
      site_pos(r.g, s, 0.0, 0, q);
      if (dist2(p, q) < rc2) return true;
    }
    return false;
  }

  int32_t new_grain(const double p[3], const double q[4]) {
    Grain g;
    for (int a_ = 0; a_ < 3; ++a_) g.c[a_] = p[a_];
    quat_to_R(q, g.R);
    grains.push_back(g);
    return (int32_t)grains.size() - 1;
  }

  // Sec. 2.1.2, Step 0 of Fig. 2: upon nucleation six tracking points start at the
  // nucleus, one per <100> direction.  The nucleus site is reached and the six
  // first targets are claimed.
  void nucleate(int32_t g) {
    SiteKey k0{g, 0, 0, 0};
    reached.push_back(k0);
    claimed[k0] = 1;
    for (int k = 0; k < 6; ++k) {
      Particle p;
      p.grain = g;
      p.s[0] = p.s[1] = p.s[2] = 0;
      p.k = k;
      p.ell = 0.0;
      p.state = ACTIVE;
      int32_t t[3] = {0, 0, 0};
      t[axis_of(k)] += sign_of(k);
      claimed[SiteKey{g, t[0], t[1], t[2]}] = 1;
      parts.push_back(p);
    }
  }

  // Melting (Sec. 2.1.3): where the temperature rises above the liquidus the solid
  // melts, and the envelope is redefined by walking back to the tracking points at
  // the edge between undercooled and superheated melt.  Reading r17, at t_n before
  // the spatial hash:
  //  (M1) every reached site with Delta T < 0 at its position melts: it is no
  //       longer reached and no longer claimed;
  //  (M2) every live particle whose position has Delta T < 0, or whose site has
  //       melted, is removed, and its (never reached) target is released;
  //  (M3) walk-back: for every site melted in (M1), the first direction k = 0..5
  //       whose neighbour m - e_k is still reached gets a new ACTIVE particle at that
  //       neighbour heading k to the melted site, which it claims.  The surviving
  //       site and the melted one straddle the Delta T = 0 surface, closer to it than
  //       the paper's search distance of 2 lambda_0;
  //  (M4) a grain left without reached sites is melted entirely: its seed stays and
  //       nucleates again, with the same grain id, once its nucleation undercooling
  //       is reached and it lies in no grain (the nucleation pass below).
  void melt(double t) {
    std::vector<SiteKey> kept, melted;
    kept.reserve(reached.size());
    for (const SiteKey& r : reached) {
      int32_t sr[3] = {r.x, r.y, r.z};
      double q[3];
      site_pos(r.g, sr, 0.0, 0, q);
      if (undercooling(q, t) < 0) {
        melted.push_back(r);
        claimed.erase(r);
      } else {
        kept.push_back(r);
      }
    }
    reached.swap(kept);
    st.n_melted += (int64_t)melted.size();
    std::unordered_set<SiteKey, SiteKeyHash> alive(reached.begin(), reached.end());
    std::vector<Particle> out;
    out.reserve(parts.size());
    for (const Particle& p : parts) {
      double x[3];
      part_pos(p, x);
      if (undercooling(x, t) < 0 || !alive.count(SiteKey{p.grain, p.s[0], p.s[1], p.s[2]})) {
        SiteKey tk{p.grain, p.s[0], p.s[1], p.s[2]};
        if (axis_of(p.k) == 0) tk.x += sign_of(p.k);
        if (axis_of(p.k) == 1) tk.y += sign_of(p.k);
        if (axis_of(p.k) == 2) tk.z += sign_of(p.k);
        if (!alive.count(tk)) claimed.erase(tk);
        continue;
      }
      out.push_back(p);
    }
    for (const SiteKey& m : melted) {
      for (int k = 0; k < 6; ++k) {
        SiteKey nb = m;
        if (axis_of(k) == 0) nb.x -= sign_of(k);
        if (axis_of(k) == 1) nb.y -= sign_of(k);
        if (axis_of(k) == 2) nb.z -= sign_of(k);
        if (!alive.count(nb)) continue;
        Particle w;
        w.grain = m.g;
        w.s[0] = nb.x;
        w.s[1] = nb.y;
        w.s[2] = nb.z;
        w.k = k;
        w.ell = 0.0;
        w.state = ACTIVE;
        claimed[m] = 1;
        out.push_back(w);
        ++st.n_walkback;
        break;
      }
    }
    parts.swap(out);
    std::vector<int64_t> count(grains.size(), 0);
    for (const SiteKey& r : reached) ++count[r.g];
    for (const SiteKey& m : melted)
      if (count[m.g] == 0) grains[m.g].dormant = 1;
  }

  // One timestep n -> n+1, in the order fixed for this implementation:
  // [melting], hash + contact, sample, advance, spawn, clip, nucleate.
  void step_once() {
    const double t = (double)step * dt;
    if (melting) melt(t);
    const size_t N = parts.size();
    std::vector<std::array<double, 3>> X(N);
    for (size_t i = 0; i < N; ++i) part_pos(parts[i], X[i].data());

    // (1)-(2) spatial hash + impingement.
    std::vector<uint8_t> fr = contact_f64(X);

    // (3)-(5) thermal sample at (x_n, t_n), growth law, explicit Euler advance of
    // the progress ell (reading r2).  Reading r6: the progress made in one step is
    // capped at one lattice spacing, so a particle reaches at most one site per
    // step; the excess over the reached site is carried into its children.  The
    // target counts as reached once the progress is within 2^-20 of a full
    // spacing, so that a step commensurate with h (v dt = h/4, say) spawns on the
    // same step whatever the rounding of the accumulated progress.
    std::vector<uint8_t> cross(N, 0);
    std::vector<double> carry(N, 0.0);
    int64_t active_at_start = 0;
    for (size_t i = 0; i < N; ++i) {
      Particle& p = parts[i];
      if (p.state != ACTIVE) continue;
      ++active_at_start;
      if (fr[i]) {
        p.state = FROZEN;
        ++st.n_frozen_new;
        continue;
      }
      double dT = undercooling(X[i].data(), t);
      double v = velocity(dT);
      double dl = v * dt / h;
      if (dl > 1.0) {
        dl = 1.0;
        ++st.n_clamped;
      }
      double e = p.ell + dl;
      if (e >= 1.0 - reach_tol) {
        cross[i] = 1;
        carry[i] = e > 1.0 ? e - 1.0 : 0.0;
      } else {
        p.ell = e;
      }
    }
    st.particle_steps += active_at_start;

    // (6) spawning (Sec. 2.1.2, Fig. 2).  A particle that reached its target s'
    // generates one new point per outer direction k' at s', heading to
    // s' + e_k'.  Reading r5: each lattice site of a grain is claimed once.  A
    // target claimed in an earlier step is refused; among claimants of the same
    // step the one with the lowest direction index wins (at most one claimant per
    // axis can exist).  The parent itself is replaced by its children.
    std::unordered_map<SiteKey, int, SiteKeyHash> best;
    for (size_t i = 0; i < N; ++i) {
      if (!cross[i]) continue;
      const Particle& p = parts[i];
      int32_t sp[3] = {p.s[0], p.s[1], p.s[2]};
      sp[axis_of(p.k)] += sign_of(p.k);
      for (int k2 = 0; k2 < 6; ++k2) {
        if (!is_outer(sp, k2)) continue;
        SiteKey tk{p.grain, sp[0], sp[1], sp[2]};
        if (k2 >> 1 == 0) tk.x += sign_of(k2);
        if (k2 >> 1 == 1) tk.y += sign_of(k2);
        if (k2 >> 1 == 2) tk.z += sign_of(k2);
        if (is_claimed(tk)) continue;
        auto it = best.find(tk);
        if (it == best.end() || k2 < it->second) best[tk] = k2;
      }
    }

    std::vector<Particle> out;
    out.reserve(N + N / 2);
    std::vector<SiteKey> won;
    for (size_t i = 0; i < N; ++i) {
      const Particle& p = parts[i];
      if (p.state == REMOVED) continue;
      if (p.state == FROZEN) {
        out.push_back(p);
        continue;
      }
      if (!cross[i]) {
        // (7) domain clip (reading r8): a particle outside [lo, hi] is removed.
        double x[3];
        part_pos(p, x);
        if (inside(x))
          out.push_back(p);
        else
          ++st.n_clipped;
        continue;
      }
      int32_t sp[3] = {p.s[0], p.s[1], p.s[2]};
      sp[axis_of(p.k)] += sign_of(p.k);
      reached.push_back(SiteKey{p.grain, sp[0], sp[1], sp[2]});
      ++st.n_reached;
      for (int k2 = 0; k2 < 6; ++k2) {
        if (!is_outer(sp, k2)) continue;
        SiteKey tk{p.grain, sp[0], sp[1], sp[2]};
        if (k2 >> 1 == 0) tk.x += sign_of(k2);
        if (k2 >> 1 == 1) tk.y += sign_of(k2);
        if (k2 >> 1 == 2) tk.z += sign_of(k2);
        auto it = best.find(tk);
        bool win = (it != best.end() && it->second == k2);
        if (!win) {
          ++st.n_claims_lost;
          continue;
        }
        won.push_back(tk);
        Particle c;
        c.grain = p.grain;
        c.s[0] = sp[0];
        c.s[1] = sp[1];
        c.s[2] = sp[2];
        c.k = k2;
        c.ell = carry[i];
        c.state = ACTIVE;
        if (k2 != p.k) ++st.n_spawned;
        double x[3];
        part_pos(c, x);
        if (inside(x))
          out.push_back(c);
        else
          ++st.n_clipped;
      }
    }
    for (const SiteKey& k : won) claimed[k] = 1;
    parts.swap(out);

    // (8) nucleation at t_{n+1} (Sec. 2.1.1): a pending site activates once its
    // undercooling reaches its nucleation undercooling and it is not inside an
    // existing grain (reading r12).  All pending sites are tested against the
    // grains as they stand before this pass, then activated in list order.
    const double t1 = (double)(step + 1) * dt;
    std::vector<size_t> act;
    for (size_t j = 0; j < nuclei.size(); ++j) {
      Nucleus& nu = nuclei[j];
      if (nu.done) continue;
      if (undercooling(nu.p, t1) >= nu.dTn && !suppressed(nu.p)) act.push_back(j);
    }
    std::vector<int32_t> again;  // seeds of grains melted entirely (reading r17, M4)
    for (size_t g = 0; g < grains.size(); ++g)
      if (grains[g].dormant && undercooling(grains[g].c, t1) >= grains[g].dTn &&
          !suppressed(grains[g].c))
        again.push_back((int32_t)g);
    for (size_t j : act) {
      Nucleus& nu = nuclei[j];
      nu.done = 1;
      int32_t g = new_grain(nu.p, nu.q);
      grains[g].dTn = nu.dTn;
      nucleate(g);
      ++st.n_nucleated;
    }
    for (int32_t g : again) {
      grains[g].dormant = 0;
      nucleate(g);
      ++st.n_nucleated;
    }
    ++step;
    ++st.steps;
  }

  // Sec. 2.3 (Voronoi interpolation for rendering): the grain at a point is the
  // grain of the closest tracking information.  Reading r13: the closest reached
  // lattice site within h (ties to the smaller grain id), else -1 (liquid).
  int32_t grain_at(const double p[3],
                   const std::unordered_map<int64_t, std::vector<size_t>>& cells,
                   const int n[3], const std::vector<std::array<double, 3>>& RP) const {
    double rc2 = h * h;
    double pw[3] = {p[0], p[1], p[2]};
    wrap(pw);
    int c[3];
    for (int a_ = 0; a_ < 3; ++a_) c[a_] = (int)std::floor((pw[a_] - lo[a_]) / edge(a_, n));
    double best = rc2;
    int32_t bg = -1;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int d3[3] = {dx, dy, dz}, cc[3];
          for (int a_ = 0; a_ < 3; ++a_)
            cc[a_] = per(a_) ? (((c[a_] + d3[a_]) % n[a_]) + n[a_]) % n[a_]
                             : std::min(std::max(c[a_] + d3[a_], 0), n[a_] - 1);
          // clamping may visit a boundary cell more than once; harmless.
          auto it = cells.find(((int64_t)cc[2] * n[1] + cc[1]) * n[0] + cc[0]);
          if (it == cells.end()) continue;
          for (size_t r : it->second) {
            double d2 = dist2(pw, RP[r].data());
            int32_t g = reached[r].g;
            if (d2 >= rc2) continue;
            if (d2 < best || (d2 == best && g < bg)) {
              best = d2;
              bg = g;
            }
          }
        }
    return bg;
  }
};

// ---------- binary32 predicates for the stand-alone hash / contact functions ----
// Cell key (reading r3): with cell edge e = h (1 + 2^-9), lo_f = (float)lo,
// inv = (float)(1/e) and n_a = max(1, ceil((hi-lo)/e)), the cell index along an
// axis is clamp(floor((x - lo_f) * inv), 0, n_a - 1) evaluated in binary32, and
// the key is the linear index (cz * ny + cy) * nx + cx.  The 2^-9 margin exceeds
// the binary32 rounding of the cell coordinate for up to 4096 cells per axis, so
// any two points closer than h fall in neighbouring cells.
struct F32Grid {
  float lo[3];
  float inv;
  int n[3];
};
F32Grid make_f32grid(const double lo[3], const double hi[3], double h) {
  F32Grid g;
  const double e = h * (1.0 + 1.0 / 512.0);
  for (int a = 0; a < 3; ++a) {
    g.lo[a] = (float)lo[a];
    int v = (int)std::ceil((hi[a] - lo[a]) / e);
    g.n[a] = v < 1 ? 1 : v;
  }
  g.inv = (float)(1.0 / e);
  return g;
}
inline int f32cell(float x, float lo, float inv, int n) {
  float d = x - lo;
  float u = d * inv;
  int c = (int)std::floor(u);
  if (c < 0) c = 0;
  if (c > n - 1) c = n - 1;
  return c;
}
inline uint32_t f32key(const float* x, const F32Grid& g) {
  int cx = f32cell(x[0], g.lo[0], g.inv, g.n[0]);
  int cy = f32cell(x[1], g.lo[1], g.inv, g.n[1]);
  int cz = f32cell(x[2], g.lo[2], g.inv, g.n[2]);
  return (uint32_t)(((uint64_t)cz * g.n[1] + cy) * g.n[0] + cx);
}
// Contact distance (reading r3): d2 = ((dx*dx + dy*dy) + dz*dz) in binary32 with
// every product and sum rounded, compared strictly against hf*hf, hf = (float)h.
inline bool f32near(const float* a, const float* b, float rc2) {
  float dx = a[0] - b[0];
  float dy = a[1] - b[1];
  float dz = a[2] - b[2];
  float xx = dx * dx;
  float yy = dy * dy;
  float zz = dz * dz;
  float s = xx + yy;
  float d2 = s + zz;
  return d2 < rc2;
}

}  // namespace

extern "C" {

void* go_create(const double lo[3], const double hi[3], double h, double dt, int nterms,
                const double a[2], const double b[2], double TL) {
  Sim* S = new Sim();
  for (int i = 0; i < 3; ++i) {
    S->lo[i] = lo[i];
    S->hi[i] = hi[i];
  }
  S->h = h;
  S->dt = dt;
  S->nterms = nterms;
  for (int i = 0; i < 2; ++i) {
    S->a[i] = a[i];
    S->b[i] = b[i];
  }
  S->TL = TL;
  return S;
}

void go_destroy(void* s) { delete (Sim*)s; }

void go_set_thermal_analytic(void* s, double T0, const double G[3], const double xref[3],
                             double Tdot) {
  Sim* S = (Sim*)s;
  S->thermal_mode = 1;
  S->T0 = T0;
  for (int i = 0; i < 3; ++i) {
    S->G[i] = G[i];
    S->xref[i] = xref[i];
  }
  S->Tdot = Tdot;
}

// Composition field w (node-centred, x fastest, moving at vel) and the linear
// liquidus T_L(w) = T_m + m_L w.
void go_set_solute_grid(void* s, const float* w, const int32_t n[3], const double origin[3],
                        const double spacing[3], const double vel[3], double Tm, double mL) {
  Sim* S = (Sim*)s;
  S->solute = true;
  size_t tot = (size_t)n[0] * n[1] * n[2];
  S->wgrid.assign(w, w + tot);
  for (int i = 0; i < 3; ++i) {
    S->wn[i] = n[i];
    S->worigin[i] = origin[i];
    S->wspacing[i] = spacing[i];
    S->wvel[i] = vel[i];
  }
  S->Tm = Tm;
  S->mL = mL;
}

void go_set_thermal_grid(void* s, const float* T, const int32_t n[3], const double origin[3],
                         const double spacing[3], const double vel[3]) {
  Sim* S = (Sim*)s;
  S->thermal_mode = 2;
  size_t tot = (size_t)n[0] * n[1] * n[2];
  S->grid.assign(T, T + tot);
  for (int i = 0; i < 3; ++i) {
    S->gn[i] = n[i];
    S->gorigin[i] = origin[i];
    S->gspacing[i] = spacing[i];
    S->gvel[i] = vel[i];
  }
}

// Registers grains and, if nucleate != 0, starts each with its six nucleation
// points (Fig. 2, Step 0).  Returns the id of the first new grain.
int64_t go_add_grains(void* s, int64_t n, const double* pos3, const double* quat4,
                      int nucleate) {
  Sim* S = (Sim*)s;
  int64_t first = (int64_t)S->grains.size();
  for (int64_t i = 0; i < n; ++i) {
    int32_t g = S->new_grain(pos3 + 3 * i, quat4 + 4 * i);
    if (nucleate) S->nucleate(g);
  }
  return first;
}

// Seeds grain g with the state an isotropic envelope has after n0 complete lattice
// shells (Sec. 2.1.2, Fig. 2 repeated n0 times in a uniform melt): one particle
// per target site t with |t|_1 = n0 + 1, sitting at the parent site reached from
// the lowest axis a with t_a != 0 (the claimant that wins under reading r5), with
// progress ell0.  Sites with |s|_1 = n0 are recorded as reached (interior sites
// too if interior != 0); reached sites and the targets of the seeded particles are
// claimed.  Particles outside the domain are not seeded.
void go_seed_shell(void* s, int64_t ng, const int32_t* grains, int32_t n0, double ell0,
                   int interior) {
  Sim* S = (Sim*)s;
  int m = n0 + 1;
  for (int64_t gi = 0; gi < ng; ++gi) {
    int32_t g = grains[gi];
    for (int tx = -m; tx <= m; ++tx)
      for (int ty = -(m - std::abs(tx)); ty <= m - std::abs(tx); ++ty) {
        int rz = m - std::abs(tx) - std::abs(ty);
        for (int sgn = -1; sgn <= 1; sgn += 2) {
          if (rz == 0 && sgn > 0) continue;
          int tz = rz == 0 ? 0 : sgn * rz;
          int32_t t[3] = {tx, ty, tz};
          int a = t[0] != 0 ? 0 : (t[1] != 0 ? 1 : 2);
          int sg = t[a] > 0 ? 1 : -1;
          Particle p;
          p.grain = g;
          for (int q = 0; q < 3; ++q) p.s[q] = t[q];
          p.s[a] -= sg;
          p.k = 2 * a + (sg > 0 ? 0 : 1);
          p.ell = ell0;
          p.state = ACTIVE;
          double x[3];
          S->part_pos(p, x);
          if (!S->inside(x)) continue;
          S->parts.push_back(p);
          S->claimed[SiteKey{g, t[0], t[1], t[2]}] = 1;
        }
      }
    int lo_n = interior ? 0 : n0;
    for (int r = lo_n; r <= n0; ++r)
      for (int sx = -r; sx <= r; ++sx)
        for (int sy = -(r - std::abs(sx)); sy <= r - std::abs(sx); ++sy) {
          int rz = r - std::abs(sx) - std::abs(sy);
          for (int sgn = -1; sgn <= 1; sgn += 2) {
            if (rz == 0 && sgn > 0) continue;
            SiteKey k{g, sx, sy, rz == 0 ? 0 : sgn * rz};
            S->reached.push_back(k);
            S->claimed[k] = 1;
          }
        }
  }
}

void go_nucleation_sites(void* s, int64_t n, const double* pos3, const double* dTn,
                         const double* quat4) {
  Sim* S = (Sim*)s;
  for (int64_t i = 0; i < n; ++i) {
    Nucleus nu;
    for (int a = 0; a < 3; ++a) nu.p[a] = pos3[3 * i + a];
    nu.dTn = dTn[i];
    for (int a = 0; a < 4; ++a) nu.q[a] = quat4[4 * i + a];
    nu.done = 0;
    S->nuclei.push_back(nu);
  }
}

void go_step(void* s, int32_t nsteps) {
  Sim* S = (Sim*)s;
  for (int i = 0; i < nsteps; ++i) S->step_once();
}

int64_t go_num_particles(void* s) { return (int64_t)((Sim*)s)->parts.size(); }
int64_t go_num_grains(void* s) { return (int64_t)((Sim*)s)->grains.size(); }
int64_t go_get_step(void* s) { return ((Sim*)s)->step; }
void go_set_step(void* s, int64_t n) { ((Sim*)s)->step = n; }

void go_get_particles(void* s, int32_t* grain, int32_t* site3, int8_t* dir, double* ell,
                      uint8_t* state, double* x3) {
  Sim* S = (Sim*)s;
  for (size_t i = 0; i < S->parts.size(); ++i) {
    const Particle& p = S->parts[i];
    if (grain) grain[i] = p.grain;
    if (site3)
      for (int a = 0; a < 3; ++a) site3[3 * i + a] = p.s[a];
    if (dir) dir[i] = (int8_t)p.k;
    if (ell) ell[i] = p.ell;
    if (state) state[i] = (uint8_t)p.state;
    if (x3) S->part_pos(p, x3 + 3 * i);
  }
}

// Replaces the particle set (state import for single-step comparisons).
void go_load_particles(void* s, int64_t n, const int32_t* grain, const int32_t* site3,
                       const int8_t* dir, const double* ell, const uint8_t* state) {
  Sim* S = (Sim*)s;
  S->parts.clear();
  for (int64_t i = 0; i < n; ++i) {
    Particle p;
    p.grain = grain[i];
    for (int a = 0; a < 3; ++a) p.s[a] = site3[3 * i + a];
    p.k = dir[i];
    p.ell = ell[i];
    p.state = state[i];
    S->parts.push_back(p);
  }
}

int64_t go_num_reached(void* s) { return (int64_t)((Sim*)s)->reached.size(); }
void go_get_reached(void* s, int32_t* grain, int32_t* site3) {
  Sim* S = (Sim*)s;
  for (size_t i = 0; i < S->reached.size(); ++i) {
    grain[i] = S->reached[i].g;
    site3[3 * i + 0] = S->reached[i].x;
    site3[3 * i + 1] = S->reached[i].y;
    site3[3 * i + 2] = S->reached[i].z;
  }
}
void go_add_reached(void* s, int64_t n, const int32_t* grain, const int32_t* site3) {
  Sim* S = (Sim*)s;
  for (int64_t i = 0; i < n; ++i)
    S->reached.push_back(SiteKey{grain[i], site3[3 * i], site3[3 * i + 1], site3[3 * i + 2]});
}
int64_t go_num_claimed(void* s) { return (int64_t)((Sim*)s)->claimed.size(); }
// Claimed sites in lexicographic (grain, x, y, z) order.
void go_get_claimed(void* s, int32_t* grain, int32_t* site3) {
  Sim* S = (Sim*)s;
  std::vector<SiteKey> v;
  v.reserve(S->claimed.size());
  for (auto& kv : S->claimed) v.push_back(kv.first);
  std::sort(v.begin(), v.end());
  for (size_t i = 0; i < v.size(); ++i) {
    grain[i] = v[i].g;
    site3[3 * i + 0] = v[i].x;
    site3[3 * i + 1] = v[i].y;
    site3[3 * i + 2] = v[i].z;
  }
}
void go_add_claimed(void* s, int64_t n, const int32_t* grain, const int32_t* site3) {
  Sim* S = (Sim*)s;
  for (int64_t i = 0; i < n; ++i)
    S->claimed[SiteKey{grain[i], site3[3 * i], site3[3 * i + 1], site3[3 * i + 2]}] = 1;
}

// out[9]: steps, particle_steps, frozen (new), spawned, claims lost, clipped,
// clamped, nucleated, reached (new).
void go_get_stats(void* s, int64_t* out) {
  Sim* S = (Sim*)s;
  out[0] = S->st.steps;
  out[1] = S->st.particle_steps;
  out[2] = S->st.n_frozen_new;
  out[3] = S->st.n_spawned;
  out[4] = S->st.n_claims_lost;
  out[5] = S->st.n_clipped;
  out[6] = S->st.n_clamped;
  out[7] = S->st.n_nucleated;
  out[8] = S->st.n_reached;
  out[9] = S->st.n_melted;
  out[10] = S->st.n_walkback;
}

// Axes with periodic conditions: bit a set for axis a (reading r18).  A periodic
// axis needs at least three cells of the contact search along it.
void go_set_periodic(void* s, int axes) { ((Sim*)s)->periodic = axes & 7; }

// Tolerance of the reached-target test (reading r6): a particle whose progress
// reaches 1 - tol counts as having reached its target (carry max(0, ell - 1)).
void go_set_reach_tol(void* s, double tol) { ((Sim*)s)->reach_tol = tol; }

// Enables (1) or disables (0) the melting walk-back pass (reading r17).
void go_set_melting(void* s, int on) { ((Sim*)s)->melting = on != 0; }

void go_get_grain(void* s, int32_t g, double c[3], double R[9]) {
  Sim* S = (Sim*)s;
  for (int i = 0; i < 3; ++i) c[i] = S->grains[g].c[i];
  for (int i = 0; i < 9; ++i) R[i] = S->grains[g].R[i];
}

double go_undercooling(void* s, const double x[3], double t) {
  return ((Sim*)s)->undercooling(x, t);
}
double go_velocity(void* s, double dT) { return ((Sim*)s)->velocity(dT); }
int go_is_outer(const int32_t s3[3], int k) { return is_outer(s3, k) ? 1 : 0; }

// Grain-id map on a voxel grid of centres origin + (i + 1/2) * spacing (reading
// r13), x fastest.  Uses a cell list over the reached sites.
void go_grain_map(void* s, const double origin[3], const double spacing[3],
                  const int32_t nv[3], int32_t* out) {
  Sim* S = (Sim*)s;
  int n[3];
  S->ncells(n);
  std::vector<std::array<double, 3>> RP(S->reached.size());
  std::unordered_map<int64_t, std::vector<size_t>> cells;
  for (size_t r = 0; r < S->reached.size(); ++r) {
    int32_t st3[3] = {S->reached[r].x, S->reached[r].y, S->reached[r].z};
    S->site_pos(S->reached[r].g, st3, 0.0, 0, RP[r].data());
    int c[3];
    S->cell_of(RP[r].data(), c, n);
    cells[((int64_t)c[2] * n[1] + c[1]) * n[0] + c[0]].push_back(r);
  }
  for (int k = 0; k < nv[2]; ++k)
    for (int j = 0; j < nv[1]; ++j)
      for (int i = 0; i < nv[0]; ++i) {
        double p[3] = {origin[0] + (i + 0.5) * spacing[0], origin[1] + (j + 0.5) * spacing[1],
                       origin[2] + (k + 0.5) * spacing[2]};
        out[((size_t)k * nv[1] + j) * nv[0] + i] = S->grain_at(p, cells, n, RP);
      }
}

// Same map by exhaustive search over every reached site (pin for the above).
void go_grain_map_bruteforce(void* s, const double origin[3], const double spacing[3],
                             const int32_t nv[3], int32_t* out) {
  Sim* S = (Sim*)s;
  std::vector<std::array<double, 3>> RP(S->reached.size());
  for (size_t r = 0; r < S->reached.size(); ++r) {
    int32_t st3[3] = {S->reached[r].x, S->reached[r].y, S->reached[r].z};
    S->site_pos(S->reached[r].g, st3, 0.0, 0, RP[r].data());
  }
  double rc2 = S->h * S->h;
  for (int k = 0; k < nv[2]; ++k)
    for (int j = 0; j < nv[1]; ++j)
      for (int i = 0; i < nv[0]; ++i) {
        double p[3] = {origin[0] + (i + 0.5) * spacing[0], origin[1] + (j + 0.5) * spacing[1],
                       origin[2] + (k + 0.5) * spacing[2]};
        double best = rc2;
        int32_t bg = -1;
        for (size_t r = 0; r < RP.size(); ++r) {
          double d2 = S->dist2(p, RP[r].data());
          if (d2 >= rc2) continue;
          int32_t g = S->reached[r].g;
          if (d2 < best || (d2 == best && g < bg)) {
            best = d2;
            bg = g;
          }
        }
        out[((size_t)k * nv[1] + j) * nv[0] + i] = bg;
      }
}

// FP64 contact flags of the current particle set, by cell list and by exhaustive
// pair search (the latter is the pin of the former).
void go_contact_f64(void* s, uint8_t* freeze, int bruteforce) {
  Sim* S = (Sim*)s;
  size_t N = S->parts.size();
  std::vector<std::array<double, 3>> X(N);
  for (size_t i = 0; i < N; ++i) S->part_pos(S->parts[i], X[i].data());
  if (!bruteforce) {
    std::vector<uint8_t> fr = S->contact_f64(X);
    std::memcpy(freeze, fr.data(), N);
    return;
  }
  double rc2 = S->h * S->h;
  for (size_t i = 0; i < N; ++i) {
    freeze[i] = 0;
    if (S->parts[i].state != ACTIVE) continue;
    for (size_t j = 0; j < N; ++j) {
      if (S->parts[j].state == REMOVED || S->parts[j].grain == S->parts[i].grain) continue;
      if (S->dist2(X[i].data(), X[j].data()) < rc2) {
        freeze[i] = 1;
        break;
      }
    }
  }
}

// Stand-alone spatial hash of binary32 positions: cell keys, stable sort of
// (key, id) and the start of every occupied cell.  Returns the number of
// occupied cells.
int64_t go_hash_build_f32(const float* x3, int64_t n, const double lo[3], const double hi[3],
                          double h, uint32_t* keys_sorted, int32_t* ids_sorted,
                          uint32_t* cell_keys, int32_t* cell_start) {
  F32Grid g = make_f32grid(lo, hi, h);
  std::vector<std::pair<uint32_t, int32_t>> kv((size_t)n);
  for (int64_t i = 0; i < n; ++i) kv[i] = {f32key(x3 + 3 * i, g), (int32_t)i};
  std::stable_sort(kv.begin(), kv.end(),
                   [](const std::pair<uint32_t, int32_t>& A,
                      const std::pair<uint32_t, int32_t>& B) { return A.first < B.first; });
  int64_t nc = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (keys_sorted) keys_sorted[i] = kv[i].first;
    if (ids_sorted) ids_sorted[i] = kv[i].second;
    if (i == 0 || kv[i].first != kv[i - 1].first) {
      if (cell_keys) cell_keys[nc] = kv[i].first;
      if (cell_start) cell_start[nc] = (int32_t)i;
      ++nc;
    }
  }
  return nc;
}

void go_cell_keys_f32(const float* x3, int64_t n, const double lo[3], const double hi[3],
                      double h, uint32_t* keys) {
  F32Grid g = make_f32grid(lo, hi, h);
  for (int64_t i = 0; i < n; ++i) keys[i] = f32key(x3 + 3 * i, g);
}

// Stand-alone binary32 contact search over a cell list (cell edge h).  freeze[i]
// = 1 when i is ACTIVE (state 0) and a non-removed particle of another grain is
// within h.  If pairs != NULL, every unordered pair (i < j) of non-removed
// particles of different grains within h is listed (up to pair_cap), sorted.
// Returns the number of such pairs.
int64_t go_contact_f32(const float* x3, const int32_t* grain, const uint8_t* state, int64_t n,
                       const double lo[3], const double hi[3], double h, uint8_t* freeze,
                       int32_t* pairs, int64_t pair_cap) {
  F32Grid g = make_f32grid(lo, hi, h);
  float hf = (float)h;
  float rc2 = hf * hf;
  std::map<uint32_t, std::vector<int64_t>> cells;
  for (int64_t i = 0; i < n; ++i)
    if (state[i] != REMOVED) cells[f32key(x3 + 3 * i, g)].push_back(i);
  std::vector<std::pair<int32_t, int32_t>> pl;
  for (int64_t i = 0; i < n; ++i) {
    if (freeze) freeze[i] = 0;
    if (state[i] == REMOVED) continue;
    int c[3] = {f32cell(x3[3 * i], g.lo[0], g.inv, g.n[0]),
                f32cell(x3[3 * i + 1], g.lo[1], g.inv, g.n[1]),
                f32cell(x3[3 * i + 2], g.lo[2], g.inv, g.n[2])};
    bool hit = false;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int cx = c[0] + dx, cy = c[1] + dy, cz = c[2] + dz;
          if (cx < 0 || cy < 0 || cz < 0 || cx >= g.n[0] || cy >= g.n[1] || cz >= g.n[2])
            continue;
          auto it = cells.find((uint32_t)(((uint64_t)cz * g.n[1] + cy) * g.n[0] + cx));
          if (it == cells.end()) continue;
          for (int64_t j : it->second) {
            if (grain[j] == grain[i]) continue;
            if (!f32near(x3 + 3 * i, x3 + 3 * j, rc2)) continue;
            hit = true;
            if (j > i) pl.push_back({(int32_t)i, (int32_t)j});
          }
        }
    if (freeze && state[i] == ACTIVE && hit) freeze[i] = 1;
  }
  std::sort(pl.begin(), pl.end());
  if (pairs)
    for (size_t p = 0; p < pl.size() && (int64_t)p < pair_cap; ++p) {
      pairs[2 * p] = pl[p].first;
      pairs[2 * p + 1] = pl[p].second;
    }
  return (int64_t)pl.size();
}

// Exhaustive O(N^2) version of go_contact_f32 (pin for the cell-list search).
int64_t go_contact_bruteforce_f32(const float* x3, const int32_t* grain, const uint8_t* state,
                                  int64_t n, double h, uint8_t* freeze, int32_t* pairs,
                                  int64_t pair_cap) {
  float hf = (float)h;
  float rc2 = hf * hf;
  int64_t np = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (freeze) freeze[i] = 0;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (state[i] == REMOVED) continue;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i || state[j] == REMOVED || grain[j] == grain[i]) continue;
      if (!f32near(x3 + 3 * i, x3 + 3 * j, rc2)) continue;
      if (freeze && state[i] == ACTIVE) freeze[i] = 1;
      if (j > i) {
        if (pairs && np < pair_cap) {
          pairs[2 * np] = (int32_t)i;
          pairs[2 * np + 1] = (int32_t)j;
        }
        ++np;
      }
    }
  }
  return np;
}

}  // extern "C"
