"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
(the isotropic octahedron of Sec. 2.1.2 / Fig. 1, lattice counting), an
independent ODE integration (the single grain in a gradient of Sec. 3.1),
exhaustive searches (contacts, grain map), exact interpolation of linear fields,
or invariants (no interpenetration, hash ordering).  The orientation convention
is pinned separately against rotation matrices written out from their
definitions and against the quaternion sandwich product.  A plausible mistake in
the oracle (dropped term, wrong sign, wrong index, transposed or wrong-handed
rotation) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import Oracle
from paper_2504_12858_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def l1(v):
    return np.abs(v).sum(axis=-1)


def _uniform_sim(dT, a=(1e-5,), b=(2.0,), h=2e-6, dt=2e-3, half=200e-6, seed=1, n_grains=1,
                 centre=None):
    T_L = 1000.0
    lo, hi = (0.0, 0.0, 0.0), (2 * half,) * 3
    o = Oracle(lo, hi, h, dt, a, b, T_L)
    o.set_thermal_analytic(T_L - dT, (0, 0, 0), (0, 0, 0), 0.0)
    q = inputs.shoemake_quaternions(n_grains, inputs.rng(seed))
    c = np.array([[half, half, half]]) if centre is None else np.asarray(centre)
    o.add_grains(c, q)
    return o


# ----------------------------------------------------------------------------------
# Outer directions (Sec. 2.1.2): a direction is outer iff it increases the grain
# volume, i.e. moves the point away from the nucleus in the L1 sense.
# ----------------------------------------------------------------------------------
def test_outer_directions_match_volume_increase():
    g = inputs.rng(11)
    E = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
    for _ in range(500):
        s = g.integers(-4, 5, size=3)
        for k in range(6):
            assert oracle.is_outer(s, k) == (l1(s + E[k]) > l1(s))


@pytest.mark.parametrize("site,count", [((0, 0, 0), 6), ((3, 0, 0), 5), ((0, -2, 0), 5),
                                        ((2, -1, 0), 4), ((0, 1, 5), 4), ((1, 1, 1), 3),
                                        ((-2, 3, -1), 3)])
def test_outer_counts_by_site_class(site, count):
    # nucleus 6; fewer than six afterwards (Sec. 2.1.2): vertex 5, edge 4, face 3
    assert sum(oracle.is_outer(site, k) for k in range(6)) == count


# ----------------------------------------------------------------------------------
# Orientation convention (reading r10): a unit quaternion q = (w, x, y, z) maps the
# crystal frame to the lab frame, d_k = R(q) e_k, with the growth directions along the
# rotated <100> axes (Sec. 2.1.2).  Pinned against the elementary rotation matrices
# written out from their definitions, the Bunge Z-X-Z product of Sec. 3.1's Euler
# angles, and the quaternion sandwich product q (0, v) q*.
# ----------------------------------------------------------------------------------
def _rx(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def _ry(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def _rz(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _hamilton(p, q):
    w1, x1, y1, z1 = p
    w2, x2, y2, z2 = q
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 + y1 * w2 + z1 * x2 - x1 * z2,
                     w1 * z2 + z1 * w2 + x1 * y2 - y1 * x2])


def _oracle_R(quats):
    o = Oracle((0, 0, 0), (1e-4,) * 3, 2e-6, 1e-3, (1e-5,), (2.0,), 1000.0)
    quats = np.asarray(quats, np.float64).reshape(-1, 4)
    o.add_grains(np.full((len(quats), 3), 5e-5), quats, nucleate=False)
    return [o.grain(i)[1] for i in range(len(quats))]


@pytest.mark.parametrize("deg", [90.0, 30.0, -47.5, 180.0])
def test_rotation_about_each_axis_is_the_elementary_matrix(deg):
    t = math.radians(deg)
    c2, s2 = math.cos(t / 2), math.sin(t / 2)
    Rx, Ry, Rz = _oracle_R([[c2, s2, 0, 0], [c2, 0, s2, 0], [c2, 0, 0, s2]])
    assert np.allclose(Rx, _rx(t), atol=1e-15)
    assert np.allclose(Ry, _ry(t), atol=1e-15)
    assert np.allclose(Rz, _rz(t), atol=1e-15)
    # the crystal x axis turned about z lands at (cos t, sin t, 0): counter-clockwise
    assert np.allclose(Rz @ [1.0, 0.0, 0.0], [math.cos(t), math.sin(t), 0.0], atol=1e-15)


def test_rotation_of_bunge_euler_angles_is_the_zxz_product():
    # Sec. 3.1 gives the grain orientation as Euler angles (20, 20, 20) degrees; under
    # the Bunge convention crystal -> lab is Rz(psi) Rx(theta) Rz(phi)
    for ang in [(20.0, 20.0, 20.0), (4.0, 0.0, 0.0), (130.0, 75.0, -20.0)]:
        (R,) = _oracle_R(inputs.euler_zxz_to_quaternion(*ang))
        psi, th, phi = (math.radians(a) for a in ang)
        assert np.allclose(R, _rz(psi) @ _rx(th) @ _rz(phi), atol=1e-14)


def test_rotation_equals_quaternion_sandwich_and_is_proper():
    g = inputs.rng(21)
    q = inputs.shoemake_quaternions(40, g)
    scale = g.uniform(0.2, 5.0, size=(40, 1))        # the oracle normalises its input
    Rs = _oracle_R(q * scale)
    for qi, R in zip(q, Rs):
        qc = qi * np.array([1.0, -1.0, -1.0, -1.0])
        for v in np.eye(3):
            w = _hamilton(_hamilton(qi, np.concatenate([[0.0], v])), qc)
            assert abs(w[0]) < 1e-15
            assert np.allclose(R @ v, w[1:], atol=1e-14)
        assert np.allclose(R.T @ R, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)


def test_grown_tips_follow_the_closed_form_rotation():
    # 90 degrees about z: the crystal +x arm grows along lab +y and the crystal +y arm
    # along lab -x; the vertices sit at c + v t R e_a with R written out, not read back
    dT, h = 5.0, 2e-6
    v = 1e-5 * dT ** 2
    dt = 0.2718281828 * h / v
    c = np.array([60e-6, 60e-6, 60e-6])
    t = math.radians(90.0)
    for q, R in [((math.cos(t / 2), 0.0, 0.0, math.sin(t / 2)), _rz(t)),
                 (inputs.euler_zxz_to_quaternion(20.0, 20.0, 20.0),
                  _rz(math.radians(20)) @ _rx(math.radians(20)) @ _rz(math.radians(20)))]:
        T_L = 1000.0
        o = Oracle((0, 0, 0), (120e-6,) * 3, h, dt, (1e-5,), (2.0,), T_L)
        o.set_thermal_analytic(T_L - dT, (0, 0, 0), (0, 0, 0), 0.0)
        o.add_grains(c[None], np.asarray(q)[None])
        n = 50
        o.step(n)
        p = o.particles()
        for k in range(6):
            ax, sg = k // 2, (1 if k % 2 == 0 else -1)
            others = [a for a in range(3) if a != ax]
            m = ((p["dir"] == k) & (p["site"][:, ax] * sg >= 0)
                 & (p["site"][:, others] == 0).all(axis=1))
            assert m.sum() == 1
            assert np.allclose(p["x"][m][0], c + v * n * dt * sg * R[:, ax], rtol=0, atol=1e-15)
        if R is not None and np.allclose(R, _rz(t)):
            tip = p["x"][(p["dir"] == 0) & (p["site"][:, 1:] == 0).all(axis=1)
                         & (p["site"][:, 0] >= 0)][0]
            assert tip[1] - c[1] == pytest.approx(v * n * dt, rel=1e-12)
            assert abs(tip[0] - c[0]) < 1e-15


# ----------------------------------------------------------------------------------
# Reached-target tolerance (reading r6): a target counts as reached at progress
# 1 - 2^-20, so a step commensurate with h (v dt = h/4) spawns on the same step in
# binary32 and FP64.  The snap moves a particle by at most 2^-20 h, and only when
# its progress lands within 2^-20 of a full spacing; on steps that are not
# commensurate with h the tolerance changes nothing.
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("ratio,field", [(0.2718281828, "uniform"), (0.41421356237, "uniform"),
                                         (0.0, "gradient")])
def test_reach_tolerance_changes_nothing_off_commensurate_steps(ratio, field):
    def run(tol):
        if field == "uniform":
            dT, h = 5.0, 2e-6
            v = 1e-5 * dT ** 2
            o = _uniform_sim(dT, dt=ratio * h / v, half=60e-6)
            n = 90
            prog = np.arange(1, n + 1) * ratio
            assert np.min(np.abs(prog - np.round(prog))[prog > 0.5]) > 1e-4
        else:   # the single grain in the Sec. 3.1 gradient: progress varies continuously
            a, b, dT0, Tdot, G, h, T_L = 1e-4, 2.0, 2.0, -0.1, 250.0, 200e-6, 1000.0
            c = np.array([4e-3] * 3)
            o = Oracle((0, 0, 0), (8e-3,) * 3, h, 0.01, (a,), (b,), T_L)
            o.set_thermal_analytic(T_L - dT0, (0.0, 0.0, G), c, Tdot)
            o.add_grains(c[None], inputs.euler_zxz_to_quaternion(20.0, 20.0, 20.0)[None])
            n = 300
        if tol is not None:
            o.set_reach_tol(tol)
        o.step(n)
        return o.particles(), o.stats(), o.reached()
    p0, s0, r0 = run(None)
    p1, s1, r1 = run(0.0)
    assert s0 == s1
    for k in p0:
        assert np.array_equal(p0[k], p1[k]), k
    assert np.array_equal(r0[0], r1[0]) and np.array_equal(r0[1], r1[1])
    assert s0["reached"] > 100


def test_reach_tolerance_snap_is_bounded_on_commensurate_steps():
    # v dt = h/4 exactly: with the tolerance the spawns come every fourth step; without
    # it the FP64 sum of four quarters may stop short of 1 and lose a step.  Either
    # way the positions of the particles both runs share differ by at most 2^-20 h
    # per snap taken.
    dT, h = 5.0, 2e-6
    v = 1e-5 * dT ** 2
    o = _uniform_sim(dT, dt=0.25 * h / v, half=60e-6)
    o.step(40)
    p = o.particles()
    assert np.abs(p["ell"] - np.round(p["ell"] * 4) / 4).max() <= 40 * 2.0 ** -20


# ----------------------------------------------------------------------------------
# Isotropic octahedron (Sec. 2.1.2, Fig. 1): in a uniform undercooling the grain
# is an octahedron whose vertex distance is integral v dt, with v from Eq. (1) or
# Eq. (2).  Every tracking point lies on its surface |R^T (x - c)|_1 = v t.
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("a,b,dT", [
    ((1e-5,), (2.0,), 4.3),                           # Eq. (1), integer exponent
    ((8.26e-6, 8.18e-5), (2.0, 3.0), 1.7),            # Eq. (2), Sec. 3.3 coefficients
    ((8.315e-6, 9.628e-7), (2.49, 3.622), 3.1),       # Eq. (2), Sec. 4.1 coefficients
    ((1.834e-4,), (2.282,), 0.6),                     # Eq. (1), Sec. 3.4 coefficients
])
def test_octahedron_vertex_law(a, b, dT):
    v = sum(ai * dT ** bi for ai, bi in zip(a, b))
    h = 2e-6
    dt = 0.37 * h / v          # a non-commensurate step: no spawn-timing ties
    o = _uniform_sim(dT, a=a, b=b, h=h, dt=dt, half=60e-6)
    assert o.velocity(dT) == pytest.approx(v, rel=1e-14)
    c, R = o.grain(0)
    nsteps = 60
    o.step(nsteps)
    p = o.particles()
    assert (p["state"] == 0).all()
    r = (p["x"] - c) @ R          # crystal-frame coordinates (R^T (x - c))
    dist = v * nsteps * dt
    assert np.allclose(l1(r), dist, rtol=1e-11, atol=0)
    # the six vertices lie on the rotated <100> axes at distance v t
    vert = []
    for k in range(6):
        ax, sg = k // 2, (1 if k % 2 == 0 else -1)
        others = [q for q in range(3) if q != ax]
        m = ((p["dir"] == k) & ((p["site"][:, ax] * sg) >= 0)
             & (p["site"][:, others] == 0).all(axis=1))
        assert m.sum() == 1
        x = p["x"][m][0]
        vert.append(x)
        d = np.linalg.norm(x - c)
        assert d == pytest.approx(dist, rel=1e-11)
        assert np.allclose((x - c) / d, sg * R[:, ax], atol=1e-9)
    assert len(vert) == 6


def test_lattice_counts_uniform_growth():
    # Each lattice site of a grain is reached once; after m complete shells the
    # reached sites are exactly {s : |s|_1 <= m}: (2m+1)(2m^2+2m+3)/3 of them, and
    # one particle heads to each of the 4(m+1)^2 + 2 sites of the next shell.
    dT = 5.0
    v = 1e-5 * dT ** 2
    h = 2e-6
    dt = 0.2718281828 * h / v
    o = _uniform_sim(dT, dt=dt, half=100e-6)
    for n in range(1, 120):
        o.step(1)
        prog = n * v * dt / h
        frac = prog - math.floor(prog)
        assert min(frac, 1 - frac) > 1e-6
        m = int(math.floor(prog))
        g, s = o.reached()
        assert len(g) == (2 * m + 1) * (2 * m * m + 2 * m + 3) // 3
        assert l1(s).max() == m
        assert len({tuple(x) for x in s}) == len(g)
        assert o.n_particles == 4 * (m + 1) ** 2 + 2
        gc, sc = o.claimed()
        assert len(gc) == len(g) + 4 * (m + 1) ** 2 + 2
        shell = s[l1(s) == m]
        assert len(shell) == (4 * m * m + 2 if m > 0 else 1)


def test_shell_seeding_equals_grown_state():
    # A grain seeded as an n0-shell envelope equals the state a nucleus reaches in a
    # uniform melt (Fig. 2 repeated): same particles, sites, directions, progress.
    dT = 5.0
    v = 1e-5 * dT ** 2
    h = 2e-6
    dt = 0.2718281828 * h / v
    n = 40
    prog = n * v * dt / h
    n0, ell0 = int(math.floor(prog)), prog - math.floor(prog)
    grown = _uniform_sim(dT, dt=dt, half=100e-6)
    grown.step(n)
    pg = grown.particles()
    seeded = _uniform_sim(dT, dt=dt, half=100e-6)
    seeded.load_particles(np.zeros(0, np.int32), np.zeros((0, 3), np.int32),
                          np.zeros(0, np.int8), np.zeros(0), np.zeros(0, np.uint8))
    seeded.seed_shell([0], n0, ell0)
    ps = seeded.particles()

    def canon(p):
        key = np.lexsort((p["dir"], p["site"][:, 2], p["site"][:, 1], p["site"][:, 0]))
        return {k: v[key] for k, v in p.items()}

    a, b = canon(pg), canon(ps)
    assert np.array_equal(a["site"], b["site"])
    assert np.array_equal(a["dir"], b["dir"])
    assert np.allclose(a["ell"], b["ell"], atol=1e-12)
    assert np.allclose(a["x"], b["x"], atol=1e-15)
    # and it keeps growing identically
    grown.step(7)
    seeded.set_step(n)
    seeded.step(7)
    a, b = canon(grown.particles()), canon(seeded.particles())
    assert np.array_equal(a["site"], b["site"]) and np.array_equal(a["dir"], b["dir"])
    assert np.allclose(a["x"], b["x"], atol=1e-15)


# ----------------------------------------------------------------------------------
# Single grain in a gradient (Sec. 3.1, E1): each primary arm tip moves along its
# rotated <100> direction d with dr/dt = a dT(c + r d, t)^b, dT = dT0 - G (z - z_c)
# + |Tdot| t.  The oracle's explicit Euler tip must converge to the ODE solution
# (RK4, 2e4 substeps) at first order in dt.
# ----------------------------------------------------------------------------------
def _gradient_tips(dt, t_end=5.0):
    a, b = 1e-4, 2.0
    dT0, Tdot, G = 2.0, -0.1, 250.0
    h = 200e-6
    T_L = 1000.0
    half = 4e-3                 # tips travel about 2.6 mm in 5 s
    c = np.array([half, half, half])
    o = Oracle((0, 0, 0), (2 * half,) * 3, h, dt, (a,), (b,), T_L)
    o.set_thermal_analytic(T_L - dT0, (0.0, 0.0, G), c, Tdot)
    q = inputs.euler_zxz_to_quaternion(20.0, 20.0, 20.0)
    o.add_grains(c[None], q[None])
    n = int(round(t_end / dt))
    o.step(n)
    p = o.particles()
    cc, R = o.grain(0)
    tips = []
    for k in range(6):
        ax, sg = k // 2, (1 if k % 2 == 0 else -1)
        s = p["site"]
        others = [q for q in range(3) if q != ax]
        m = (p["dir"] == k) & (s[:, ax] * sg >= 0) & (s[:, others] == 0).all(axis=1)
        assert m.sum() == 1
        tips.append(np.linalg.norm(p["x"][m][0] - cc))
    return np.array(tips), R, (a, b, dT0, Tdot, G)


def _rk4_tip(dz, a, b, dT0, Tdot, G, t_end, nsub=20000):
    def f(t, r):
        dT = dT0 - G * dz * r - Tdot * t
        return a * dT ** b if dT > 0 else 0.0
    r, t = 0.0, 0.0
    hs = t_end / nsub
    for _ in range(nsub):
        k1 = f(t, r)
        k2 = f(t + hs / 2, r + hs / 2 * k1)
        k3 = f(t + hs / 2, r + hs / 2 * k2)
        k4 = f(t + hs, r + hs * k3)
        r += hs / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += hs
    return r


def test_gradient_single_grain_converges_to_ode():
    tips1, R, (a, b, dT0, Tdot, G) = _gradient_tips(0.01)
    tips2, _, _ = _gradient_tips(0.005)
    ref = np.array([_rk4_tip((1 if k % 2 == 0 else -1) * R[2, k // 2], a, b, dT0, Tdot, G, 5.0)
                    for k in range(6)])
    e1 = np.abs(tips1 - ref)
    e2 = np.abs(tips2 - ref)
    assert (e1 / ref).max() < 5e-3          # close at the paper's dt = 0.01 s
    ratio = e1 / e2
    assert ((ratio > 1.8) & (ratio < 2.2)).all(), ratio   # first order in dt
    # up-gradient arms (d_z > 0) grow less than down-gradient ones
    dz = np.array([(1 if k % 2 == 0 else -1) * R[2, k // 2] for k in range(6)])
    order = np.argsort(dz)
    assert np.all(np.diff(tips1[order]) < 0)


# ----------------------------------------------------------------------------------
# Local liquidus T_L(w) = T_m + m_L w(x) (Sec. 2.1.3 extends the nominal liquidus to
# the local composition; Sec. 3.3/3.4 take the undercooling with respect to the
# local solute concentration).  (1) A uniform composition at which T_m + m_L w is
# exactly the nominal T_L changes nothing.  (2) A composition linear in z with
# m_L dw/dz = -G under a uniform temperature is the thermal gradient G of the
# Sec. 3.1 case: the tips must coincide with that (RK4-pinned) case.
# ----------------------------------------------------------------------------------
def _w_grid_linear_z(w0, gw, zc, L=8e-3, nz=17):
    z = np.linspace(0.0, L, nz)
    w = (w0 + gw * (z - zc)).astype(np.float32)
    return np.broadcast_to(w[:, None, None], (nz, 2, 2)).copy(), (0.0, 0.0, 0.0), (L, L, L / (nz - 1))


def test_uniform_composition_at_nominal_liquidus_changes_nothing():
    T_L = 1000.0
    runs = []
    for solute in (False, True):
        o = Oracle((0, 0, 0), (60e-6,) * 3, 2e-6, 1.3e-3, (1e-5,), (2.0,), T_L)
        o.set_thermal_analytic(T_L - 4.0, (3e4, -2e4, 1e4), (30e-6,) * 3, -20.0)
        if solute:   # 1013 - 6.5 * 2 = 1000 exactly
            o.set_solute_grid(np.full((3, 3, 3), 2.0, np.float32), (0, 0, 0), (30e-6,) * 3,
                              1013.0, -6.5)
        g = inputs.rng(5)
        o.add_grains(g.random((8, 3)) * 60e-6, inputs.shoemake_quaternions(8, g))
        o.step(30)
        runs.append(o.particles())
    a, b = runs
    assert len(a["grain"]) == len(b["grain"]) > 400
    for k in ("grain", "site", "dir", "state"):
        assert np.array_equal(a[k], b[k])
    assert np.array_equal(a["x"], b["x"])


def test_solute_gradient_equals_thermal_gradient():
    a, b, dT0, Tdot, G, T_L, h, half = 1e-4, 2.0, 2.0, -0.1, 250.0, 1000.0, 200e-6, 4e-3
    c = np.array([half, half, half])
    q = inputs.euler_zxz_to_quaternion(20.0, 20.0, 20.0)
    tips = []
    for solute in (False, True):
        o = Oracle((0, 0, 0), (2 * half,) * 3, h, 0.01, (a,), (b,), T_L)
        if solute:   # T_L(z) = 1020 - 2 (10 + 125 (z - z_c)) = T_L - G (z - z_c)
            o.set_thermal_analytic(T_L - dT0, (0.0, 0.0, 0.0), c, Tdot)
            w, org, sp = _w_grid_linear_z(10.0, 125.0, half)
            o.set_solute_grid(w, org, sp, T_L + 20.0, -2.0)
        else:
            o.set_thermal_analytic(T_L - dT0, (0.0, 0.0, G), c, Tdot)
        o.add_grains(c[None], q[None])
        o.step(500)
        p = o.particles()
        cc, R = o.grain(0)
        t = []
        for k in range(6):
            ax, sg = k // 2, (1 if k % 2 == 0 else -1)
            others = [i for i in range(3) if i != ax]
            m = ((p["dir"] == k) & (p["site"][:, ax] * sg >= 0)
                 & (p["site"][:, others] == 0).all(axis=1))
            assert m.sum() == 1
            t.append(np.linalg.norm(p["x"][m][0] - cc))
        tips.append(np.array(t))
        assert o.undercooling(c + np.array([0, 0, 1e-3]), 1.0) == pytest.approx(
            dT0 - G * 1e-3 + 0.1, rel=1e-12)
    assert np.allclose(tips[0], tips[1], rtol=1e-10, atol=0)


# ----------------------------------------------------------------------------------
# Trilinear sampling: exact on a field that is linear in x, y, z; moving frame.
# ----------------------------------------------------------------------------------
def test_trilinear_grid_exact_on_linear_field():
    nx, ny, nz = 9, 7, 5
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    T = (1000.0 + 2.0 * i + 3.0 * j - 5.0 * k).astype(np.float32)
    sp = np.array([1e-6, 2e-6, 3e-6])
    origin = np.array([1e-6, -2e-6, 5e-6])
    vel = np.array([0.01, 0.0, -0.02])
    o = Oracle((0, 0, 0), (1e-4,) * 3, 1e-6, 1e-3, (1.0,), (2.0,), 1010.0)
    o.set_thermal_grid(T, origin, sp, vel)
    g = inputs.rng(5)
    for _ in range(200):
        t = g.uniform(0, 1e-3)
        u = g.uniform([0, 0, 0], [nx - 1, ny - 1, nz - 1])
        x = origin + vel * t + u * sp
        expect = 1010.0 - (1000.0 + 2 * u[0] + 3 * u[1] - 5 * u[2])
        assert o.undercooling(x, t) == pytest.approx(expect, abs=1e-9)
    # clamped outside the table (edge value continues)
    x = origin + np.array([-5.0, 0.0, 0.0]) * sp
    assert o.undercooling(x, 0.0) == pytest.approx(1010.0 - 1000.0, abs=1e-9)


def test_analytic_field_and_growth_law_zero_when_superheated():
    o = Oracle((0, 0, 0), (1e-3,) * 3, 2e-6, 1e-3, (1e-5,), (2.0,), 1000.0)
    o.set_thermal_analytic(990.0, (10.0, -20.0, 30.0), (1e-4, 2e-4, 3e-4), -7.0)
    x = np.array([3e-4, 1e-4, 5e-4])
    t = 0.25
    T = 990.0 + 10 * 2e-4 - 20 * (-1e-4) + 30 * 2e-4 - 7 * t
    assert o.undercooling(x, t) == pytest.approx(1000.0 - T, abs=1e-12)
    assert o.velocity(-1.0) == 0.0 and o.velocity(0.0) == 0.0
    assert o.velocity(3.0) == pytest.approx(9e-5, rel=1e-14)


# ----------------------------------------------------------------------------------
# Contacts (Sec. 2.1.2 impingement): the cell-list search equals exhaustive search,
# in binary32 (stand-alone reference) and in FP64 (the dynamics).
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("n,ng,seed", [(1, 1, 0), (2, 2, 1), (300, 3, 2), (1500, 7, 3),
                                       (2000, 40, 4)])
def test_contact_f32_cell_list_equals_bruteforce(n, ng, seed):
    g = inputs.rng(seed)
    h = 2e-6
    lo, hi = np.zeros(3), np.array([30e-6, 20e-6, 10e-6])
    x = (g.random((n, 3)) * hi).astype(np.float32)
    grain = g.integers(0, ng, n).astype(np.int32)
    state = g.choice(np.array([0, 0, 0, 1, 2], np.uint8), n)
    fr1, p1 = oracle.contact_f32(x, grain, state, lo, hi, h, want_pairs=True)
    fr2, p2 = oracle.contact_f32(x, grain, state, lo, hi, h, want_pairs=True, bruteforce=True)
    assert np.array_equal(fr1, fr2)
    assert np.array_equal(p1, p2)
    if n > 100:
        assert fr1.sum() > 0 and (fr1 <= (state == 0)).all()


def test_contact_f64_cell_list_equals_bruteforce_in_a_polycrystal():
    h, dt = 2e-6, 2e-3
    T_L = 1000.0
    o = Oracle((0, 0, 0), (60e-6,) * 3, h, dt, (1e-5,), (2.0,), T_L)
    o.set_thermal_analytic(T_L - 5.0, (0, 0, 0), (0, 0, 0), 0.0)
    g = inputs.rng(9)
    o.add_grains(g.random((6, 3)) * 60e-6, inputs.shoemake_quaternions(6, g))
    for _ in range(12):
        o.step(5)
        assert np.array_equal(o.contact_flags(), o.contact_flags(bruteforce=True))
    assert (o.particles()["state"] == 1).sum() > 0


def test_grains_never_interpenetrate():
    # After every step no particle of one grain is closer to a particle of another
    # grain than h - 2 v_max dt (the contact radius minus what two particles can
    # cover in one step).
    h, dT = 2e-6, 5.0
    v = 1e-5 * dT ** 2
    dt = 0.3 * h / v
    T_L = 1000.0
    o = Oracle((0, 0, 0), (80e-6, 60e-6, 60e-6), h, dt, (1e-5,), (2.0,), T_L)
    o.set_thermal_analytic(T_L - dT, (0, 0, 0), (0, 0, 0), 0.0)
    g = inputs.rng(21)
    centres = np.array([[25e-6, 30e-6, 30e-6], [55e-6, 30e-6, 30e-6], [40e-6, 50e-6, 20e-6]])
    o.add_grains(centres, inputs.shoemake_quaternions(3, g))
    gap = h - 2 * v * dt
    for _ in range(60):
        o.step(1)
        p = o.particles()
        x, gr = p["x"], p["grain"]
        d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)
        other = gr[:, None] != gr[None, :]
        assert (d2[other] >= gap * gap * (1 - 1e-12)).all()
    assert (p["state"] == 1).sum() > 10


# ----------------------------------------------------------------------------------
# Spatial hash (binary32): ordering properties and cell geometry.
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [0, 1, 7, 5000])
def test_hash_f32_properties(n):
    g = inputs.rng(30 + n)
    h = 2e-6
    lo, hi = np.array([1e-6, -3e-6, 0.0]), np.array([41e-6, 17e-6, 9e-6])
    x = (lo + g.random((n, 3)) * (hi - lo)).astype(np.float32)
    if n > 10:
        x[:10] = x[10:20]         # duplicates exercise stability
    ks, ids, ck, cs = oracle.hash_build_f32(x, lo, hi, h)
    e = h * (1 + 1 / 512)
    nx = [max(1, math.ceil((hi[a] - lo[a]) / e)) for a in range(3)]
    assert sorted(ids.tolist()) == list(range(n))
    assert np.all(np.diff(ks.astype(np.int64)) >= 0)
    same = np.diff(ks.astype(np.int64)) == 0
    assert np.all(np.diff(ids)[same] > 0)          # stable
    keys = oracle.cell_keys_f32(x, lo, hi, h)
    assert np.array_equal(keys[ids], ks)
    # the cell of each point contains it (up to binary32 rounding at a cell face)
    cx = keys % nx[0]
    cy = (keys // nx[0]) % nx[1]
    cz = keys // (nx[0] * nx[1])
    cell = np.stack([cx, cy, cz], 1).astype(np.float64)
    u = (x.astype(np.float64) - lo) / e
    assert (u >= cell - 1e-4).all() and (u < cell + 1 + 1e-4).all()
    # cell starts
    assert len(ck) == len(np.unique(ks))
    if n:
        assert cs[0] == 0 and np.array_equal(ks[cs], ck)


# ----------------------------------------------------------------------------------
# Clip and step cap.
# ----------------------------------------------------------------------------------
def test_domain_clip_removes_points_leaving_the_box():
    dT = 5.0
    v = 1e-5 * dT ** 2
    h = 2e-6
    dt = 0.37 * h / v
    o = _uniform_sim(dT, dt=dt, half=10e-6, seed=3)
    c, R = o.grain(0)
    for n in range(1, 80):
        o.step(1)
        p = o.particles()
        assert ((p["x"] >= 0) & (p["x"] <= 20e-6)).all()
    assert o.stats()["clipped"] > 0
    # the vertex closest to a wall leaves when its distance exceeds the wall distance
    assert o.n_particles < 4 * 30 ** 2


def test_progress_capped_at_one_site_per_step():
    dT = 1000.0                              # v dt / h = 2500: capped at 1
    o = _uniform_sim(dT, half=60e-6)
    c, R = o.grain(0)
    o.step(9)
    p = o.particles()
    r = (p["x"] - c) @ R
    assert np.allclose(l1(r), 9 * 2e-6, rtol=1e-12)
    st = o.stats()
    assert st["clamped"] == st["particle_steps"]


# ----------------------------------------------------------------------------------
# Nucleation (Sec. 2.1.1): activation step and suppression inside grains.
# ----------------------------------------------------------------------------------
def test_nucleation_activation_time_and_suppression():
    h, dt = 2e-6, 1e-3
    T_L = 1000.0
    Tdot = -10.0                 # cooling: dT grows by 0.01 K per step
    G = 1e3
    o = Oracle((0, 0, 0), (200e-6,) * 3, h, dt, (1e-5,), (2.0,), T_L)
    o.set_thermal_analytic(T_L, (0.0, 0.0, G), (0, 0, 0), Tdot)
    pos = np.array([[50e-6, 50e-6, 10e-6],     # dT(t) = 0.01 n - 0.01
                    [150e-6, 150e-6, 100e-6],  # dT(t) = 0.01 n - 0.1
                    [50e-6, 50e-6, 11e-6]])    # inside the first grain once it grows
    dTn = np.array([0.0555, 0.1234, 0.5])
    q = inputs.shoemake_quaternions(3, inputs.rng(4))
    o.nucleation_sites(pos, dTn, q)
    act = {}
    for n in range(400):
        before = o.n_grains
        o.step(1)
        for gidx in range(before, o.n_grains):
            c, _ = o.grain(gidx)
            act[int(np.argmin(np.linalg.norm(pos - c, axis=1)))] = n
    # site j activates at the first step n whose end time t_{n+1} has dT >= dTn
    for j, dT0 in ((0, -G * pos[0, 2]), (1, -G * pos[1, 2])):
        n_expect = math.ceil((dTn[j] - dT0) / (-Tdot * dt)) - 1
        assert act[j] == n_expect
    assert 2 not in act                        # suppressed: inside grain 0
    assert o.stats()["nucleated"] == 2


# ----------------------------------------------------------------------------------
# Grain map (Sec. 2.3 Voronoi interpolation): cell-list search equals exhaustive
# search, and a single grain maps to its octahedron.
# ----------------------------------------------------------------------------------
def test_grain_map_equals_bruteforce_and_octahedron():
    h, dT = 2e-6, 5.0
    v = 1e-5 * dT ** 2
    dt = 0.31 * h / v
    T_L = 1000.0
    o = Oracle((0, 0, 0), (50e-6,) * 3, h, dt, (1e-5,), (2.0,), T_L)
    o.set_thermal_analytic(T_L - dT, (0, 0, 0), (0, 0, 0), 0.0)
    g = inputs.rng(8)
    o.add_grains(np.array([[18e-6, 25e-6, 25e-6], [34e-6, 22e-6, 27e-6]]),
                 inputs.shoemake_quaternions(2, g))
    o.step(30)
    nv = (25, 25, 25)
    sp = (2e-6, 2e-6, 2e-6)
    m1 = o.grain_map((0, 0, 0), sp, nv)
    m2 = o.grain_map((0, 0, 0), sp, nv, bruteforce=True)
    assert np.array_equal(m1, m2)
    assert (m1 == 0).sum() > 100 and (m1 == 1).sum() > 100 and (m1 == -1).sum() > 100

    o1 = _uniform_sim(dT, dt=dt, half=30e-6, seed=12)
    o1.step(40)
    c, R = o1.grain(0)
    nvox = (30, 30, 30)
    mp = o1.grain_map((0, 0, 0), sp, nvox)
    k, j, i = np.meshgrid(*[np.arange(nn) for nn in nvox[::-1]], indexing="ij")
    centres = np.stack([(i + 0.5) * sp[0], (j + 0.5) * sp[1], (k + 0.5) * sp[2]], -1)
    r = l1((centres - c) @ R) / h
    m = int(math.floor(40 * v * dt / h))
    assert (mp[r <= m - 1.0] == 0).all()
    assert (mp[r >= m + 2.0] == -1).all()


def test_commensurate_step_spawns_on_schedule():
    # v dt = h / 4 exactly (the 200 um single-grain configuration): the target is
    # reached every fourth step, so after 4k steps exactly the k-ball of sites is
    # reached, whatever the rounding of the accumulated progress.
    o = _uniform_sim(5.0, half=100e-6)          # A = 1e-5, dT = 5 K, dt = 2 ms, h = 2 um
    for k in range(1, 16):
        o.step(4)
        g, _ = o.reached()
        assert len(g) == (2 * k + 1) * (2 * k * k + 2 * k + 3) // 3
        assert o.n_particles == 4 * (k + 1) ** 2 + 2
        assert np.all(o.particles()["ell"] < 1e-9)


# ----------------------------------------------------------------------------------
# Melting walk-back (Sec. 2.1.3, reading r17).  A grain with lattice axes along the
# lab axes is grown, then the melt above a plane between two lattice planes is
# superheated by a vanishing amount (so nothing grows in that step).  The state
# after the step is rebuilt here from the state before it: reached sites above the
# plane melt; particles above the plane or on a melted site go, and release their
# targets; every melted site of the first layer above the plane gets one particle
# from the surviving site below it, heading up (+z, the first direction whose
# neighbour survives).
# ----------------------------------------------------------------------------------
def _keyset(grain, site, extra=None):
    out = set()
    for i in range(len(grain)):
        k = (int(grain[i]), *(int(v) for v in site[i]))
        out.add(k + ((int(extra[i]),) if extra is not None else ()))
    return out


def test_melting_above_a_plane_walks_back_to_the_surviving_layer():
    h, dT, T_L = 2e-6, 5.0, 1000.0
    v = 1e-5 * dT ** 2
    dt = 0.37 * h / v
    c = np.array([60e-6, 60e-6, 60e-6])
    o = Oracle((0, 0, 0), (120e-6,) * 3, h, dt, (1e-5,), (2.0,), T_L)
    o.set_thermal_analytic(T_L - dT, (0, 0, 0), (0, 0, 0), 0.0)
    o.add_grains(c[None], np.array([[1.0, 0.0, 0.0, 0.0]]))
    o.step(40)
    p0 = o.particles()
    g0, s0 = o.reached()
    cg, cs = o.claimed()
    zc = 3                                   # lattice plane z = 3 survives, z = 4 melts
    z_cut = c[2] + (zc + 0.5) * h
    o.set_thermal_analytic(T_L, (0.0, 0.0, 1.0), (0.0, 0.0, z_cut), 0.0)   # dT = z_cut - z
    o.set_melting(True)
    o.step(1)
    p1 = o.particles()
    g1, s1 = o.reached()
    st = o.stats()

    alive = s0[:, 2] <= zc
    assert _keyset(g1, s1) == _keyset(g0[alive], s0[alive])
    assert st["melted"] == int((~alive).sum()) > 100
    alive_set = _keyset(g0[alive], s0[alive])
    keep = (p0["x"][:, 2] < z_cut) & np.array([(int(g), *map(int, s)) in alive_set
                                                 for g, s in zip(p0["grain"], p0["site"])])
    expect = _keyset(p0["grain"][keep], p0["site"][keep], p0["dir"][keep])
    walk = set()
    for g, s in zip(g0[~alive], s0[~alive]):
        if s[2] == zc + 1 and (int(g), int(s[0]), int(s[1]), zc) in alive_set:
            walk.add((int(g), int(s[0]), int(s[1]), zc, 4))
    assert st["walkback"] == len(walk) > 50
    assert _keyset(p1["grain"], p1["site"], p1["dir"]) == expect | walk
    # the old particles kept their progress (the superheat grows nothing); the new start at 0
    i0 = {(int(g), *map(int, s), int(d)): e for g, s, d, e in
          zip(p0["grain"], p0["site"], p0["dir"], p0["ell"])}
    for g, s, d, e in zip(p1["grain"], p1["site"], p1["dir"], p1["ell"]):
        k = (int(g), *map(int, s), int(d))
        assert abs(e - (0.0 if k in walk else i0[k])) < 1e-9
    # claims: melted sites and the targets of removed particles are released; the
    # walk-back targets are claimed again
    removed = ~keep
    tgt = p0["site"][removed].copy()
    ax = p0["dir"][removed] // 2
    sg = np.where(p0["dir"][removed] % 2 == 0, 1, -1)
    tgt[np.arange(len(tgt)), ax] += sg
    released = _keyset(p0["grain"][removed], tgt) | _keyset(g0[~alive], s0[~alive])
    expect_claimed = (_keyset(cg, cs) - released) | {(k[0], k[1], k[2], zc + 1) for k in walk}
    ng, ns = o.claimed()
    assert _keyset(ng, ns) == expect_claimed


def test_grain_melted_entirely_nucleates_again_from_its_seed():
    h, T_L = 2e-6, 1000.0
    o = Oracle((0, 0, 0), (80e-6,) * 3, h, 2e-3, (1e-5,), (2.0,), T_L)
    c = np.array([[40e-6, 40e-6, 40e-6]])
    o.nucleation_sites(c, np.array([0.5]), inputs.shoemake_quaternions(1, inputs.rng(2)))
    o.set_melting(True)
    o.set_thermal_analytic(T_L - 5.0, (0, 0, 0), (0, 0, 0), 0.0)
    o.step(30)
    assert o.n_grains == 1 and o.n_particles > 100
    o.set_thermal_analytic(T_L + 1.0, (0, 0, 0), (0, 0, 0), 0.0)     # superheat everywhere
    o.step(3)
    assert o.n_particles == 0 and len(o.reached()[0]) == 0
    o.set_thermal_analytic(T_L - 0.4, (0, 0, 0), (0, 0, 0), 0.0)     # below its dT_n = 0.5
    o.step(3)
    assert o.n_particles == 0 and o.stats()["nucleated"] == 1
    o.set_thermal_analytic(T_L - 0.6, (0, 0, 0), (0, 0, 0), 0.0)
    o.step(1)
    p = o.particles()
    assert o.n_grains == 1 and o.stats()["nucleated"] == 2
    assert sorted(p["dir"].tolist()) == list(range(6)) and (p["grain"] == 0).all()
    assert (p["site"] == 0).all()


# ----------------------------------------------------------------------------------
# Periodic axes (Sec. 3.4 applies periodic conditions normal to x and y; reading
# r18).  Two grains that meet across the x face of a periodic box must evolve exactly
# as the same two grains in a wider, non-periodic box in which the second grain is
# shifted by the period: lattice state, contacts and progress are identical.
# ----------------------------------------------------------------------------------
def _pair_run(periodic):
    h, dT, T_L = 2e-6, 5.0, 1000.0
    dt = 0.37 * h / (1e-5 * dT ** 2)
    L = 60e-6
    g = inputs.rng(31)
    q = inputs.shoemake_quaternions(2, g)
    a = [52e-6, 30e-6, 30e-6]
    b = [6e-6 + (0.0 if periodic else L), 31e-6, 29e-6]
    hi = (L if periodic else 2 * L, 60e-6, 60e-6)
    o = Oracle((0, 0, 0), hi, h, dt, (1e-5,), (2.0,), T_L)
    if periodic:
        o.set_periodic(1)
    o.set_thermal_analytic(T_L - dT, (0, 0, 0), (0, 0, 0), 0.0)
    o.add_grains(np.array([a, b]), q)
    o.step(24)
    return o


def test_periodic_box_equals_shifted_grains_in_a_wider_box():
    op, ow = _pair_run(True), _pair_run(False)
    p, q = op.particles(), ow.particles()
    kp = {(int(g), *map(int, s), int(d)): (int(st), e) for g, s, d, st, e in
          zip(p["grain"], p["site"], p["dir"], p["state"], p["ell"])}
    kq = {(int(g), *map(int, s), int(d)): (int(st), e) for g, s, d, st, e in
          zip(q["grain"], q["site"], q["dir"], q["state"], q["ell"])}
    assert kp.keys() == kq.keys()
    assert sum(st == 1 for st, _ in kp.values()) > 20          # they met across the face
    assert all(kp[k][0] == kq[k][0] and abs(kp[k][1] - kq[k][1]) < 1e-12 for k in kp)
    assert op.stats()["clipped"] == ow.stats()["clipped"] == 0
    # grain 0 crosses the face x = L: some of its sites lie beyond it
    gr, s = op.reached()
    c0, R0 = op.grain(0)
    assert (c0[0] + 2e-6 * (s[gr == 0] @ R0.T)[:, 0] > 60e-6).any()
