"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds input generation only: seed positions, orientations, thermal
fields and parameter sets.  It contains none of the particle method's arithmetic
(no growth law, no advance, no spawning, no contact search), so that both
implementations can be fed identical inputs without sharing method code.

Workloads (sizes and parameters follow the paper's benchmark families; every
random draw comes from numpy's PCG64 with the stated seed):

* ``single_grain``  - one grain at the centre of a 200 um cube, uniform
  undercooling, v = A dT^2 (the octahedron check of Sec. 2.1.2 / Fig. 1).
* ``columnar_slab`` - 50 seeds on the bottom face of a 1 mm x 1 mm x 50 um slab,
  frozen-temperature field T = T_L + G z - Tdot t (competitive columnar growth,
  the situation of Sec. 3.3 / 3.4).
* ``weld_fixture``  - a 4 x 2 x 1 mm plate (half domain, y >= 0 from the weld
  centre line), Rosenthal moving point source tabulated on a 512 x 256 x 128
  FP32 grid in the frame of the source, 1e4 Voronoi seeds with random
  orientations, each seeded as an octahedral shell (the laser-welding
  application of Sec. 4.2, with an analytic field standing in for the CFD).
* ``weld_natural``  - the same plate, field and seeds, with the base-metal grains
  cut by the fusion line: each grain (Voronoi cell of its seed) starts as the
  lattice sites of its own lattice lying in the solid within one spacing of the
  t = 0 liquidus surface, with particles heading into the melt (the weld
  application of Sec. 4.2, growth from the fusion boundary).
* ``cet_runs``      - per-run parameters of an ensemble of cubes with columnar
  bottom seeds and bulk nucleation sites (Sec. 3.5 family).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def shoemake_quaternions(n: int, g: np.random.Generator) -> np.ndarray:
    """Uniformly distributed unit quaternions (w, x, y, z).

    K. Shoemake, "Uniform random rotations", Graphics Gems III (1992): with
    u1, u2, u3 ~ U[0, 1), q = (sqrt(1-u1) sin 2pi u2, sqrt(1-u1) cos 2pi u2,
    sqrt(u1) sin 2pi u3, sqrt(u1) cos 2pi u3).
    """
    u = g.random((n, 3))
    a = np.sqrt(1.0 - u[:, 0])
    b = np.sqrt(u[:, 0])
    t1 = 2.0 * math.pi * u[:, 1]
    t2 = 2.0 * math.pi * u[:, 2]
    q = np.stack([b * np.cos(t2), a * np.sin(t1), a * np.cos(t1), b * np.sin(t2)], axis=1)
    return np.ascontiguousarray(q)


def euler_zxz_to_quaternion(psi_deg: float, theta_deg: float, phi_deg: float) -> np.ndarray:
    """Bunge (Z-X-Z) Euler angles in degrees -> unit quaternion (w, x, y, z).

    The paper quotes orientations as Euler angles (psi, theta, phi) without a
    convention; the Z-X-Z (Bunge) convention is the one taken here.
    """
    def qz(a):
        return np.array([math.cos(a / 2), 0.0, 0.0, math.sin(a / 2)])

    def qx(a):
        return np.array([math.cos(a / 2), math.sin(a / 2), 0.0, 0.0])

    def mul(p, q):
        w1, x1, y1, z1 = p
        w2, x2, y2, z2 = q
        return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                         w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                         w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])

    r = math.radians
    return mul(mul(qz(r(psi_deg)), qx(r(theta_deg))), qz(r(phi_deg)))


def truncated_normal(n: int, mean: float, sigma: float, lo: float, hi: float,
                     g: np.random.Generator) -> np.ndarray:
    """Normal(mean, sigma) draws restricted to [lo, hi] by rejection and redraw."""
    out = np.empty(n)
    filled = 0
    while filled < n:
        d = g.normal(mean, sigma, size=max(16, 2 * (n - filled)))
        d = d[(d >= lo) & (d <= hi)]
        take = min(d.size, n - filled)
        out[filled:filled + take] = d[:take]
        filled += take
    return out


@dataclass
class Workload:
    """Parameters of one simulation, in SI units."""
    name: str
    lo: tuple
    hi: tuple
    h: float
    dt: float
    a: tuple
    b: tuple
    T_L: float
    steps: int
    seeds: np.ndarray = None          # (n, 3) nucleus positions
    quats: np.ndarray = None          # (n, 4)
    analytic: dict = None             # T0, G, xref, Tdot
    grid: dict = None                 # T (nz, ny, nx) float32, origin, spacing, vel
    shell_n0: int = 0                 # > 0: seed each grain as a shell of n0 lattice shells
    nuclei: dict = None               # pos (m,3), dTn (m,), quat (m,4)
    solute: dict = None               # w (nz, ny, nx) float32, origin, spacing, vel, Tm, mL
    extra: dict = field(default_factory=dict)


def single_grain(seed: int = 1, steps: int = 400, dT: float = 5.0) -> Workload:
    """One grain, uniform undercooling dT, A = 1e-5 m/s/K^2, h = 2 um, dt = 2 ms."""
    g = rng(seed)
    q = shoemake_quaternions(1, g)
    T_L = 1000.0
    return Workload(
        name="single_grain", lo=(0.0, 0.0, 0.0), hi=(200e-6, 200e-6, 200e-6), h=2e-6,
        dt=2e-3, a=(1e-5,), b=(2.0,), T_L=T_L, steps=steps,
        seeds=np.array([[100e-6, 100e-6, 100e-6]]), quats=q,
        analytic=dict(T0=T_L - dT, G=(0.0, 0.0, 0.0), xref=(0.0, 0.0, 0.0), Tdot=0.0))


def columnar_slab(seed: int = 2, n_seeds: int = 50, size_xy: float = 1e-3,
                  height: float = 50e-6, steps: int = 600) -> Workload:
    """Seeds on z = 0, T = T_L + G z - Tdot t with G = 1e4 K/m, Tdot = 10 K/s."""
    g = rng(seed)
    xy = g.random((n_seeds, 2)) * size_xy
    seeds = np.concatenate([xy, np.zeros((n_seeds, 1))], axis=1)
    q = shoemake_quaternions(n_seeds, g)
    T_L = 1000.0
    return Workload(
        name="columnar_slab", lo=(0.0, 0.0, 0.0), hi=(size_xy, size_xy, height), h=2e-6,
        dt=1e-3, a=(1e-5,), b=(2.0,), T_L=T_L, steps=steps, seeds=seeds, quats=q,
        analytic=dict(T0=T_L, G=(0.0, 0.0, 1e4), xref=(0.0, 0.0, 0.0), Tdot=-10.0))


def rosenthal_T(x, y, z, Lz, q=1000.0, k=30.0, alpha=6e-6, V=1.0 / 60.0, T0=300.0,
                T_cap=3134.0, x_src=3e-3):
    """Thick-plate moving point source (Rosenthal) in the frame of the source, which
    sits at (x_src, 0, Lz): T = T0 + q / (2 pi k R) exp(-V (xi + R) / (2 alpha)), with
    xi = x - x_src along the travel direction and R the distance to the source,
    capped at T_cap (boiling point of 316L, Table S8)."""
    X = x - x_src
    Zd = Lz - z
    R = np.maximum(np.sqrt(X * X + y * y + Zd * Zd), 1e-9)
    T = T0 + q / (2.0 * math.pi * k * R) * np.exp(-V * (X + R) / (2.0 * alpha))
    return np.minimum(T, T_cap)


def rosenthal_table(shape=(128, 256, 512), extent=(4e-3, 2e-3, 1e-3), q=1000.0, k=30.0,
                    alpha=6e-6, V=1.0 / 60.0, T0=300.0, T_cap=3134.0, x_src=3e-3):
    """Thick-plate moving point source (Rosenthal) tabulated in the source frame.

    T = T0 + q / (2 pi k R) exp(-V (xi + R) / (2 alpha)), xi = x - x_src along the
    travel direction, R the distance to the source at the top surface
    (z = extent_z, y = 0).  Capped at T_cap (boiling point of 316L, Table S8)
    near the source.  Nodes are at origin + i * spacing, i = 0..n-1 (x fastest).
    Returns (T[nz, ny, nx] float32, origin, spacing).
    """
    nz, ny, nx = shape
    Lx, Ly, Lz = extent
    sp = (Lx / (nx - 1), Ly / (ny - 1), Lz / (nz - 1))
    x = np.arange(nx) * sp[0]
    y = np.arange(ny) * sp[1]
    z = np.arange(nz) * sp[2]
    T = rosenthal_T(x[None, None, :], y[None, :, None], z[:, None, None], Lz, q=q, k=k,
                    alpha=alpha, V=V, T0=T0, T_cap=T_cap, x_src=x_src).astype(np.float32)
    return np.ascontiguousarray(T), (0.0, 0.0, 0.0), sp


def weld_fixture(seed: int = 3, n_grains: int = 10000, shell_n0: int = 50,
                 steps: int = 2000, grid_shape=(128, 256, 512),
                 extent=(4e-3, 2e-3, 1e-3)) -> Workload:
    """Rosenthal plate with 1e4 grains, each seeded as an octahedral shell.

    A = 3e-6 m/s/K^3 (v = A dT^3), h = 2 um, dt = 0.1 ms, T_L = 1780 K; the
    1 kW, 1 m/min source moves along +x (the table is sampled in its frame, so
    the particle position is shifted by -V t before the lookup) and sits at 3/4
    of the plate length.  A smaller ``extent`` with proportionally fewer grains
    keeps the grain density of the full plate (used for profiling captures).
    """
    g = rng(seed)
    ext = tuple(float(v) for v in extent)
    seeds = g.random((n_grains, 3)) * np.array(ext)
    q = shoemake_quaternions(n_grains, g)
    V = 1.0 / 60.0
    T, origin, sp = rosenthal_table(shape=grid_shape, extent=ext, V=V, x_src=0.75 * ext[0])
    return Workload(
        name="weld_fixture", lo=(0.0, 0.0, 0.0), hi=ext, h=2e-6, dt=1e-4, a=(3e-6,), b=(3.0,),
        T_L=1780.0, steps=steps, seeds=seeds, quats=q,
        grid=dict(T=T, origin=origin, spacing=sp, vel=(V, 0.0, 0.0)), shell_n0=shell_n0)


def quaternion_matrix(q: np.ndarray) -> np.ndarray:
    """Rotation matrices (n, 3, 3), crystal -> lab, of unit quaternions (w, x, y, z)
    (normalised here); used to place the lattice sites of an initial state."""
    q = np.asarray(q, np.float64).reshape(-1, 4)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], 1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], 1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1)],
                    1)


def weld_natural(seed: int = 3, n_grains: int = 10000, steps: int = 500,
                 grid_shape=(128, 256, 512), extent=(4e-3, 2e-3, 1e-3),
                 chunk: int = 1 << 18) -> Workload:
    """The weld plate of ``weld_fixture`` with the base metal cut by the fusion line.

    Same plate, Rosenthal field, growth law, seeds and orientations as the fixture.
    The base metal is the solid (T <= T_L at t = 0) and each grain owns the points
    closest to its seed (Voronoi).  The initial particles of a grain sit at the sites
    s of its lattice (x = c + h R s) that lie in its Voronoi cell, in the solid and
    inside the plate, for each direction k that is outer at s (it increases |s|_1)
    and whose target s + e_k lies in the melt (T > T_L): the sites within one spacing
    of the liquidus surface, heading into the melt.  A target claimed by several such
    particles goes to the lowest direction index.  Their sites are reached and claimed,
    their targets claimed.  extra: particles (grain, site, dir, ell, state), reached
    and claimed (grain, site).  The field is the analytic Rosenthal temperature at
    t = 0, the one the table samples.

    The claimed boundary layer keeps the grains out of the base metal around the t = 0
    pool only; the state records no other solid.  So the run is 500 steps of 0.1 ms,
    over which the source moves 0.83 mm of the pool's 4.2 mm length and the grains grow
    inside the t = 0 pool; over much longer runs they would reach the never-melted
    base metal beside the new weld track and grow into it.

    Candidate sites: the grid cells whose corner temperatures straddle T_L hold the
    liquidus surface; for each grain that may own part of such a cell, the blocks of
    4 x 4 x 4 sites of its lattice that the cell touches are listed once, and all their
    sites are tested.
    """
    from scipy.spatial import cKDTree
    w = weld_fixture(seed=seed, n_grains=n_grains, shell_n0=0, steps=steps,
                     grid_shape=grid_shape, extent=extent)
    ext = np.array(w.hi, np.float64)
    h, T_L = w.h, w.T_L
    T, origin, sp = w.grid["T"], np.array(w.grid["origin"]), np.array(w.grid["spacing"])
    x_src = 0.75 * ext[0]
    B = 4                                           # lattice block edge, in sites

    def temp(p):
        return rosenthal_T(p[..., 0], p[..., 1], p[..., 2], ext[2], x_src=x_src)

    # grid cells whose eight corner temperatures straddle T_L hold the liquidus surface
    a = T > T_L
    corners = [a[dz:a.shape[0] - 1 + dz, dy:a.shape[1] - 1 + dy, dx:a.shape[2] - 1 + dx]
               for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
    vz, vy, vx = np.nonzero(np.logical_or.reduce(corners) & ~np.logical_and.reduce(corners))
    vlo = origin + np.stack([vx, vy, vz], 1) * sp   # low corner of each surface cell
    seeds = w.seeds
    tree = cKDTree(seeds)
    kq = min(8, len(seeds))
    rad = 0.5 * np.linalg.norm(sp) + h
    dist, cand = tree.query(vlo + 0.5 * sp, k=kq)
    dist, cand = dist.reshape(len(vlo), kq), cand.reshape(len(vlo), kq)
    pv, pg = np.nonzero(dist <= dist[:, :1] + 2 * rad)   # (cell, grain) pairs
    gi = cand[pv, pg]
    hR = h * quaternion_matrix(w.quats)             # (n, 3, 3), columns h R e_a
    Rinv = np.transpose(hR, (0, 2, 1)) / (h * h)    # lab -> lattice coordinates
    cube = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], np.float64)
    # lattice blocks touched by each pair's cell (its 8 corners give the block range)
    u = np.einsum("mij,mcj->mci", Rinv[gi], vlo[pv][:, None, :] + cube[None] * sp - seeds[gi][:, None])
    b0 = np.floor(u.min(1) / B).astype(np.int64)
    b1 = np.floor(u.max(1) / B).astype(np.int64)
    span = b1 - b0 + 1                              # blocks per axis, 1..3
    o = np.array([[i, j, k] for i in range(3) for j in range(3) for k in range(3)])
    blk = b0[:, None, :] + o[None]                  # (m, 27, 3)
    valid = np.all(o[None] < span[:, None, :], -1)
    m_, q_ = np.nonzero(valid)
    bb = blk[m_, q_] + (1 << 15)                    # block coordinates, made positive
    packed = (((gi[m_].astype(np.int64) << 16 | bb[:, 0]) << 16 | bb[:, 1]) << 16) | bb[:, 2]
    packed = np.unique(packed)                      # (grain, block) listed once
    keys = np.column_stack([packed >> 48, ((packed >> 32) & 0xFFFF) - (1 << 15),
                            ((packed >> 16) & 0xFFFF) - (1 << 15), (packed & 0xFFFF) - (1 << 15)])
    # keep the blocks that the liquidus can cross: over the corners of the block grown by
    # one spacing, T reaches T_L - 5 K and T_L + 5 K (the field is smooth on this scale)
    corners8 = np.array([[i, j, k] for i in (-1, B) for j in (-1, B) for k in (-1, B)], np.float64)
    keep = np.zeros(len(keys), bool)
    cb = 1 << 16
    for c0 in range(0, len(keys), cb):
        kb = keys[c0:c0 + cb]
        Rb = hR[kb[:, 0]]
        xc = seeds[kb[:, 0]][:, None, :] + np.matmul(Rb[:, None], (kb[:, None, 1:] * B + corners8)[..., None])[..., 0]
        tc = temp(xc)
        keep[c0:c0 + cb] = (tc.min(1) <= T_L + 5.0) & (tc.max(1) >= T_L - 5.0)
    keys = keys[keep]
    site_off = np.array([[i, j, k] for i in range(B) for j in range(B) for k in range(B)])
    E = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
    out_g, out_s, out_k = [], [], []
    per = max(1, chunk // len(site_off))
    for c0 in range(0, len(keys), per):
        kb = keys[c0:c0 + per]
        gb = kb[:, 0]
        Rb = hR[gb]                                 # one rotation per block
        sb = kb[:, None, 1:] * B + site_off[None]   # (nb, 64, 3) sites
        xs = (seeds[gb] + np.matmul(Rb, (kb[:, 1:] * B)[..., None])[..., 0])[:, None, :] + \
            np.swapaxes(np.matmul(Rb, site_off.T.astype(np.float64)), 1, 2)
        bi, si = np.nonzero(np.all((xs >= 0) & (xs <= ext), -1) & (temp(xs) <= T_L))
        g_, ss, xs = gb[bi], sb[bi, si], xs[bi, si]
        sel = np.zeros((6, len(g_)), bool)
        for k in range(6):
            ax, sg = k // 2, 1 - 2 * (k % 2)
            outer = (ss[:, ax] == 0) | (np.sign(ss[:, ax]) == sg)
            sel[k] = outer & (temp(xs + Rb[bi, :, ax] * sg) > T_L)
        keep = sel.any(0)
        # Voronoi: the nearest seed owns the site
        _, near = tree.query(xs[keep])
        own = np.zeros(len(g_), bool)
        own[np.flatnonzero(keep)] = near == g_[keep]
        for k in range(6):
            ok = sel[k] & own
            out_g.append(g_[ok])
            out_s.append(ss[ok])
            out_k.append(np.full(int(ok.sum()), k))
    grain = np.concatenate(out_g).astype(np.int32)
    site = np.concatenate(out_s).astype(np.int64)
    dirk = np.concatenate(out_k).astype(np.int64)
    # one particle per target: the lowest direction index among its claimants
    tgt = site + E[dirk]
    order = np.lexsort((dirk, tgt[:, 2], tgt[:, 1], tgt[:, 0], grain))
    grain, site, dirk, tgt = grain[order], site[order], dirk[order], tgt[order]
    first = np.r_[True, np.any(np.diff(np.column_stack([grain, tgt]), axis=0) != 0, 1)]
    grain, site, dirk, tgt = grain[first], site[first], dirk[first], tgt[first]
    reached = np.unique(np.column_stack([grain, site]), axis=0)
    n = len(grain)
    w.name = "weld_natural"
    w.extra = dict(
        particles=dict(grain=grain, site=site.astype(np.int32), dir=dirk.astype(np.int8),
                       ell=np.zeros(n, np.float32), state=np.zeros(n, np.uint8)),
        reached=(reached[:, 0].astype(np.int32), reached[:, 1:].astype(np.int32)),
        claimed=(grain.copy(), tgt.astype(np.int32)))
    return w


def cet_runs(n_runs: int = 256, base_seed: int = 1000, L_range=(0.5e-3, 2e-3),
             seed_density: float = 50e6, nuc_density: float = 1e11, G_range=(100.0, 1e4),
             Tdot_range=(0.5, 20.0), steps: int = 400):
    """Per-run parameters of the columnar-to-equiaxed ensemble (Sec. 3.5 family).

    Run r (seed base_seed + r): cube edge L ~ U[L_range], columnar seeds on the
    bottom face (Poisson, seed_density per m^2, at least one) that start growing at
    once, bulk nucleation sites (Poisson, nuc_density per m^3, uniform in the cube)
    with dT_n ~ N(5, 1) K truncated to >= 0, T = T_L + G z - Tdot t with
    G ~ U[G_range] K/m and Tdot ~ U[Tdot_range] K/s, v = 1e-5 dT^2, h = 2 um,
    dt = 1 ms.  The defaults are the 256-run ensemble of 0.5-2 mm cubes over 400
    steps, after which its runs hold between 45 and 8e5 particles.
    """
    runs = []
    for r in range(n_runs):
        g = rng(base_seed + r)
        L = g.uniform(*L_range)
        nb = max(1, g.poisson(seed_density * L ** 2))
        bottom = np.concatenate([g.random((nb, 2)) * L, np.zeros((nb, 1))], axis=1)
        qb = shoemake_quaternions(nb, g)
        nv = g.poisson(nuc_density * L ** 3)
        bulk = g.random((nv, 3)) * L
        dTn = truncated_normal(nv, 5.0, 1.0, 0.0, np.inf, g)
        qv = shoemake_quaternions(nv, g)
        G = g.uniform(*G_range)
        Tdot = g.uniform(*Tdot_range)
        T_L = 1000.0
        runs.append(Workload(
            name=f"cet_run_{r}", lo=(0.0, 0.0, 0.0), hi=(L, L, L), h=2e-6, dt=1e-3,
            a=(1e-5,), b=(2.0,), T_L=T_L, steps=steps, seeds=bottom, quats=qb,
            analytic=dict(T0=T_L, G=(0.0, 0.0, G), xref=(0.0, 0.0, 0.0), Tdot=-Tdot),
            nuclei=dict(pos=bulk, dTn=dTn, quat=qv)))
    return runs


def thin_sample(lambda0: float = 48e-6, steps: int = 200) -> Workload:
    """Directional solidification of a quasi-2D thin sample (Sec. 3.3, Table S2).

    Growth along +y in a frozen temperature field T = T_L + G y + Tdot t with
    G = 1900 K/m and Tdot = -0.1634 K/s (pulling at 86 um/s), T_L = 937.65 K; v from
    Eq. (2) with a1 = 8.26e-6, b1 = 2, a2 = 8.18e-5, b2 = 3; dt = 0.1 s; h = lambda0.
    Fifteen nuclei at y = 0.15 um, x = L_x / 2 + i 360 um (i = -7..7), mid-thickness,
    rotated about the sample normal z by psi = 4 deg (i <= -5), 30 deg (|i| <= 4) and
    11 deg (i >= 5).  The sample is 400 um thick and 2 mm long (Table S2); its width
    is taken as 15 x 360 um = 5.4 mm so that every nucleus lies in it (the table's
    4 mm width is shorter than the nucleus row).
    """
    Lx, Ly, Lz = 15 * 360e-6, 2e-3, 400e-6
    i = np.arange(-7, 8)
    seeds = np.stack([Lx / 2 + i * 360e-6, np.full(15, 0.15e-6), np.full(15, Lz / 2)], 1)
    psi = np.where(i <= -5, 4.0, np.where(i >= 5, 11.0, 30.0))
    quats = np.array([euler_zxz_to_quaternion(p, 0.0, 0.0) for p in psi])
    T_L = 937.65
    return Workload(name=f"thin_sample_{lambda0 * 1e6:.0f}um", lo=(0.0, 0.0, 0.0),
                    hi=(Lx, Ly, Lz), h=lambda0, dt=0.1, a=(8.26e-6, 8.18e-5), b=(2.0, 3.0),
                    T_L=T_L, steps=steps, seeds=seeds, quats=quats,
                    analytic=dict(T0=T_L, G=(0.0, 1900.0, 0.0), xref=(0.0, 0.0, 0.0),
                                  Tdot=-0.1634),
                    extra=dict(psi=psi))


def adjoint_cube(seed: int = 5, n_grains: int = 32, steps: int = 200, A: float = 1e-5,
                 n: float = 2.0, G: float = 1e3, Tdot: float = 10.0,
                 height: float = 200e-6) -> Workload:
    """Calibration case of the adjoint: the 200 um single-grain cube with 32 grains
    (seed 5), T = T_L - 5 + G (z - z_c) - Tdot t, v = A dT^n, h = 2 um, dt = 2 ms.
    With height > 200 um the box is taller than the cube that holds the seeds, so the
    highest point of the envelope grows freely (the front height stays ACTIVE)."""
    g = rng(seed)
    L = 200e-6
    seeds = g.random((n_grains, 3)) * L
    q = shoemake_quaternions(n_grains, g)
    T_L = 1000.0
    return Workload(
        name="adjoint_cube", lo=(0.0, 0.0, 0.0), hi=(L, L, height), h=2e-6, dt=2e-3, a=(A,),
        b=(n,), T_L=T_L, steps=steps, seeds=seeds, quats=q,
        analytic=dict(T0=T_L - 5.0, G=(0.0, 0.0, G), xref=(0.0, 0.0, L / 2), Tdot=-Tdot))
