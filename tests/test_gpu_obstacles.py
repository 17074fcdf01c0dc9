"""Obstacle store and ordering of the particle step (GPU tests).

A FROZEN particle never moves again (Sec. 2.1.2: points of two grains that meet
stop and form the grain boundary); the library moves such particles into an
obstacle store ordered by cell, whose positions every step's ordering places beside
those of the moving particles for the contact search.  These tests check that:
- the three modes (off, automatic, a flush every step) give bit-identical results:
  every particle's grain, site, direction, state, progress and position, the step
  counters and the grain map, on a polycrystal in a gradient, on a small weld plate
  and on a state with crowded cells;
- the ordering the step builds (the per-step store grouped by tile of 1024 cells and
  ordered by cell inside each tile, together with the obstacles) equals a stable sort
  of the same tiled cell keys, up to the order of particles inside one cell; the keys
  themselves equal the tiled form of the oracle's binary32 cell of each exported
  position; the cell table (first index, count, 4-bit cell counts, saturation flag) is
  recomputed from the sorted keys and compared entry by entry; the obstacle store is
  ordered by key;
- melting, periodic axes, the adjoint tape and gp_load_particles bring the
  obstacles back into the per-step store without changing the particle set;
- behind a moving weld pool, where the ordering reads the obstacles of tiles without
  moving particles in place from the store, the run equals the one without the store.
"""
import numpy as np
import pytest

import oracle
from paper_2504_12858_gb300 import inputs
from tests.helpers import canon, oracle_from, sim_from

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2504_12858_gb300 import build, native  # noqa: E402

build.build()
native.load()

STATS = ("particle_steps", "n_frozen_new", "n_spawned", "n_claims_lost", "n_clipped",
         "n_clamped", "n_reached", "n_live", "n_frozen", "n_active", "n_grains", "error_flags")


def _polycrystal(seed=5, n_grains=12, L=60e-6, steps=40, dT=4.0):
    g = inputs.rng(seed)
    T_L = 1000.0
    return inputs.Workload(name="poly", lo=(0, 0, 0), hi=(L,) * 3, h=2e-6, dt=1.3e-3, a=(1e-5,),
                           b=(2.0,), T_L=T_L, steps=steps, seeds=g.random((n_grains, 3)) * L,
                           quats=inputs.shoemake_quaternions(n_grains, g),
                           analytic=dict(T0=T_L - dT, G=(3e4, -2e4, 1e4), xref=(L / 2,) * 3,
                                         Tdot=-20.0))


def _weld_plate():
    # the bench's grain density (1250 grains per mm^3, 50-shell envelopes) on a
    # 0.5 x 0.5 x 0.25 mm plate
    return inputs.weld_fixture(n_grains=78, shell_n0=50, grid_shape=(32, 64, 64),
                               extent=(0.5e-3, 0.5e-3, 0.25e-3))


def _run(w, mode, steps, capacity, **kw):
    s = sim_from(w, capacity=capacity, reached_capacity=8 * capacity, **kw)
    s.gp_set_obstacle_store(mode)
    n_obs = []
    for _ in range(steps):
        s.gp_step(1)
        n_obs.append(len(s.gp_inspect_order(1)["keys_sorted"]))
    return s, n_obs


def _same(a, b):
    pa, pb = canon(a.gp_get_particles()), canon(b.gp_get_particles())
    for f in ("grain", "site", "dir", "state"):
        assert np.array_equal(pa[f], pb[f]), f
    assert np.array_equal(pa["ell"].view(np.uint32), pb["ell"].view(np.uint32))
    assert np.array_equal(pa["x"].view(np.uint32), pb["x"].view(np.uint32))
    sa, sb = a.gp_stats(), b.gp_stats()
    assert {k: sa[k] for k in STATS} == {k: sb[k] for k in STATS}


@pytest.mark.parametrize("case", ["polycrystal", "weld_plate"])
def test_obstacle_modes_give_identical_results(case):
    if case == "polycrystal":
        w, steps, cap = _polycrystal(), 40, 400000
    else:
        w, steps, cap = _weld_plate(), 8, 3000000
    kw = {} if w.grid is None else dict(claim_blocks=len(w.seeds) * 2500)
    ref, n0 = _run(w, 0, steps, cap, **kw)
    assert max(n0) == 0
    for mode in (1, 2):
        s, n_obs = _run(w, mode, steps, cap, **kw)
        assert max(n_obs) > 0, mode
        _same(s, ref)
        if w.grid is None:
            nv, sp = (30, 30, 30), (2e-6,) * 3
        else:
            nv, sp = (50, 50, 25), (10e-6,) * 3
        assert np.array_equal(s.gp_grain_map((0, 0, 0), sp, nv), ref.gp_grain_map((0, 0, 0), sp, nv))
        s.close()
    ref.close()


def _tiled_keys(x, lo, hi, h):
    """Cell keys of the particle step: the oracle's binary32 cell of each position,
    in tiles of 16 x 8 x 8 cells ordered z, y, x, x fastest inside a tile."""
    lin = oracle.cell_keys_f32(x, lo, hi, h).astype(np.int64)
    e = h * (1.0 + 1.0 / 512.0)
    nx, ny, nz = (max(1, int(np.ceil((hi[a] - lo[a]) / e))) for a in range(3))
    cx, cy, cz = lin % nx, (lin // nx) % ny, lin // (nx * ny)
    tx, ty = (nx + 15) // 16, (ny + 7) // 8
    tile = ((cz >> 3) * ty + (cy >> 3)) * tx + (cx >> 4)
    return (tile * 1024 + ((cz & 7) * 8 + (cy & 7)) * 16 + (cx & 15)).astype(np.uint32)


def _check_table(keys_sorted, table, valid):
    """Recomputes the cell table from the sorted keys and compares every entry;
    valid(table) marks the entries that are occupied (vectorised over the table)."""
    seg = keys_sorted >> 4
    starts = np.flatnonzero(np.r_[True, seg[1:] != seg[:-1]]) if len(seg) else np.zeros(0, int)
    ends = np.r_[starts[1:], len(seg)]
    occupied = np.zeros(len(table), bool)
    for a, b in zip(starts, ends):
        sg = int(seg[a])
        occupied[sg] = True
        e = table[sg]
        assert e[0] == a and (e[1] & 0x7FFF) == b - a, (sg, e, a, b)
        cnt = np.bincount(keys_sorted[a:b] & 15, minlength=16)
        nib = np.minimum(cnt, 15)
        assert e[2] == sum(int(nib[c]) << (4 * c) for c in range(8)), sg
        assert e[3] == sum(int(nib[8 + c]) << (4 * c) for c in range(8)), sg
        assert bool(e[1] & 0x8000) == bool((cnt >= 15).any()), sg
    assert np.array_equal(valid(table), occupied)


def _check_ordering(s, w):
    """The cell-ordered sequence of the next step (moving particles and obstacles) and
    the obstacle store, against the oracle's cells of the exported positions."""
    p = s.gp_get_particles()
    d, o = s.gp_inspect_order(0), s.gp_inspect_order(1)
    n, no = len(p["grain"]), len(o["keys_sorted"])
    nd = n - no
    assert len(d["keys_sorted"]) == n
    lo, hi = np.array(w.lo, np.float64), np.array(w.hi, np.float64)
    keys = _tiled_keys(p["x"], lo, hi, w.h)
    # every particle's key; the sequence is a stable sort of them up to the order inside
    # a cell; every entry of the table
    assert np.array_equal(d["keys_in"], keys)
    stable = np.argsort(keys, kind="stable")
    assert np.array_equal(d["keys_sorted"], keys[stable])
    assert np.array_equal(np.sort(d["src"]), np.arange(n, dtype=np.uint32))
    assert np.array_equal(keys[d["src"]], d["keys_sorted"])
    _check_table(d["keys_sorted"], d["table"], lambda t: (t[:, 1] >> 16) == d["stamp"])
    # the obstacle store: frozen particles, the last ones listed, in key order
    assert (p["state"][nd:] == 1).all()
    assert np.array_equal(o["src"], np.arange(nd, n, dtype=np.uint32))
    assert np.array_equal(o["keys_sorted"], keys[nd:])
    assert np.all(np.diff(o["keys_sorted"].astype(np.int64)) >= 0)
    return nd, no, d


def test_ordering_and_tables_match_the_oracle_cells():
    w = _polycrystal(seed=7, n_grains=16, L=80e-6, dT=8.0)
    s, n_obs = _run(w, 2, 30, 600000)
    nd, no, _ = _check_ordering(s, w)
    assert nd > 1000 and no > 1000
    s.gp_step(1)
    _check_ordering(s, w)


def test_crowded_cells_in_both_stores():
    # 40 grains nucleated inside one cell: 240 particles there (saturated 4-bit
    # counts), half of them FROZEN from the start, among a sparse polycrystal
    w = _polycrystal(seed=9, n_grains=8, L=60e-6)
    g = inputs.rng(10)
    crowd = np.array([31e-6, 29e-6, 33e-6]) + g.random((40, 3)) * 1.5e-6
    w = inputs.Workload(**{**w.__dict__,
                           "seeds": np.concatenate([w.seeds, crowd]),
                           "quats": np.concatenate([w.quats, inputs.shoemake_quaternions(40, g)])})
    runs = {}
    for mode in (0, 2):
        s = sim_from(w, capacity=400000)
        s.gp_set_obstacle_store(mode)
        p = s.gp_get_particles()
        st = np.where(np.arange(len(p["grain"])) % 2 == 0, 1, 0).astype(np.uint8)
        st[p["grain"] < 8] = 0
        s.gp_load_particles(p["grain"], p["site"], p["dir"], p["ell"], st, 0)
        for _ in range(4):
            s.gp_step(1)
        runs[mode] = s
    o = runs[2].gp_inspect_order(1)
    assert len(o["keys_sorted"]) > 100
    _, _, d = _check_ordering(runs[2], w)
    sat = np.flatnonzero(((d["table"][:, 1] >> 16) == d["stamp"]) & (d["table"][:, 1] & 0x8000 != 0))
    assert len(sat) > 0                                # saturated cells hold obstacles
    crowd_seg = np.unique(o["keys_sorted"] >> 4)
    assert np.isin(sat, crowd_seg).any()
    _check_ordering(runs[0], w)
    _same(runs[2], runs[0])


def test_obstacles_return_to_the_per_step_store():
    w = _polycrystal(seed=5)
    for action in ("melting", "tape", "periodic", "load", "off"):
        s = sim_from(w, capacity=400000, tape_steps=2)
        for _ in range(30):
            s.gp_step(1)
        n_obs = len(s.gp_inspect_order(1)["keys_sorted"])
        assert n_obs > 0
        before, st0 = canon(s.gp_get_particles()), s.gp_stats()
        if action == "melting":
            s.gp_set_melting(True)
        elif action == "tape":
            s.gp_tape_begin()
        elif action == "periodic":
            s.gp_set_periodic(1)
        elif action == "off":
            s.gp_set_obstacle_store(0)
        else:
            p = s.gp_get_particles()
            s.gp_load_particles(p["grain"], p["site"], p["dir"], p["ell"], p["state"], 30)
        assert len(s.gp_inspect_order(1)["keys_sorted"]) == 0, action
        after, st1 = canon(s.gp_get_particles()), s.gp_stats()
        for f in ("grain", "site", "dir", "state", "ell"):
            assert np.array_equal(before[f], after[f]), (action, f)
        assert (st0["n_live"], st0["n_frozen"]) == (st1["n_live"], st1["n_frozen"]), action
        s.close()


def test_obstacle_run_matches_the_oracle_grain_map():
    w = _polycrystal(seed=11, n_grains=10, L=50e-6, steps=45)
    o = oracle_from(w)
    s = sim_from(w, capacity=400000)
    s.gp_set_obstacle_store(2)
    o.step(w.steps)
    s.gp_step(w.steps)
    nv, sp = (50, 50, 50), (1e-6,) * 3
    assert (o.grain_map((0, 0, 0), sp, nv) == s.gp_grain_map((0, 0, 0), sp, nv)).mean() >= 0.995
    assert len(s.gp_inspect_order(1)["src"]) > 0


def test_modes_identical_behind_a_moving_weld_pool():
    # growth from the t = 0 fusion line of the weld plate (inputs.weld_natural): after 150
    # steps much of the solid lies in tiles of 16 x 8 x 8 cells without moving particles,
    # whose obstacles the ordering reads in place from the store instead of copying them;
    # the state equals that of the run without the store, bit for bit
    w = inputs.weld_natural(steps=150)
    runs = {}
    for mode in (0, 1):
        s = sim_from(w, capacity=30000000, reached_capacity=250000000, claim_blocks=1500000)
        s.gp_set_obstacle_store(mode)
        s.gp_step(150)
        runs[mode] = s
    assert len(runs[1].gp_inspect_order(1)["keys_sorted"]) > 1000000
    _same(runs[1], runs[0])
    for s in runs.values():
        s.close()
