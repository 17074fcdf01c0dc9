"""Batched ensembles (several independent runs per context) on the GPU.

A run of a batch context uses only its own domain, cells, field and nuclei, in the
same binary32 arithmetic as a single-run context, so its particles must equal,
bit for bit, those of the same run stepped alone.  Grain ids differ between the
two contexts (a batch reserves nucleus ids at registration, a single run numbers
them at activation), so grains are matched by their nucleus.  One run is also
compared with the FP64 oracle through its grain map.
"""
import numpy as np
import pytest

from paper_2504_12858_gb300 import ensemble, inputs, native
from tests.helpers import nucleus_keys, oracle_from, sim_from

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def small_ensemble(n_runs=5, steps=400):
    # 100-200 um cubes, denser seeding so that each run holds a few grains of both
    # kinds; Tdot high enough for bulk nucleation within the run
    return inputs.cet_runs(n_runs=n_runs, base_seed=2000, L_range=(100e-6, 200e-6),
                           seed_density=1e9, nuc_density=3e12, Tdot_range=(14.0, 20.0),
                           steps=steps)


def _canon(p):
    key = np.lexsort((p["dir"], p["site"][:, 2], p["site"][:, 1], p["site"][:, 0], p["grain"]))
    return {k: v[key] for k, v in p.items()}


@pytest.fixture(scope="module")
def stepped_batch():
    native.load()
    runs = small_ensemble()
    b = ensemble.batch_from(runs, capacity=3_000_000, reached_capacity=8_000_000)
    b.gp_step(runs[0].steps)
    return runs, b


def test_batch_runs_equal_single_runs_bit_for_bit(stepped_batch):
    runs, b = stepped_batch
    live, active = b.gp_run_counts()
    tot = 0
    nucleated = 0
    for r, w in enumerate(runs):
        s = sim_from(w, capacity=1_000_000, reached_capacity=3_000_000)
        s.gp_step(w.steps)
        ps = _canon(nucleus_keys(s, s.gp_get_particles(), w))
        pb = _canon(nucleus_keys(b, ensemble.run_particles(b, r), w))
        assert len(ps["grain"]) == live[r] > 1000, r
        assert (ps["state"] == 0).sum() == active[r]
        assert (ps["grain"] >= 0).all() and (pb["grain"] >= 0).all()
        for k in ("grain", "site", "dir", "state"):
            assert np.array_equal(ps[k], pb[k]), (r, k)
        assert np.array_equal(ps["ell"].view(np.uint32), pb["ell"].view(np.uint32)), r
        assert np.array_equal(ps["x"].view(np.uint32), pb["x"].view(np.uint32)), r
        st = s.gp_stats()
        tot += st["particle_steps"]
        nucleated += st["n_nucleated"]
        # grain maps of the run agree voxel for voxel (after mapping grain ids)
        L = w.hi[0]
        nv, sp = (24, 24, 24), (L / 24,) * 3
        ms = s.gp_grain_map((0, 0, 0), sp, nv)
        mb = b.gp_run_grain_map(r, (0, 0, 0), sp, nv)
        c3s, _ = native.grain_table(s)
        c3b, _ = native.grain_table(b)
        pos_s = {g: tuple(c3s[g]) for g in np.unique(ms[ms >= 0])}
        pos_b = {g: tuple(c3b[g]) for g in np.unique(mb[mb >= 0])}
        assert np.array_equal(ms >= 0, mb >= 0)
        assert all(pos_s[a] == pos_b[c] for a, c in zip(ms[ms >= 0], mb[mb >= 0]))
        s.close()
    sb = b.gp_stats()
    assert sb["particle_steps"] == tot
    assert sb["n_nucleated"] == nucleated > 0


def test_batch_run_grain_map_matches_oracle(stepped_batch):
    runs, b = stepped_batch
    r = 0
    w = runs[r]
    o = oracle_from(w)
    o.step(w.steps)
    L = w.hi[0]
    nv, sp = (30, 30, 30), (L / 30,) * 3
    mo = o.grain_map((0, 0, 0), sp, nv)
    mb = b.gp_run_grain_map(r, (0, 0, 0), sp, nv)
    c3b, _ = native.grain_table(b)
    # oracle grains: seeds first, then nuclei in activation order; compare by nucleus
    po = {g: tuple(np.float32(v) for v in o.grain(g)[0]) for g in np.unique(mo[mo >= 0])}
    agree = np.mean([(a < 0 and c < 0) or (a >= 0 and c >= 0 and po[a] == tuple(c3b[c]))
                     for a, c in zip(mo.ravel(), mb.ravel())])
    assert agree >= 0.995, agree
    assert (mo >= 0).mean() > 0.05


def test_batch_errors():
    native.load()
    runs = small_ensemble(n_runs=2, steps=1)
    b = ensemble.batch_from(runs, capacity=10_000)
    with pytest.raises(native.GPError):
        b.gp_run_grain_map(2, (0, 0, 0), (1e-5,) * 3, (2, 2, 2))   # no such run
    with pytest.raises(native.GPError):
        b.gp_set_thermal_grid(np.zeros((2, 2, 2), np.float32), (0, 0, 0), (1, 1, 1))
    with pytest.raises(native.GPError):
        b.gp_tape_begin()


def _state(b):
    p = _canon(b.gp_get_particles())
    st = b.gp_stats()
    return p, {k: st[k] for k in ("n_live", "n_active", "n_reached", "particle_steps",
                                  "n_spawned", "n_nucleated", "n_clipped", "n_frozen_new")}


def test_graphs_launch_configs_and_autotuner_keep_results_identical():
    """The batch step sizes every launch on the device; replaying it from captured
    CUDA graphs, with other persistent grids, or with the autotuner's choice gives
    the same particles and counters, bit for bit."""
    native.load()
    runs = small_ensemble(n_runs=4, steps=300)
    ref = ensemble.batch_from(runs, capacity=2_000_000, reached_capacity=6_000_000)
    ref.gp_step(300)
    p0, s0 = _state(ref)
    ref.close()
    assert s0["n_nucleated"] > 0 and s0["n_live"] > 10000

    g = ensemble.batch_from(runs, capacity=2_000_000, reached_capacity=6_000_000)
    g.gp_set_launch_config(build_ctas_per_sm=2, advance_ctas_per_sm=1, emit_ctas_per_sm=3,
                           graph_steps=25)
    g.gp_step(130)          # 5 graphs of 25 steps and one of 5
    g.gp_step(170)
    p1, s1 = _state(g)
    g.close()

    t = ensemble.batch_from(runs, capacity=2_000_000, reached_capacity=6_000_000)
    t.gp_step(100)
    cfg = t.gp_autotune(trial_steps=2)         # 8 candidates x 2 real steps
    assert t.gp_stats()["step"] == 116
    t.gp_set_launch_config(graph_steps=16)
    t.gp_step(184)
    p2, s2 = _state(t)
    t.close()
    assert cfg["build_ctas_per_sm"] in (4, 8) and cfg["advance_ctas_per_sm"] in (4, 8)
    assert cfg["emit_ctas_per_sm"] in (4, 6)

    for p, s in ((p1, s1), (p2, s2)):
        assert s == s0
        for k in ("grain", "site", "dir", "state"):
            assert np.array_equal(p[k], p0[k]), k
        assert np.array_equal(p["ell"].view(np.uint32), p0["ell"].view(np.uint32))
