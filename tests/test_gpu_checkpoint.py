"""Checkpoints of a single-run context (gp_save / gp_load) on the GPU.

A run saved between steps and loaded into a new context steps on as the saved run
does: after further steps every particle's grain, site, direction, state, progress
bits and position bits, the reached sites, the step counters and the grain map are
equal.  The cases:
- a polycrystal in a gradient with bulk nucleation sites, some active and some still
  pending at the save, and FROZEN particles in the obstacle store;
- a heating and cooling cycle saved in the middle of the heating, with melting on:
  melted entries in the reached-site list, particles walked back, grains that may
  nucleate again;
- periodic axes;
- a load into a context of other capacities.
Refused, leaving the new context usable: a checkpoint with one byte changed, one cut
short, one of another domain, a context that is not new, a batch context, and a
context too small for the state.
"""
import numpy as np
import pytest

from paper_2504_12858_gb300 import inputs
from tests.helpers import canon, sim_from

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2504_12858_gb300 import build, native  # noqa: E402

build.build()
native.load()

STATS = ("step", "particle_steps", "n_frozen_new", "n_spawned", "n_claims_lost", "n_clipped",
         "n_clamped", "n_reached", "n_live", "n_frozen", "n_active", "n_grains",
         "n_nucleated", "n_claim_blocks", "n_melted", "n_walkback", "error_flags")


def _polycrystal(seed=5, n_grains=12, L=60e-6, n_nuclei=40):
    g = inputs.rng(seed)
    T_L = 1000.0
    nuc = dict(pos=g.random((n_nuclei, 3)) * L, dTn=4.0 + 1.5 * g.random(n_nuclei),
               quat=inputs.shoemake_quaternions(n_nuclei, g)) if n_nuclei else None
    return inputs.Workload(name="poly", lo=(0, 0, 0), hi=(L,) * 3, h=2e-6, dt=1.3e-3, a=(1e-5,),
                           b=(2.0,), T_L=T_L, steps=60, seeds=g.random((n_grains, 3)) * L,
                           quats=inputs.shoemake_quaternions(n_grains, g),
                           analytic=dict(T0=T_L - 4.0, G=(3e4, -2e4, 1e4), xref=(L / 2,) * 3,
                                         Tdot=-20.0), nuclei=nuc)


MEM = dict(capacity=400000, reached_capacity=2000000, claim_blocks=60000, max_nuclei=64)


def _saved(w, **kw):
    """The run to save (sim_from sizes its grain table for the seeds and sites)."""
    return sim_from(w, **{**MEM, **kw})


def _new(w, **kw):
    """A new context of the workload's domain, h, dt and growth law (no grains yet)."""
    mem = {**MEM, "max_grains": 128, **kw}
    return native.Sim(w.lo, w.hi, w.h, w.dt, w.a, w.b, w.T_L, **mem)


def _sites(s):
    g, x = s.gp_get_reached()
    return sorted(zip(g.tolist(), map(tuple, x.tolist())))


def _same(a, b):
    pa, pb = canon(a.gp_get_particles()), canon(b.gp_get_particles())
    for f in ("grain", "site", "dir", "state"):
        assert np.array_equal(pa[f], pb[f]), f
    assert np.array_equal(pa["ell"].view(np.uint32), pb["ell"].view(np.uint32))
    assert np.array_equal(pa["x"].view(np.uint32), pb["x"].view(np.uint32))
    sa, sb = a.gp_stats(), b.gp_stats()
    assert {k: sa[k] for k in STATS} == {k: sb[k] for k in STATS}
    assert _sites(a) == _sites(b)
    L = a.hi[0] - a.lo[0]
    nv, sp = (30, 30, 30), (L / 30,) * 3
    assert np.array_equal(a.gp_grain_map(a.lo, sp, nv), b.gp_grain_map(b.lo, sp, nv))


def test_resume_continues_the_saved_run():
    w = _polycrystal()
    a = _saved(w)
    a.gp_set_obstacle_store(2)       # FROZEN particles join the store every step
    a.gp_step(30)
    st = a.gp_stats()
    assert st["n_frozen"] > 0
    assert st["n_nucleated"] > 0 and st["n_nucleated"] < len(w.nuclei["pos"])  # some pending
    assert len(a.gp_inspect_order(1)["keys_sorted"]) > 0                       # obstacles
    ck = a.gp_save()
    info = native.checkpoint_check(ck)
    assert info == {"step": 30, "n_particles": st["n_live"]}
    b = _new(w)
    b.gp_load(ck)
    _same(a, b)                      # the loaded state itself
    a.gp_step(30)
    b.gp_step(30)
    assert a.gp_stats()["n_nucleated"] > st["n_nucleated"]
    _same(a, b)
    # a checkpoint of the resumed run equals one of the saved run, but for the order of
    # the particle records inside the store (all of b's started in the dynamic store)
    assert native.checkpoint_check(b.gp_save())["n_particles"] == a.gp_stats()["n_live"]
    a.close()
    b.close()


def test_resume_in_a_context_of_other_capacities():
    w = _polycrystal(seed=7)
    a = _saved(w)
    a.gp_step(25)
    b = _new(w, capacity=250000, reached_capacity=900000, claim_blocks=30000, max_grains=64,
             max_nuclei=40)
    b.gp_load(a.gp_save())
    a.gp_step(20)
    b.gp_step(20)
    _same(a, b)


def test_resume_in_the_middle_of_a_remelting_cycle():
    g = inputs.rng(21)
    h, T_L, L, dt = 2e-6, 1000.0, 50e-6, 1.3e-3
    w = inputs.Workload(name="remelt", lo=(0, 0, 0), hi=(L,) * 3, h=h, dt=dt, a=(1e-5,),
                        b=(2.0,), T_L=T_L, steps=45, seeds=g.random((10, 3)) * L,
                        quats=inputs.shoemake_quaternions(10, g),
                        analytic=dict(T0=T_L - 5.0, G=(0, 0, 0), xref=(0, 0, 0), Tdot=0.0))
    mem = dict(capacity=600000, reached_capacity=4000000, claim_blocks=60000, max_nuclei=16)
    a = _saved(w, **mem)
    a.gp_step(45)
    a.gp_set_melting(True)
    G, t0 = (0.0, 0.0, -3e5), 45 * dt
    a.gp_set_thermal_analytic(T_L - 5.0 - 400.0 * t0, G, (0.0, 0.0, L / 2), 400.0)
    a.gp_step(10)                    # heating: sites melt, particles walk back
    st = a.gp_stats()
    assert st["n_melted"] > 100 and st["n_walkback"] > 10
    b = _new(w, **mem)
    b.gp_load(a.gp_save())           # melting on and the heating field come with it
    _same(a, b)
    for s in (a, b):
        s.gp_step(10)
        s.gp_set_thermal_analytic(T_L - 5.0 + 400.0 * (t0 + 20 * dt), G, (0.0, 0.0, L / 2),
                                  -400.0)
        s.gp_step(30)                # quench and cooling: regrowth into the melt
    _same(a, b)


def test_resume_with_periodic_axes():
    w = _polycrystal(seed=9, n_nuclei=0)
    a = _saved(w)
    a.gp_set_periodic(3)
    a.gp_step(20)
    b = _new(w)
    b.gp_load(a.gp_save())
    a.gp_step(20)
    b.gp_step(20)
    _same(a, b)


def test_checkpoints_refused():
    w = _polycrystal(seed=11)
    a = _saved(w)
    a.gp_step(15)
    ck = a.gp_save()
    b = _new(w)

    def refused(data, status, ctx=b):
        with pytest.raises(native.GPError) as e:
            ctx.gp_load(data)
        assert e.value.status == status, str(e.value)

    bad = bytearray(ck)
    bad[len(bad) // 2] ^= 0x10           # one bit of the particle or site sections
    with pytest.raises(native.GPError):
        native.checkpoint_check(bytes(bad))
    refused(bytes(bad), 1)
    refused(ck[:-16], 1)                 # cut short
    refused(ck + bytes(16), 1)           # padded
    other = native.Sim(w.lo, (70e-6,) * 3, w.h, w.dt, w.a, w.b, w.T_L, max_grains=128, **MEM)
    refused(ck, 1, other)                # another domain
    other.close()
    small = _new(w, capacity=200)
    refused(ck, 2, small)                # the particles do not fit
    small.close()
    refused(ck, 5, a)                    # not a new context
    bt = native.Batch([(w.lo, w.hi)], w.h, w.dt, w.a, w.b, w.T_L, capacity=10_000,
                      max_grains=16, max_nuclei=16)
    with pytest.raises(native.GPError) as e:
        bt.gp_save()
    assert e.value.status == 5
    bt.close()
    b.gp_load(ck)                        # b is still new after the refusals
    a.gp_step(10)
    b.gp_step(10)
    _same(a, b)
