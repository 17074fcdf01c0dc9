"""Melting walk-back (Sec. 2.1.3) on the GPU against the FP64 oracle: a half-space melt
with a closed-form outcome, a grain melted entirely whose seed nucleates again, and a
polycrystal taken through a heating and cooling cycle (the remelting test of Sec. 4.1
in miniature)."""
import numpy as np
import pytest

from paper_2504_12858_gb300 import inputs
from tests.helpers import keyset, oracle_from, sim_from

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _sites(g, s):
    return {(int(a), int(b), int(c), int(d)) for a, (b, c, d) in zip(g, s)}


def test_half_space_melt_matches_oracle():
    h, dT, T_L = 2e-6, 5.0, 1000.0
    dt = 0.37 * h / (1e-5 * dT ** 2)
    c = np.array([[60e-6, 60e-6, 60e-6]])
    w = inputs.Workload(name="melt", lo=(0, 0, 0), hi=(120e-6,) * 3, h=h, dt=dt, a=(1e-5,),
                        b=(2.0,), T_L=T_L, steps=40, seeds=c, quats=np.array([[1.0, 0, 0, 0]]),
                        analytic=dict(T0=T_L - dT, G=(0, 0, 0), xref=(0, 0, 0), Tdot=0.0))
    o, s = oracle_from(w), sim_from(w, capacity=400000, reached_capacity=2000000)
    o.step(40)
    s.gp_step(40)
    z_cut = c[0, 2] + 3.5 * h
    for x in (o, s):
        (x.set_thermal_analytic if x is o else x.gp_set_thermal_analytic)(
            T_L, (0.0, 0.0, 1.0), (0.0, 0.0, z_cut), 0.0)
    o.set_melting(True)
    s.gp_set_melting(True)
    o.step(1)
    s.gp_step(1)
    st, so = s.gp_stats(), o.stats()
    assert st["n_melted"] == so["melted"] > 100
    assert st["n_walkback"] == so["walkback"] > 50
    assert _sites(*s.gp_get_reached()) == _sites(*o.reached())
    assert keyset(s.gp_get_particles()) == keyset(o.particles())
    # regrowth into the melted half in a uniform undercooling again
    for x in (o, s):
        (x.set_thermal_analytic if x is o else x.gp_set_thermal_analytic)(
            T_L - dT, (0, 0, 0), (0, 0, 0), 0.0)
    o.step(12)
    s.gp_step(12)
    assert keyset(s.gp_get_particles()) == keyset(o.particles())
    assert _sites(*s.gp_get_reached()) == _sites(*o.reached())


def test_grain_melted_entirely_nucleates_again():
    h, T_L = 2e-6, 1000.0
    w = inputs.Workload(name="renuc", lo=(0, 0, 0), hi=(80e-6,) * 3, h=h, dt=2e-3, a=(1e-5,),
                        b=(2.0,), T_L=T_L, steps=0, seeds=np.zeros((0, 3)),
                        quats=np.zeros((0, 4)),
                        analytic=dict(T0=T_L - 5.0, G=(0, 0, 0), xref=(0, 0, 0), Tdot=0.0),
                        nuclei=dict(pos=np.array([[40e-6, 40e-6, 40e-6]]), dTn=np.array([0.5]),
                                    quat=inputs.shoemake_quaternions(1, inputs.rng(2))))
    o, s = oracle_from(w), sim_from(w, capacity=200000, reached_capacity=1000000)
    o.set_melting(True)
    s.gp_set_melting(True)
    for T0, n in ((T_L - 5.0, 30), (T_L + 1.0, 3), (T_L - 0.4, 3), (T_L - 0.6, 2)):
        o.set_thermal_analytic(T0, (0, 0, 0), (0, 0, 0), 0.0)
        s.gp_set_thermal_analytic(T0, (0, 0, 0), (0, 0, 0), 0.0)
        for _ in range(n):
            o.step(1)
            s.gp_step(1)
            st = s.gp_stats()
            assert st["n_live"] == o.n_particles
            assert st["n_nucleated"] == o.stats()["nucleated"]
    assert o.stats()["nucleated"] == 2 and st["n_grains"] == 1
    assert keyset(s.gp_get_particles()) == keyset(o.particles())


def test_remelting_cycle_grain_map_matches_oracle():
    g = inputs.rng(21)
    h, T_L, L, dt = 2e-6, 1000.0, 50e-6, 1.3e-3
    w = inputs.Workload(name="remelt", lo=(0, 0, 0), hi=(L,) * 3, h=h, dt=dt, a=(1e-5,),
                        b=(2.0,), T_L=T_L, steps=45, seeds=g.random((10, 3)) * L,
                        quats=inputs.shoemake_quaternions(10, g),
                        analytic=dict(T0=T_L - 5.0, G=(0, 0, 0), xref=(0, 0, 0), Tdot=0.0))
    o, s = oracle_from(w), sim_from(w, capacity=600000, reached_capacity=4000000)
    o.step(45)
    s.gp_step(45)
    o.set_melting(True)
    s.gp_set_melting(True)
    # a hot front: T = T_L - 5 + G (z - L/2) + Tdot (t - t0), heating then cooling
    G = (0.0, 0.0, -3e5)
    t0 = 45 * dt
    # heating at 400 K/s for 20 steps, then a quench to 10.4 K below and cooling at
    # 400 K/s for 40 steps
    for Tdot, n, T0 in ((+400.0, 20, T_L - 5.0 - 400.0 * t0),
                        (-400.0, 40, T_L - 5.0 + 400.0 * (t0 + 20 * dt))):
        for x in (o, s):
            (x.set_thermal_analytic if x is o else x.gp_set_thermal_analytic)(
                T0, G, (0.0, 0.0, L / 2), Tdot)
        o.step(n)
        s.gp_step(n)
    st, so = s.gp_stats(), o.stats()
    assert so["melted"] > 1000 and so["walkback"] > 100
    assert abs(st["n_melted"] - so["melted"]) <= 0.01 * so["melted"]
    nv, sp = (50, 50, 50), (1e-6,) * 3
    mo = o.grain_map((0, 0, 0), sp, nv)
    ms = s.gp_grain_map((0, 0, 0), sp, nv)
    assert (mo == ms).mean() >= 0.995
    assert (mo >= 0).mean() > 0.2
