"""Failure paths of the library, driven without a GPU fault.

Every device-side wait of the library is bounded and every table has a capacity;
running out of either sets a sticky device error bit that the host turns into a
status, and the host refuses bad arguments before any device work.  These tests
provoke each case on purpose, in forms that fault, trap or hang nothing:
- the claim-block pool of the lattice-site claim table too small for the run:
  GP_ERR_HASH_FULL from gp_step, and the context refuses further steps;
- each bounded wait (the radix sort's look-back, the claim table's slot wait) run
  by gp_selftest_wait on a word that nothing publishes: GP_ERR_TIMEOUT within its
  poll limit, and the device stays usable;
- zero or non-finite quaternions, non-finite nucleation data and degenerate
  thermal grids: GP_ERR_ARG, with the context still usable;
- a particle store too small: GP_ERR_CAPACITY;
- results that do not depend on what the device memory held before the library
  initialised it: the arena filled with 0x00, 0xFF or 0xA5 bytes gives bit-identical
  particles, reached sites, counters and grain maps, in a single run and in a batch
  (the stand-in for the poison-filled buffers of a memory checker, which is closed on
  this pool).
"""
import math
import time

import numpy as np
import pytest

from paper_2504_12858_gb300 import ensemble, inputs
from tests.helpers import canon, sim_from

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2504_12858_gb300 import build, native  # noqa: E402

build.build()
native.load()

GP_ERR_ARG, GP_ERR_CAPACITY, GP_ERR_HASH_FULL, GP_ERR_TIMEOUT = 1, 2, 3, 6


def _small_sim(**kw):
    w = inputs.single_grain()
    return w, sim_from(w, capacity=kw.pop("capacity", 200000), **kw)


def test_claim_pool_exhausted_is_hash_full():
    # the nucleus and its six first targets take four 8^3-site blocks; a grain
    # growing past eight lattice shells needs more than eight blocks
    w, s = _small_sim(claim_blocks=8)
    with pytest.raises(native.GPError) as e:
        s.gp_step(200)
    assert e.value.status == GP_ERR_HASH_FULL
    assert s.gp_stats()["error_flags"] & 2          # the sticky device bit
    with pytest.raises(native.GPError):
        s.gp_step(1)                                # the context stays in the error state
    s.close()
    # a fresh context on the same device works
    w, s2 = _small_sim()
    s2.gp_step(5)
    assert s2.gp_stats()["error_flags"] == 0


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_waits_give_up_and_report_timeout(which):
    for limit in (1, 1000, 200000):
        t0 = time.perf_counter()
        st = native.gp_selftest_wait(which, limit)
        assert st == GP_ERR_TIMEOUT, (which, limit, st)
        assert time.perf_counter() - t0 < 30.0
    assert native.gp_selftest_wait(which, 0) == GP_ERR_ARG
    assert native.gp_selftest_wait(2, 10) == GP_ERR_ARG
    # the device is still usable: a short run gives its usual result
    w, s = _small_sim()
    s.gp_step(20)
    st = s.gp_stats()
    assert st["error_flags"] == 0 and st["n_live"] > 6


@pytest.mark.parametrize("q", [(0.0, 0.0, 0.0, 0.0), (math.nan, 0.0, 0.0, 1.0),
                               (1.0, math.inf, 0.0, 0.0)])
def test_bad_quaternions_are_refused(q):
    w, s = _small_sim()
    n0 = s.gp_stats()["n_grains"]
    with pytest.raises(native.GPError) as e:
        s.gp_add_grains(np.array([[50e-6, 50e-6, 50e-6]]), np.array([q]))
    assert e.value.status == GP_ERR_ARG
    with pytest.raises(native.GPError) as e:
        s.gp_nucleation_sites(np.array([[50e-6, 50e-6, 50e-6]]), np.array([1.0]), np.array([q]))
    assert e.value.status == GP_ERR_ARG
    # nothing was added and the context still steps
    assert s.gp_stats()["n_grains"] == n0
    s.gp_step(3)
    assert s.gp_stats()["error_flags"] == 0


def test_non_finite_nucleation_data_is_refused():
    w, s = _small_sim()
    q = inputs.shoemake_quaternions(1, inputs.rng(3))
    for pos, dtn in [((math.nan, 1e-5, 1e-5), 1.0), ((1e-5, 1e-5, 1e-5), math.inf)]:
        with pytest.raises(native.GPError) as e:
            s.gp_nucleation_sites(np.array([pos]), np.array([dtn]), q)
        assert e.value.status == GP_ERR_ARG


@pytest.mark.parametrize("shape,spacing", [((1, 4, 4), (1e-6,) * 3), ((4, 4, 4), (1e-6, 0.0, 1e-6)),
                                           ((4, 4, 4), (1e-6, math.nan, 1e-6))])
def test_degenerate_thermal_grids_are_refused(shape, spacing):
    w, s = _small_sim()
    T = np.full(shape, 990.0, np.float32)
    with pytest.raises(native.GPError) as e:
        s.gp_set_thermal_grid(T, (0, 0, 0), spacing)
    assert e.value.status == GP_ERR_ARG
    s.gp_step(2)                                     # the analytic field stays in force
    assert s.gp_stats()["error_flags"] == 0


def test_particle_store_too_small_is_capacity():
    w, s = _small_sim(capacity=1000)
    with pytest.raises(native.GPError) as e:
        s.gp_step(200)
    assert e.value.status == GP_ERR_CAPACITY


def _poly(seed, L=60e-6, n_nuclei=30):
    g = inputs.rng(seed)
    T_L = 1000.0
    return inputs.Workload(name="poly", lo=(0, 0, 0), hi=(L,) * 3, h=2e-6, dt=1.3e-3, a=(1e-5,),
                           b=(2.0,), T_L=T_L, steps=40, seeds=g.random((12, 3)) * L,
                           quats=inputs.shoemake_quaternions(12, g),
                           analytic=dict(T0=T_L - 4.0, G=(3e4, -2e4, 1e4), xref=(L / 2,) * 3,
                                         Tdot=-20.0),
                           nuclei=dict(pos=g.random((n_nuclei, 3)) * L,
                                       dTn=4.0 + 1.5 * g.random(n_nuclei),
                                       quat=inputs.shoemake_quaternions(n_nuclei, g)))


def _bits(p):
    p = canon(p)
    return {k: (v.view(np.uint32) if v.dtype == np.float32 else v) for k, v in p.items()}


def _equal_particles(pa, pb):
    assert pa.keys() == pb.keys()
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k


MEM = dict(capacity=400000, reached_capacity=2000000, claim_blocks=60000)


@pytest.mark.parametrize("fill", [0xFF, 0xA5])
def test_results_do_not_depend_on_the_arena_contents(fill):
    w = _poly(5)
    out = []
    for f in (0x00, fill):
        s = sim_from(w, arena_fill=f, **MEM)
        s.gp_step(40)
        g, x = s.gp_get_reached()
        out.append((_bits(s.gp_get_particles()), s.gp_stats(),
                    s.gp_grain_map((0, 0, 0), (2e-6,) * 3, (30, 30, 30)),
                    sorted(zip(g.tolist(), map(tuple, x.tolist())))))
        s.close()
    (pa, sa, ma, ra), (pb, sb, mb, rb) = out
    assert sa["n_nucleated"] > 0 and sa["n_frozen"] > 0
    _equal_particles(pa, pb)
    assert sa == sb
    assert np.array_equal(ma, mb)
    assert ra == rb


def test_batch_results_do_not_depend_on_the_arena_contents():
    runs = [_poly(6), _poly(7)]
    out = []
    for f in (0x00, 0xFF):
        b = ensemble.batch_from(runs, arena_fill=f, **MEM)
        b.gp_step(40)
        out.append(([_bits(ensemble.run_particles(b, r)) for r in range(len(runs))],
                    b.gp_stats()))
        b.close()
    (pa, sa), (pb, sb) = out
    assert sa["n_nucleated"] > 0
    for a, c in zip(pa, pb):
        _equal_particles(a, c)
    assert sa == sb
