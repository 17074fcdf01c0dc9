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
- a particle store too small: GP_ERR_CAPACITY.
"""
import math
import time

import numpy as np
import pytest

from paper_2504_12858_gb300 import inputs
from tests.helpers import sim_from

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
