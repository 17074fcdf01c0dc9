"""Periodic axes (Sec. 3.4, reading r18) on the GPU: two grains meeting across the x
face of a periodic box, against the FP64 oracle (particles, contacts, reached sites,
grain map with nearest images), and against the same grains in a wider non-periodic
box with the second grain shifted by the period."""
import numpy as np
import pytest

from paper_2504_12858_gb300 import inputs
from tests.helpers import canon, keyset, oracle_from, sim_from

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _pair(periodic, steps=24):
    h, dT, T_L = 2e-6, 5.0, 1000.0
    dt = 0.37 * h / (1e-5 * dT ** 2)
    L = 60e-6
    g = inputs.rng(31)
    q = inputs.shoemake_quaternions(2, g)
    a = [52e-6, 30e-6, 30e-6]
    b = [6e-6 + (0.0 if periodic else L), 31e-6, 29e-6]
    return inputs.Workload(name="pair", lo=(0, 0, 0), hi=(L if periodic else 2 * L, 60e-6, 60e-6),
                           h=h, dt=dt, a=(1e-5,), b=(2.0,), T_L=T_L, steps=steps,
                           seeds=np.array([a, b]), quats=q,
                           analytic=dict(T0=T_L - dT, G=(0, 0, 0), xref=(0, 0, 0), Tdot=0.0))


def test_periodic_pair_matches_oracle_and_shifted_pair():
    w = _pair(True)
    o = oracle_from(w)
    o.set_periodic(1)
    s = sim_from(w, capacity=300000)
    s.gp_set_periodic(1)
    o.step(w.steps)
    s.gp_step(w.steps)
    p, q = canon(s.gp_get_particles()), canon(o.particles())
    assert keyset(p) == keyset(q)
    assert np.array_equal(p["state"], q["state"]) and (p["state"] == 1).sum() > 20
    assert np.allclose(p["ell"], q["ell"], atol=1e-4)
    assert s.gp_stats()["n_clipped"] == 0
    # the same two grains in a wider, non-periodic box, the second one shifted by L
    ww = _pair(False)
    sw = sim_from(ww, capacity=300000)
    sw.gp_step(ww.steps)
    pw = canon(sw.gp_get_particles())
    assert keyset(pw) == keyset(p)
    assert np.array_equal(pw["state"], p["state"])
    assert np.array_equal(pw["ell"].view(np.uint32), p["ell"].view(np.uint32))
    # grain map of the periodic box (voxels on both sides of the x face)
    nv, sp = (30, 30, 30), (2e-6,) * 3
    mo = o.grain_map((0, 0, 0), sp, nv)
    ms = s.gp_grain_map((0, 0, 0), sp, nv)
    assert (mo == ms).mean() >= 0.995
    assert (ms[:, :, 0] == 0).any() and (ms[:, :, -1] == 1).any()   # grains across the face
