"""Directional solidification of a quasi-2D thin sample (Sec. 3.3, Table S2): fifteen
nuclei in three orientation groups (psi = 4, 30 and 11 deg) grow up a frozen
temperature gradient, and the better-oriented 11-deg grains overgrow the central
30-deg grains.  The grain-boundary angle between the two groups is measured on the
grain map at mid-thickness.

On the GPU at lambda_0 = 24 um the grain map matches the oracle's and the boundary
angles agree; at lambda_0 = 12 um the angle has converged to within 3 deg of the
24 um one.  The paper quotes an experimental angle of about 19 deg, approached by
its model for lambda_0 <= 48 um; under the readings of this implementation the
angle converges to about 16-17 deg (oracle: 9.8, 10.0, 16.8 and 16.0 deg at
lambda_0 = 96, 48, 24 and 12 um).  That comparison with the paper is not pinned.
"""
import numpy as np
import pytest

from paper_2504_12858_gb300 import inputs
from tests.helpers import gb_angle_deg, oracle_from, sim_from

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

CENTRAL, RIGHT = list(range(3, 12)), [12, 13, 14]   # psi = 30 deg, psi = 11 deg


def _map(x, w):
    lam = w.h
    sp = min(lam / 2, 12e-6)
    Lx, Ly, Lz = w.hi
    nv = (int(Lx / sp), int(Ly / sp), 1)
    org = (0.0, 0.0, Lz / 2 - sp / 2)
    m = (x.grain_map(org, (sp,) * 3, nv) if hasattr(x, "grain_map")
         else x.gp_grain_map(org, (sp,) * 3, nv))
    return m[0], sp


def test_thin_sample_grain_boundary_angle():
    w = inputs.thin_sample(24e-6)
    o, s = oracle_from(w), sim_from(w, capacity=400000, reached_capacity=4000000)
    o.step(w.steps)
    s.gp_step(w.steps)
    mo, sp = _map(o, w)
    ms, _ = _map(s, w)
    assert (mo == ms).mean() >= 0.995
    ao, no = gb_angle_deg(mo, sp, (0.1e-3, 0.85e-3), CENTRAL, RIGHT)
    a24, n24 = gb_angle_deg(ms, sp, (0.1e-3, 0.85e-3), CENTRAL, RIGHT)
    assert no >= 30 and n24 >= 30
    assert abs(a24 - ao) < 1.5, (a24, ao)
    assert -25.0 < a24 < -10.0, a24            # the 11-deg grains overgrow the 30-deg ones

    w12 = inputs.thin_sample(12e-6)
    s12 = sim_from(w12, capacity=1500000, reached_capacity=20000000)
    s12.gp_step(w12.steps)
    m12, sp12 = _map(s12, w12)
    a12, n12 = gb_angle_deg(m12, sp12, (0.1e-3, 0.85e-3), CENTRAL, RIGHT)
    assert n12 >= 60
    assert abs(a12 - a24) < 3.0, (a12, a24)
    print(f"grain-boundary angle: {a24:.1f} deg (24 um), {a12:.1f} deg (12 um); "
          f"oracle {ao:.1f} deg (24 um)")
