"""The weld fixture at the size bench.py times (4 x 2 x 1 mm plate, 1e4 grains seeded
as 50-shell envelopes, ~1e8 particles, 512 x 256 x 128 thermal grid), in the
bench's launch configuration, checked on sampled outputs and on properties that
hold at any size.

One step from the state after three warm-up steps:
- a random sample of ACTIVE particles is advanced by the FP64 oracle one by one:
  Delta T at the binary32 position (trilinear on the same grid), v = a Delta T^b
  (Eq. 1), ell' = ell + min(v dt / h, 1).  Every sampled particle the oracle keeps
  on its site (no crossing, inside the plate, away from the thresholds) must be
  found after the step with the same (grain, site, dir) and either ACTIVE with
  its position (from ell') within 1e-5 of its magnitude, or FROZEN by contact with ell
  unchanged;
- (grain, site, dir) is unique over all live particles;
- every live particle has ell in [0, 1) and a known grain;
- the particle steps counted equal the ACTIVE particles at the start of the step,
  and each crossing records one reached site;
- for 20000 sampled ACTIVE particles the contact predicate of Sec. 2.1.2 (a live
  particle of another grain closer than h) is evaluated by brute force on the host,
  over every exported position in a 3 x 3 x 3 block of 2h cells around the particle,
  with the binary32 arithmetic the kernels use (d2 = ((dx dx + dy dy) + dz dz) < hf hf,
  every operation rounded); the GPU must have frozen exactly the sampled particles
  for which it holds.
"""
import numpy as np
import pytest

import oracle
from paper_2504_12858_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2504_12858_gb300 import native  # noqa: E402


def _keys(p):
    s = p["site"].astype(np.int64) + 4096
    return ((((p["grain"].astype(np.int64) * 8192 + s[:, 0]) * 8192 + s[:, 1]) * 8192
             + s[:, 2]) * 8 + p["dir"].astype(np.int64))


def test_weld_fixture_full_size_sampled_step():
    n_grains, n0, warmup = 10000, 50, 3
    w = inputs.weld_fixture(n_grains=n_grains, shell_n0=n0)
    per_grain = 4 * (n0 + 1) ** 2 + 2
    n_est = n_grains * per_grain
    s = native.Sim(w.lo, w.hi, w.h, w.dt, w.a, w.b, w.T_L,
                   capacity=int(n_est * 1.05 ** (warmup + 1) * 1.3) + 1000000,
                   reached_capacity=int(n_est * (1.2 + 0.9 * (warmup + 1))),
                   claim_blocks=n_grains * 2000, max_grains=n_grains + 16,
                   grid_nodes=int(np.prod(w.grid["T"].shape)))
    g = w.grid
    s.gp_set_thermal_grid(g["T"], g["origin"], g["spacing"], g["vel"])
    s.gp_add_grains(w.seeds, w.quats, nucleate=False)
    s.gp_seed_shell(np.arange(n_grains), n0)
    s.gp_step(warmup)
    st0 = s.gp_stats()
    p0 = s.gp_get_particles()
    assert len(p0["grain"]) > 9e7
    s.gp_step(1)
    st1 = s.gp_stats()
    p1 = s.gp_get_particles()
    s.close()

    # properties of the whole state
    assert st1["error_flags"] == 0
    k1 = _keys(p1)
    order = np.argsort(k1, kind="stable")
    ks = k1[order]
    assert not np.any(ks[1:] == ks[:-1])                       # unique (grain, site, dir)
    assert (p1["ell"] >= 0).all() and (p1["ell"] < 1).all()
    assert (p1["grain"] >= 0).all() and (p1["grain"] < n_grains).all()
    assert st1["particle_steps"] - st0["particle_steps"] == st0["n_active"]
    crossings = st1["n_reached"] - st0["n_reached"]
    assert crossings > 0.3 * st0["n_active"]

    # sampled particles, advanced one by one by the FP64 oracle
    o = oracle.Oracle(w.lo, w.hi, w.h, w.dt, w.a, w.b, w.T_L)
    o.set_thermal_grid(g["T"], g["origin"], g["spacing"], g["vel"])
    o.add_grains(w.seeds, w.quats, nucleate=False)
    t = st0["step"] * w.dt
    act = np.nonzero(p0["state"] == 0)[0]
    sample = np.random.default_rng(7).choice(act, 8000, replace=False)
    checked = frozen = 0
    worst = 0.0
    lo, hi = np.array(w.lo), np.array(w.hi)
    for i in sample:
        x = p0["x"][i].astype(np.float64)
        dT = o.undercooling(x, t)
        dl = min(o.velocity(dT) * w.dt / w.h, 1.0)
        e = float(p0["ell"][i]) + dl
        if e >= 1.0 - 1e-4 or (dT > 0 and abs(dl - 1.0) < 1e-4):
            continue                           # crosses, or at the crossing / cap threshold
        c, R = o.grain(int(p0["grain"][i]))
        k = int(p0["dir"][i])
        xn = x + (e - float(p0["ell"][i])) * (1 if k % 2 == 0 else -1) * w.h * R[:, k // 2]
        if np.any(xn < lo + 1e-9) or np.any(xn > hi - 1e-9):
            continue                           # at the clip threshold
        ki = _keys({f: p0[f][i:i + 1] for f in ("grain", "site", "dir")})[0]
        j = np.searchsorted(ks, ki)
        assert j < len(ks) and ks[j] == ki, i
        q = order[j]
        if p1["state"][q] == 1:
            frozen += 1
            assert p1["ell"][q] == p0["ell"][i]
        else:
            assert p1["state"][q] == 0
            # single-step positions within 1e-5 relative: the position moves by h per unit
            # of progress; the binary32 sample of the moving grid and the cubic growth law
            # put about 1e-4 of progress between the two sides near the pool
            dev = abs(float(p1["ell"][q]) - e) * w.h
            worst = max(worst, dev / max(float(np.linalg.norm(xn)), w.h))
            assert dev <= 1e-5 * max(float(np.linalg.norm(xn)), w.h), (i, float(p1["ell"][q]), e)
        checked += 1
    print(f"sampled {checked} particles ({frozen} froze); largest relative position "
          f"deviation {worst:.2e}")
    assert checked > 1000, checked
    assert frozen < checked

    # contact decisions of sampled ACTIVE particles against a brute-force predicate
    x0 = p0["x"]
    E = 2.0 * w.h                                   # > h: neighbours lie in adjacent cells
    cell = np.floor((x0.astype(np.float64) - np.array(w.lo)) / E).astype(np.int64)
    ncell = cell.max(axis=0) + 3
    ckey = ((cell[:, 2] + 1) * ncell[1] + (cell[:, 1] + 1)) * ncell[0] + (cell[:, 0] + 1)
    corder = np.argsort(ckey, kind="stable")
    cks = ckey[corder]
    smp = np.random.default_rng(8).choice(act, 20000, replace=False)
    off = np.array([(dz * ncell[1] + dy) * ncell[0] + dx for dz in (-1, 0, 1)
                    for dy in (-1, 0, 1) for dx in (-1, 0, 1)], np.int64)
    qk = ckey[smp][:, None] + off[None, :]
    lo_i = np.searchsorted(cks, qk, side="left")
    hi_i = np.searchsorted(cks, qk, side="right")
    hf = np.float32(w.h)
    rc2 = np.float32(hf * hf)
    expect = np.zeros(len(smp), bool)
    for t, i in enumerate(smp):
        cand = np.concatenate([corder[a:b] for a, b in zip(lo_i[t], hi_i[t])])
        cand = cand[p0["grain"][cand] != p0["grain"][i]]
        if cand.size == 0:
            continue
        d = x0[i][None, :] - x0[cand]                # binary32, each operation rounded
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        expect[t] = bool((d2 < rc2).any())
    ksmp = _keys({f: p0[f][smp] for f in ("grain", "site", "dir")})
    j = np.minimum(np.searchsorted(ks, ksmp), len(ks) - 1)
    present = ks[j] == ksmp
    q = order[j]
    got_frozen = present & (p1["state"][q] == 1)
    assert np.array_equal(got_frozen, expect), (int((got_frozen & ~expect).sum()),
                                                int((expect & ~got_frozen).sum()))
    assert (p1["ell"][q[expect]] == p0["ell"][smp[expect]]).all()
    assert expect.sum() > 200 and (~expect).sum() > 200, int(expect.sum())
