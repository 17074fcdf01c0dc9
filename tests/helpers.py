"""Test helpers: set up the same workload on the oracle and on the CUDA library."""
import numpy as np

import oracle
from paper_2504_12858_gb300 import inputs


def oracle_from(w: inputs.Workload, nucleate=True):
    o = oracle.Oracle(w.lo, w.hi, w.h, w.dt, w.a, w.b, w.T_L)
    if w.analytic:
        o.set_thermal_analytic(w.analytic["T0"], w.analytic["G"], w.analytic["xref"],
                               w.analytic["Tdot"])
    if w.grid:
        o.set_thermal_grid(w.grid["T"], w.grid["origin"], w.grid["spacing"], w.grid["vel"])
    if w.solute:
        sd = w.solute
        o.set_solute_grid(sd["w"], sd["origin"], sd["spacing"], sd["Tm"], sd["mL"], sd["vel"])
    init = w.extra.get("particles") if w.extra else None
    if w.seeds is not None and len(w.seeds):
        o.add_grains(w.seeds, w.quats, nucleate=nucleate and not w.shell_n0 and init is None)
        if w.shell_n0:
            o.seed_shell(np.arange(len(w.seeds)), w.shell_n0)
    if init is not None:      # an initial state given as particles and lattice sites
        o.load_particles(init["grain"], init["site"], init["dir"],
                         init["ell"].astype(np.float64), init["state"])
        gr, sr = w.extra["reached"]
        o.add_reached(gr, sr)
        o.add_claimed(gr, sr)
        o.add_claimed(*w.extra["claimed"])
    if w.nuclei:
        o.nucleation_sites(w.nuclei["pos"], w.nuclei["dTn"], w.nuclei["quat"])
    return o


def sim_from(w: inputs.Workload, capacity, nucleate=True, **kw):
    from paper_2504_12858_gb300.native import Sim
    grid_nodes = int(np.prod(w.grid["T"].shape)) if w.grid else 0
    if w.solute:
        kw.setdefault("solute_nodes", int(np.prod(w.solute["w"].shape)))
    s = Sim(w.lo, w.hi, w.h, w.dt, w.a, w.b, w.T_L, capacity=capacity, grid_nodes=grid_nodes,
            max_grains=max(16, 2 * (len(w.seeds) if w.seeds is not None else 0) +
                           (len(w.nuclei["pos"]) if w.nuclei else 0)), **kw)
    if w.analytic:
        s.gp_set_thermal_analytic(w.analytic["T0"], w.analytic["G"], w.analytic["xref"],
                                  w.analytic["Tdot"])
    if w.grid:
        s.gp_set_thermal_grid(w.grid["T"], w.grid["origin"], w.grid["spacing"], w.grid["vel"])
    if w.solute:
        sd = w.solute
        s.gp_set_solute_grid(sd["w"], sd["origin"], sd["spacing"], sd["Tm"], sd["mL"], sd["vel"])
    init = w.extra.get("particles") if w.extra else None
    if w.seeds is not None and len(w.seeds):
        s.gp_add_grains(w.seeds, w.quats, nucleate=nucleate and not w.shell_n0 and init is None)
        if w.shell_n0:
            s.gp_seed_shell(np.arange(len(w.seeds)), w.shell_n0)
    if init is not None:      # an initial state given as particles and lattice sites
        s.gp_load_particles(init["grain"], init["site"], init["dir"], init["ell"], init["state"], 0)
        gr, sr = w.extra["reached"]
        s.gp_add_sites(gr, sr, reached=True, claimed=True)
        s.gp_add_sites(*w.extra["claimed"], reached=False, claimed=True)
    if w.nuclei:
        s.gp_nucleation_sites(w.nuclei["pos"], w.nuclei["dTn"], w.nuclei["quat"])
    return s


def canon(p):
    """Particles sorted by (grain, site, dir): a canonical order for set comparison."""
    key = np.lexsort((p["dir"], p["site"][:, 2], p["site"][:, 1], p["site"][:, 0], p["grain"]))
    return {k: v[key] for k, v in p.items()}


def keyset(p):
    return {(int(g), int(a), int(b), int(c), int(d)) for g, (a, b, c), d in
            zip(p["grain"], p["site"], p["dir"])}


def tip_signatures(p, n_grains):
    """Per grain, the sorted (site, dir, state) tuples of its primary tips, and the
    identity (grain, site, dir) of the highest particle."""
    from paper_2504_12858_gb300.adjoint import front_outputs
    _, _, on_axis, _, ih = front_outputs(p, 1.0, n_grains)
    sig = [[] for _ in range(n_grains)]
    for i in map(int, np.nonzero(on_axis)[0]):
        sig[int(p["grain"][i])].append((tuple(int(v) for v in p["site"][i]), int(p["dir"][i]),
                                        int(p["state"][i])))
    top = (int(p["grain"][ih]), tuple(int(v) for v in p["site"][ih]), int(p["dir"][ih]),
           int(p["state"][ih]))
    return [tuple(sorted(x)) for x in sig], top


def oracle_front_run(job):
    """Oracle front outputs (H, F), tip signatures and highest particle of the adjoint
    case for job = (theta, height, steps), theta = (A, n, G, Tdot) (runs in a worker
    process)."""
    from paper_2504_12858_gb300.adjoint import front_outputs
    (A, n, G, Tdot), height, steps = job
    w = inputs.adjoint_cube(A=A, n=n, G=G, Tdot=Tdot, height=height, steps=steps)
    o = oracle_from(w)
    o.step(w.steps)
    p = o.particles()
    H, F, _, _, _ = front_outputs(p, w.h, len(w.seeds))
    sig, top = tip_signatures(p, len(w.seeds))
    return H, F, sig, top


def nucleus_keys(sim, p, w):
    """Replaces the grain ids of particles p of context sim by the index of the
    grain's nucleus in workload w (columnar seeds first, then nucleation sites),
    matched by binary32 position; grain numbering then compares across contexts."""
    from paper_2504_12858_gb300 import native
    c3, _ = native.grain_table(sim)
    pts = []
    if w.seeds is not None:
        pts += [tuple(np.float32(v) for v in x) for x in w.seeds]
    if w.nuclei:
        pts += [tuple(np.float32(v) for v in x) for x in w.nuclei["pos"]]
    index = {}
    for i, t in enumerate(pts):
        index.setdefault(t, i)
    g2n = np.array([index.get(tuple(c), -1) for c in c3], np.int64)
    q = dict(p)
    q["grain"] = g2n[p["grain"]]
    return q


def gb_angle_deg(grain_map, spacing, y_range, left_ids, right_ids):
    """Angle (degrees, from the growth direction y) of the grain boundary between the
    grains left_ids (smaller x) and right_ids (larger x) in a 2D grain map indexed
    [y, x]: per row, the midpoint between the last left-group voxel and the next
    right-group voxel after it; a straight line is fitted over y_range.  Negative:
    the boundary moves towards -x (the right-hand grains overgrow the left-hand ones)."""
    left = np.isin(grain_map, left_ids)
    right = np.isin(grain_map, right_ids)
    ys, xs = [], []
    for j in range(grain_map.shape[0]):
        y = (j + 0.5) * spacing
        if not (y_range[0] <= y <= y_range[1]):
            continue
        li = np.nonzero(left[j])[0]
        if li.size == 0:
            continue
        k = li.max()
        ri = np.nonzero(right[j, k + 1:])[0]
        if ri.size == 0:
            continue
        xs.append((k + 0.5 + (k + 1 + ri[0] + 0.5)) / 2 * spacing)
        ys.append(y)
    if len(ys) < 5:
        return float("nan"), len(ys)
    slope = np.polyfit(ys, xs, 1)[0]
    return float(np.degrees(np.arctan(slope))), len(ys)
