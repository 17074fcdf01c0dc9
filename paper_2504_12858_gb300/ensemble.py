"""Set-up of a batch context from a list of run workloads (host-side marshalling).

Every run keeps its own domain, analytic field, columnar seeds and nucleation
sites; the runs share h, dt and the growth law.  All stepping happens in the
library's kernels (``native.Batch``).
"""
from __future__ import annotations

import numpy as np

from . import native
from .inputs import Workload


def batch_from(runs: list[Workload], capacity: int, reached_capacity: int = 0,
               claim_blocks: int = 0, stream=None, device="cuda",
               arena_fill=None) -> native.Batch:
    w0 = runs[0]
    for w in runs:
        if (w.h, w.dt, tuple(w.a), tuple(w.b), w.T_L) != (w0.h, w0.dt, tuple(w0.a), tuple(w0.b),
                                                          w0.T_L):
            raise ValueError("the runs of a batch share h, dt and the growth law")
        if not w.analytic or w.grid:
            raise ValueError("a batch takes analytic fields only")
    n_seed = sum(len(w.seeds) if w.seeds is not None else 0 for w in runs)
    n_nuc = sum(len(w.nuclei["pos"]) if w.nuclei else 0 for w in runs)
    b = native.Batch([(w.lo, w.hi) for w in runs], w0.h, w0.dt, w0.a, w0.b, w0.T_L,
                     capacity=capacity, reached_capacity=reached_capacity,
                     claim_blocks=claim_blocks, max_grains=n_seed + n_nuc + 16,
                     max_nuclei=n_nuc + 16, stream=stream, device=device,
                     arena_fill=arena_fill)
    for r, w in enumerate(runs):
        a = w.analytic
        b.gp_run_set_thermal_analytic(r, a["T0"], a["G"], a["xref"], a["Tdot"])
        if w.seeds is not None and len(w.seeds):
            b.gp_run_add_grains(r, w.seeds, w.quats, nucleate=True)
        if w.nuclei and len(w.nuclei["pos"]):
            b.gp_run_nucleation_sites(r, w.nuclei["pos"], w.nuclei["dTn"], w.nuclei["quat"])
    return b


def run_particles(sim, run: int) -> dict:
    """The particles of one run of a batch context (global grain ids)."""
    p = sim.gp_get_particles()
    _, grun = native.grain_table(sim)
    keep = grun[p["grain"]] == run
    return {k: v[keep] for k, v in p.items()}


def cells_bytes(runs: list[Workload]) -> float:
    """Approximate arena bytes of the dense per-run hash tables (cell table and
    reached-site heads: 1 + 1/16 bytes per hash cell)."""
    tot = 0.0
    for w in runs:
        e = w.h * (1 + 1 / 512)
        tot += float(np.prod([np.ceil((hi - lo) / e) for lo, hi in zip(w.lo, w.hi)]))
    return (1.0 + 1.0 / 16.0) * tot
