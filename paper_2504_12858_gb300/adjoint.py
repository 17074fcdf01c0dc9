"""Gradients of front positions with respect to the growth law and the imposed
field, through the hand-written adjoint of the particle advance (gp_adjoint).

Parameters theta = (A, n, G, Tdot) of v = A dT^n (Eq. 1) in the field
T = T0 + G (z - z_ref) - Tdot t (a cooling rate Tdot > 0).  Outputs:
  * front height H: the largest z of the live particles;
  * front position F_g of every grain: the mean distance of its primary tips (the
    points on the rotated <100> axes through the nucleus) from the nucleus.
Both are functions of the particles' progress ell given the discrete events of the
run, which the adjoint holds fixed.
"""
from __future__ import annotations

import numpy as np
import torch

from . import native


def _rotation(q):
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def front_outputs(p, h, n_grains):
    """(H, F[n_grains]) and their derivatives with respect to each particle's ell.

    p: particles (grain, site, dir, ell, x) of gp_get_particles or the oracle."""
    site, d = p["site"], p["dir"].astype(np.int64)
    ax = d // 2
    sg = np.where(d % 2 == 0, 1, -1)
    rows = np.arange(len(d))
    on_axis = (site[rows, ax] * sg >= 0) & (np.abs(site).sum(1) == np.abs(site[rows, ax]))
    dist = h * (np.abs(site[rows, ax]) + p["ell"].astype(np.float64))
    F = np.zeros(n_grains)
    nt = np.bincount(p["grain"][on_axis], minlength=n_grains)
    np.add.at(F, p["grain"][on_axis], dist[on_axis])
    F = F / np.maximum(nt, 1)
    ih = int(np.argmax(p["x"][:, 2]))
    return float(p["x"][ih, 2]), F, on_axis, nt, ih


class FrontAdjoint(torch.autograd.Function):
    """forward(theta, workload, capacity, every=1) -> tensor [H, F_0 .. F_{G-1}]
    (float64); every: the tape keeps the records of every every-th step and the reverse
    sweep rebuilds the others.

    The particles of the last forward run are kept in FrontAdjoint.last_particles."""

    last_particles = None

    @staticmethod
    def forward(ctx, theta, w, capacity, every=1):
        A, n, G, Tdot = (float(v) for v in theta.detach().cpu().numpy())
        an = w.analytic
        sim = native.Sim(w.lo, w.hi, w.h, w.dt, (A,), (n,), w.T_L, capacity=capacity,
                         reached_capacity=10 * capacity, max_grains=len(w.seeds) + 8,
                         tape_steps=w.steps, tape_checkpoint_every=every)
        sim.gp_set_thermal_analytic(an["T0"], (0.0, 0.0, G), an["xref"], -Tdot)
        sim.gp_add_grains(w.seeds, w.quats)
        sim.gp_tape_begin()
        sim.gp_step(w.steps)
        p = sim.gp_get_particles()
        FrontAdjoint.last_particles = p
        G_ = len(w.seeds)
        H, F, on_axis, nt, ih = front_outputs(p, w.h, G_)
        # d z / d ell of the highest particle: sigma * (h R)[2, axis]
        R = _rotation(w.quats[p["grain"][ih]])
        k = int(p["dir"][ih])
        ctx.sim, ctx.h, ctx.n = sim, w.h, len(p["grain"])
        ctx.dz_dell = (1 if k % 2 == 0 else -1) * w.h * R[2, k // 2]
        ctx.ih, ctx.on_axis, ctx.grain, ctx.nt = ih, on_axis, p["grain"], nt
        return torch.tensor(np.concatenate([[H], F]), dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        g = grad_out.detach().cpu().numpy().astype(np.float64)
        seed = np.zeros(ctx.n, np.float64)
        seed[ctx.ih] += g[0] * ctx.dz_dell
        ta = np.nonzero(ctx.on_axis)[0]
        gr = ctx.grain[ta]
        seed[ta] += g[1 + gr] * ctx.h / np.maximum(ctx.nt[gr], 1)
        d = ctx.sim.gp_adjoint(seed.astype(np.float32))
        # theta = (A, n, G, Tdot); the field's Tdot coefficient is -Tdot
        grad = torch.tensor([d[0], d[1], d[6], -d[7]], dtype=torch.float64)
        return grad, None, None, None
