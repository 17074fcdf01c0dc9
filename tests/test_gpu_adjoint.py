"""Hand-written adjoint of the advance (GPU) against central finite differences of the
FP64 oracle.

Case: 200 um cube, 32 grains (seed 5), v = A dT^n, T = T_L - 5 + G (z - z_c) - Tdot t,
theta = (A, n, G, Tdot) = (1e-5, 2, 1e3 K/m, 10 K/s), h = 2 um, dt = 2 ms, 200 steps;
and the same grains in a box 400 um tall, where the highest point of the envelope
grows freely (182 steps).  Outputs: every grain's mean primary-tip distance F_g, and the front
height H (the largest z).  Each parameter is perturbed by 1e-4 relative.  The adjoint
holds the discrete events of the run fixed, so an output is compared only when the
events that shape it are the same in the minus, base and plus oracle runs and in the
binary32 GPU run: for F_g, the (site, direction, state) of the grain's tips; for H,
the identity of the highest particle, which must be ACTIVE.  An event can also move in
time without changing these (a tip freezing one step earlier at the same site), which
makes the output jump on one side of the base run; such outputs fail the symmetry
test |F+ - 2 F0 + F-| <= 1e-2 |F+ - F-| that a smooth output passes by orders of
magnitude (its second-order term is about 1e-4 of the first).  Excluded outputs are
reported.  Bar: 1e-3 relative.  In the tall box the front height is compared for all
four parameters.

The tape can keep the particle records of every k-th step only; the reverse sweep
then rebuilds the others by replaying the taped events.  The gradients with k = 10
and k = 7 equal those with k = 1 (up to the order of the floating-point atomics).
"""
import multiprocessing as mp

import numpy as np
import pytest

from tests.helpers import oracle_front_run, tip_signatures

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

THETA0 = np.array([1e-5, 2.0, 1e3, 10.0])
REL = 1e-4
# (box height, steps): the cube, and the tall box stopped at a step where one tip leads
# the envelope's nearly flat top face by 0.37 h and lies between two sites (progress
# 0.73).  The front height max z has a kink wherever two particles tie in z or the
# highest one crosses a site; at most other steps the lead is about 0.02 h and a relative
# change of 1e-4 of the exponent n moves the maximum to another particle.
CASES = ((200e-6, 200), (400e-6, 182))


@pytest.fixture(scope="module")
def finite_differences():
    jobs = []
    for height, steps in CASES:
        jobs.append((THETA0.copy(), height, steps))
        for p in range(4):
            for sgn in (1, -1):
                t = THETA0.copy()
                t[p] *= 1 + sgn * REL
                jobs.append((t, height, steps))
    with mp.get_context("spawn").Pool(min(len(jobs), max(1, mp.cpu_count()))) as pool:
        res = pool.map(oracle_front_run, jobs)
    return {case: res[9 * i: 9 * (i + 1)] for i, case in enumerate(CASES)}


def _gpu_jacobian(height, steps, every=1):
    from paper_2504_12858_gb300 import build, inputs, native
    from paper_2504_12858_gb300.adjoint import FrontAdjoint
    build.build()
    native.load()
    w = inputs.adjoint_cube(height=height, steps=steps)
    G = len(w.seeds)
    th = torch.tensor(THETA0, dtype=torch.float64, requires_grad=True)
    out = FrontAdjoint.apply(th, w, 400000, every)
    jac = np.stack([torch.autograd.grad(out[i], th, retain_graph=True)[0].numpy()
                    for i in range(1 + G)])            # d(H, F_0..F_G-1)/d theta
    return w, out.detach().numpy(), jac, FrontAdjoint.last_particles


@pytest.mark.parametrize("case", CASES)
def test_adjoint_gradients_match_oracle_central_differences(finite_differences, case):
    height, steps = case
    w, out, jac, parts = _gpu_jacobian(height, steps)
    G = len(w.seeds)
    gpu_sig, gpu_top = tip_signatures(parts, G)
    fd_runs = finite_differences[case]
    base = fd_runs[0]
    assert abs(out[0] - base[0]) <= 1e-5 * abs(base[0])
    compared, excluded, h_compared = 0, 0, 0
    for p in range(4):
        plus, minus = fd_runs[1 + 2 * p], fd_runs[2 + 2 * p]
        step = 2 * REL * THETA0[p]
        for g in range(G):
            same = plus[2][g] == minus[2][g] == base[2][g] == gpu_sig[g] and bool(base[2][g])
            smooth = (abs(plus[1][g] - 2 * base[1][g] + minus[1][g])
                      <= 1e-2 * abs(plus[1][g] - minus[1][g]))
            if not (same and smooth):
                excluded += 1
                continue
            fd = (plus[1][g] - minus[1][g]) / step
            scale = max(abs(fd), 1e-6 * base[1][g] / THETA0[p])
            assert abs(jac[1 + g, p] - fd) <= 1e-3 * scale, (p, g, jac[1 + g, p], fd)
            compared += 1
        if (plus[3] == minus[3] == base[3] == gpu_top and base[3][3] == 0
                and abs(plus[0] - 2 * base[0] + minus[0]) <= 1e-2 * abs(plus[0] - minus[0])):
            fd = (plus[0] - minus[0]) / step
            scale = max(abs(fd), 1e-6 * base[0] / THETA0[p])
            assert abs(jac[0, p] - fd) <= 1e-3 * scale, (p, "H", jac[0, p], fd)
            compared += 1
            h_compared += 1
        else:
            excluded += 1
    print(f"adjoint vs finite differences (box height {height * 1e6:.0f} um): {compared} "
          f"outputs compared ({h_compared} of the front height), {excluded} excluded")
    assert compared >= 2 * G
    if height > 200e-6:
        assert h_compared == 4                 # d H / d (A, n, G, Tdot), H ACTIVE


@pytest.mark.parametrize("every", [10, 7])
def test_checkpointed_tape_gives_the_same_gradients(every):
    _, out1, jac1, p1 = _gpu_jacobian(*CASES[1], 1)
    _, outk, jack, pk = _gpu_jacobian(*CASES[1], every)
    # the same forward run (its outputs are float64 sums in store order, which varies)
    assert np.allclose(out1, outk, rtol=1e-12, atol=0)
    scale = np.maximum(np.abs(jac1), 1e-12 + 1e-6 * np.abs(jac1).max(axis=0, keepdims=True))
    assert (np.abs(jack - jac1) <= 1e-5 * scale).all(), np.abs(jack - jac1).max()
