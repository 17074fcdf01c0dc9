#!/usr/bin/env python3
"""Throughput of the grain-envelope particle step on GB300.

Workload (largest configuration, one GPU): a 4 x 2 x 1 mm plate with a 1 kW,
1 m/min Rosenthal moving point source tabulated on a 512 x 256 x 128 binary32
grid (sampled trilinearly in the source frame), 1e4 grains at uniform random
seeds with uniform random orientations, each seeded as an octahedral envelope
of 50 lattice shells (about 1e8 particles), v = 3e-6 dT^3, h = 2 um, dt = 0.1 ms.
A step is one pass of the whole hot path (hash + sort, contact, thermal sample,
growth law, advance, spawn/claim, clip, compaction, nucleation check) over all
particles.  Metric: particle-steps/s = ACTIVE particles at the start of each
timed step, summed, divided by the device time of the timed steps.

Multi-GPU (torchrun): every rank runs an independent replica of the workload
(weak scaling, no collective in the data path); the timed region is bracketed by
barriers and the maximum time over ranks is used.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the first grains of the fixture) on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD_NAME = ("weld_fixture: 4x2x1 mm plate, Rosenthal 1 kW 1 m/min on a 512x256x128 FP32 "
                 "grid, 1e4 grains seeded as 50-shell octahedral envelopes (~1e8 particles), "
                 "v = 3e-6 dT^3, h = 2 um, dt = 0.1 ms")
METRIC = "particle-steps/s"


# ----------------------------------------------------------------------------------
# distributed plumbing (host logic, tested on CPU with gloo)
# ----------------------------------------------------------------------------------
def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_timing(local_ms: float, local_units: float, world: int):
    """Max of the timed region over ranks and the sum of the work of all ranks."""
    if world <= 1:
        return local_ms, local_units
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        smax = max(r["smax"] for r in rows)
        load = [r for r in rows if r["sm"] > 0.3 * smax] or rows
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                            ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": smax,
                "samples": len(rows), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------------
# workload construction
# ----------------------------------------------------------------------------------
def fixture(n_grains: int, n0: int, plate_mm=(4.0, 2.0, 1.0)):
    from paper_2504_12858_gb300 import inputs
    return inputs.weld_fixture(n_grains=n_grains, shell_n0=n0,
                               extent=tuple(v * 1e-3 for v in plate_mm))


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_sources_digest():
    """Digest of the CUDA sources with comments and blank space removed, so that the
    committed ncu figures stay valid across edits that change no code."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2504_12858_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        text = open(os.path.join(csrc, f), encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(f.encode())
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per unit of `kernel` from the committed ncu summary, if it was taken
    on the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    if d.get("sources_digest") != kernel_sources_digest():
        return None
    k = d.get("kernels", {}).get(kernel)
    return None if k is None else float(k["dram_bytes_per_unit"])


def ncu_issue(kernel: str):
    """Share of the issue slots busy in `kernel` (ncu smsp__issue_active, small-case
    capture of the same sources), if recorded for the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    if d.get("sources_digest") != kernel_sources_digest():
        return None
    k = d.get("kernels", {}).get(kernel, {})
    return None if "issue_slots_busy" not in k else float(k["issue_slots_busy"])


def ncu_step_traffic():
    """DRAM bytes per particle-step of the whole step (every step kernel), from the
    committed one-pass ncu capture of the default bench's timed steps, if it was taken
    on the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    if d.get("sources_digest") != kernel_sources_digest() or "step" not in d:
        return None
    return float(d["step"]["dram_bytes_per_particle_step"])


# algorithmic bytes of one particle-step for the whole step: read and write the
# 16-byte record, write and read back the 8-byte (cell key, index) pair
B_ALG_STEP = 48


# ----------------------------------------------------------------------------------
# CPU oracle on a bounded sample (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------------
def oracle_sample(n_grains_sample: int, n0: int):
    import oracle
    w = fixture(10000, n0)
    o = oracle.Oracle(w.lo, w.hi, w.h, w.dt, w.a, w.b, w.T_L)
    g = w.grid
    o.set_thermal_grid(g["T"], g["origin"], g["spacing"], g["vel"])
    o.add_grains(w.seeds[:n_grains_sample], w.quats[:n_grains_sample], nucleate=False)
    o.seed_shell(np.arange(n_grains_sample), n0)
    return o


def time_oracle(o, steps: int):
    before = o.stats()["particle_steps"]
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return (o.stats()["particle_steps"] - before) / dt, dt


def cpu_baseline(n_grains_sample=100, n0=50, steps=2):
    o = oracle_sample(n_grains_sample, n0)
    o.step(1)  # warm the allocator
    rate, dt = time_oracle(o, steps)
    return {"value": rate, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": (f"first {n_grains_sample} of the 1e4 grains of the same workload "
                       f"(~{o.n_particles:.2e} particles), {steps} steps after 1 untimed step, "
                       f"{dt:.1f} s of single-threaded FP64 work")}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    o = oracle_sample(args.ref_grains, args.n0)
    o.step(args.warmup)
    rate, dt = time_oracle(o, args.steps)
    cb = {"value": rate, "unit": METRIC, "cores": 1, "kind": "oracle",
          "sample": (f"first {args.ref_grains} of the 1e4 grains of the same workload, "
                     f"{args.steps} timed steps after {args.warmup} warm-up steps")}
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": METRIC,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "sample_grains": args.ref_grains},
            "cpu_baseline": cb,
            "e2e": {"value": rate, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------
def adjoint_cost(dev):
    """Cost of the gradient of the front positions (forward with the adjoint tape +
    reverse sweep) over the plain forward, on the 32-grain calibration cube
    (200 steps)."""
    import torch
    from paper_2504_12858_gb300 import inputs, native
    from paper_2504_12858_gb300.adjoint import FrontAdjoint
    w = inputs.adjoint_cube()
    an = w.analytic

    def plain():
        sim = native.Sim(w.lo, w.hi, w.h, w.dt, w.a, w.b, w.T_L, capacity=400000,
                         reached_capacity=1600000, max_grains=64, device=dev)
        sim.gp_set_thermal_analytic(an["T0"], an["G"], an["xref"], an["Tdot"])
        sim.gp_add_grains(w.seeds, w.quats)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        sim.gp_step(w.steps)
        torch.cuda.synchronize(dev)
        t = time.perf_counter() - t0
        sim.close()
        return t

    def with_gradient():
        th = torch.tensor([w.a[0], w.b[0], an["G"][2], -an["Tdot"]], dtype=torch.float64,
                          requires_grad=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        out = FrontAdjoint.apply(th, w, 400000)
        out[1:].sum().backward()
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t0

    plain()
    with_gradient()
    tp = min(plain() for _ in range(3))
    tg = min(with_gradient() for _ in range(3))
    return {"case": "adjoint_cube: 200 um cube, 32 grains, 200 steps", "plain_forward_ms": tp * 1e3,
            "forward_with_tape_plus_backward_ms": tg * 1e3, "cost_ratio": tg / tp}


def run_cost(w) -> float:
    """Relative work of one ensemble run for sharding: the envelope area grows with
    the growth distance squared (v ~ dT^2 with dT ~ Tdot t) and the number of
    grains with the volume, so cost ~ L^3 Tdot^4 (plus a constant per run)."""
    L = w.hi[0] - w.lo[0]
    return (L * 1e3) ** 3 * abs(w.analytic["Tdot"]) ** 4 + 1.0


def shard_runs(costs, world):
    """Longest-processing-time assignment of runs to ranks: run indices per rank."""
    order = sorted(range(len(costs)), key=lambda i: -costs[i])
    loads, parts = [0.0] * world, [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: loads[k])
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]


def batch_ensemble(dev, rank=0, world=1, serial_every=8, graph_steps=20):
    """The 256-run columnar-to-equiaxed ensemble (400 steps of 1 ms) in one batch
    context per GPU: every kernel of a step covers all runs of the context, sized
    on the device, and the steps replay from CUDA graphs of graph_steps steps with
    the launch configuration the autotuner picked on a rehearsal of the same runs.
    With several ranks the runs are sharded by estimated work (no collective: the
    runs are independent) and the time is the slowest rank's.  On one GPU it is
    compared with the same runs each in its own single-run context, one after the
    other (every serial_every-th run, scaled to the ensemble).  All variants give
    identical particles (batch parity tests); set-up is outside every timing."""
    import torch
    from paper_2504_12858_gb300 import ensemble, inputs, native
    runs_all = inputs.cet_runs()
    mine = shard_runs([run_cost(w) for w in runs_all], world)[rank]
    runs = [runs_all[i] for i in mine]
    steps = runs[0].steps
    f = len(runs) / len(runs_all) * 1.5 if world > 1 else 1.0
    mem = dict(capacity=int(3.2e7 * min(f, 1.0)) + 100000,
               reached_capacity=int(2.6e8 * min(f, 1.0)) + 1000000,
               claim_blocks=int(2.4e6 * min(f, 1.0)) + 20000, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(b, n):
        torch.cuda.synchronize(dev)
        ev[0].record(b.stream)
        b.gp_step(n)
        ev[1].record(b.stream)
        torch.cuda.synchronize(dev)
        return ev[0].elapsed_time(ev[1]) / 1e3

    def release(b):
        b.close()
        torch.cuda.empty_cache()

    # rehearsal: the autotuner times its candidates on the ensemble at step 300
    b = ensemble.batch_from(runs, **mem)
    b.gp_step(300)
    cfg = b.gp_autotune(trial_steps=3)
    release(b)
    # step by step with the default launches
    b = ensemble.batch_from(runs, **mem)
    t_eager = timed(b, steps)
    release(b)
    # the measured configuration: autotuned launches replayed from CUDA graphs
    b = ensemble.batch_from(runs, **mem)
    cfg["graph_steps"] = graph_steps
    b.gp_set_launch_config(**cfg)
    barrier(world)
    tb = timed(b, steps)
    st = b.gp_stats()
    live, _ = b.gp_run_counts()
    arena_gb = b.arena_bytes / 1e9
    release(b)
    tb_ms, psteps = reduce_timing(tb * 1e3, float(st["particle_steps"]), world)
    tb = tb_ms / 1e3
    out = {"workload": "cet_runs: 256 runs, 0.5-2 mm cubes, columnar + equiaxed nucleation, "
                       "400 steps of 1 ms", "runs": len(runs_all), "steps": steps,
           "sharding": f"{world} rank(s), runs by estimated work, no collective",
           "batched_s": tb, "runs_per_s": len(runs_all) / tb,
           "particle_steps_per_s": psteps / tb,
           "launch_config": cfg, "batched_step_by_step_s_rank0": t_eager,
           "particles_per_run_rank0": {"min": int(live.min()), "median": int(np.median(live)),
                                       "max": int(live.max())},
           "arena_gb_rank0": round(arena_gb, 1)}
    if world > 1 or rank != 0:
        return out
    ts, sample = 0.0, list(range(0, len(runs), serial_every))
    for r in sample:
        w = runs[r]
        an = w.analytic
        cap = int(live[r] * 1.3) + 20000
        s = native.Sim(w.lo, w.hi, w.h, w.dt, w.a, w.b, w.T_L, capacity=cap,
                       reached_capacity=12 * cap, claim_blocks=max(8192, cap // 6),
                       max_grains=len(w.seeds) + len(w.nuclei["pos"]) + 16,
                       max_nuclei=len(w.nuclei["pos"]) + 16, device=dev)
        s.gp_set_thermal_analytic(an["T0"], an["G"], an["xref"], an["Tdot"])
        s.gp_add_grains(w.seeds, w.quats)
        s.gp_nucleation_sites(w.nuclei["pos"], w.nuclei["dTn"], w.nuclei["quat"])
        ts += timed(s, steps)
        s.close()
    scale = len(runs) / len(sample)
    out.update({"serial_sample_runs": len(sample), "serial_s_scaled": ts * scale,
                "serial_runs_per_s": len(runs) / (ts * scale),
                "speedup_vs_serial": ts * scale / tb})
    return out


def run_native(args, rank, world, local_rank):
    import torch
    from paper_2504_12858_gb300 import native
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    native.load()
    w = fixture(args.grains, args.n0, args.plate)
    per_grain = 4 * (args.n0 + 1) ** 2 + 2
    n0_est = args.grains * per_grain
    e2e_steps = args.e2e_steps or args.steps
    total_steps = args.warmup + max(args.steps, e2e_steps)
    # the envelopes grow by about 4 % per step; every crossing records a reached site
    capacity = int(args.capacity or min((1 << 30) - 1, int(n0_est * 1.05 ** total_steps * 1.3)
                                        + 1000000))
    reached = int(args.reached or min((1 << 32) - 2, int(n0_est * (1.2 + 0.9 * total_steps))))
    # claim blocks: an envelope growing from 50 to 70 lattice shells touches about
    # 1200 blocks of 8^3 sites (plus reservations lost to insertion races)
    blocks = args.claim_blocks or args.grains * 2000
    g = w.grid

    def make_sim():
        s = native.Sim(w.lo, w.hi, w.h, w.dt, w.a, w.b, w.T_L, capacity=capacity,
                       reached_capacity=reached, claim_blocks=blocks,
                       max_grains=args.grains + 16, grid_nodes=int(np.prod(g["T"].shape)),
                       device=dev)
        s.gp_set_thermal_grid(g["T"], g["origin"], g["spacing"], g["vel"])
        s.gp_add_grains(w.seeds, w.quats, nucleate=False)
        s.gp_seed_shell(np.arange(args.grains), args.n0)
        return s

    sim = make_sim()
    n_start = sim.gp_stats()["n_live"]
    stream = sim.stream

    sim.gp_step(args.warmup)
    torch.cuda.synchronize(dev)
    st0 = sim.gp_stats()
    sim.gp_profile(True)
    clocks = ClockSampler(local_rank) if rank == 0 else None
    if clocks:
        clocks.start()
    barrier(world)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.gp_step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    ms_local = e0.elapsed_time(e1)
    clk = clocks.stop() if clocks else None
    st1 = sim.gp_stats()
    prof = sim.gp_profile_read()
    sim.gp_profile(False)
    units_local = float(st1["particle_steps"] - st0["particle_steps"])
    ms, units = reduce_timing(ms_local, units_local, world)
    value = units / (ms / 1e3)
    sim.close()
    del sim
    torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers, on a second context from the same
    # start (the same warm-up steps untimed, then the same steps as the timed region):
    # the thermal table is copied from pinned host memory every step (as a coupled
    # thermal solver would supply it) and the step statistics are read back every step
    sim = make_sim()
    sim.gp_step(args.warmup)
    Th = torch.from_numpy(np.ascontiguousarray(g["T"])).pin_memory()
    Th_np = Th.numpy()
    torch.cuda.synchronize(dev)
    barrier(world)
    t0 = time.perf_counter()
    sa = sim.gp_stats()
    for _ in range(e2e_steps):
        sim.gp_set_thermal_grid(Th_np, g["origin"], g["spacing"], g["vel"])
        sim.gp_step(1)
        sim.gp_stats()
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    sb = sim.gp_stats()
    sim.close()
    del sim
    torch.cuda.empty_cache()
    e2e_units = float(sb["particle_steps"] - sa["particle_steps"])
    e2e_ms, e2e_units = reduce_timing(e2e_s * 1e3, e2e_units, world)
    e2e_value = e2e_units / (e2e_ms / 1e3)

    if rank != 0:
        if not args.no_extras:
            batch_ensemble(dev, rank, world)   # this rank's shard of the ensemble
        return 0

    # roofline of the dominant kernel (largest device time in the timed region)
    peak, peak_kind = measured_peak()
    dom = max(prof, key=lambda k: k["total_ms"]) if prof else None
    roof = None
    if dom:
        achieved = dom["units"] * dom["bytes_per_unit"] / (dom["total_ms"] / 1e3) / 1e9
        # each timed entry runs once per step (some entries hold several kernels)
        per_launch_units = dom["units"] / max(args.steps, 1)
        tb = ncu_traffic(dom["name"])
        roof = {"bound": "hbm", "kernel": dom["name"], "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": None if tb is None else tb * per_launch_units,
                "issue_slots_busy": ncu_issue(dom["name"]),
                "algorithmic_bytes_per_launch": dom["bytes_per_unit"] * per_launch_units,
                "avg_launch_ms": dom["total_ms"] / max(args.steps, 1)}
    # the whole step against the copy bandwidth: measured DRAM bytes per particle-step
    # (one-pass ncu capture of the default run) and the algorithmic 48 B
    default_run = (args.grains, args.n0, tuple(args.plate), args.warmup, args.steps) == \
        (10000, 50, (4.0, 2.0, 1.0), 3, 10)
    sb = ncu_step_traffic() if default_run else None
    step_roof = {"peak": peak, "unit": "GB/s", "peak_source": peak_kind,
                 "algorithmic_bytes_per_particle_step": B_ALG_STEP,
                 "algorithmic_frac": value * B_ALG_STEP / 1e9 / peak,
                 "dram_bytes_per_particle_step": sb,
                 "dram_frac": None if sb is None else value * sb / 1e9 / peak}
    launches = sum(k["launches"] for k in prof)
    kernels = {k["name"]: {"launches": k["launches"], "ms": round(k["total_ms"], 3),
                           "share": round(k["total_ms"] / max(sum(x["total_ms"] for x in prof),
                                                               1e-9), 4)} for k in prof}
    cb = cpu_baseline(args.cpu_grains, args.n0, 2) if (world == 1 and not args.no_cpu) else None
    adj = adjoint_cost(dev) if not args.no_extras else None
    bat = batch_ensemble(dev, rank, world) if not args.no_extras else None
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "grains": args.grains, "shell_n0": args.n0,
                       "plate_mm": list(args.plate),
                       "particles_at_start": n_start,
                       "live_at_timed_start": st0["n_live"],
                       "active_at_timed_start": st0["n_active"],
                       "live_at_end": st1["n_live"], "parallelism": f"replicas x{world}",
                       "claim_blocks_used": round(st1["n_claim_blocks"] / blocks, 3),
                       "l2": "inputs larger than L2 (particle store > 1.5 GB)"},
            "roofline": roof, "step_roofline": step_roof, "kernels": kernels,
            "cpu_baseline": cb,
            "e2e": {"value": e2e_value, "unit": METRIC, "steps": e2e_steps,
                    "h2d_bytes_per_step": int(Th.numel() * 4),
                    "d2h_bytes_per_step": 160},
            "clocks": clk, "gpu_launches": launches, "adjoint": adj, "batch": bat}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--grains", type=int, default=10000)
    ap.add_argument("--n0", type=int, default=50)
    ap.add_argument("--capacity", type=int, default=0)
    ap.add_argument("--reached", type=int, default=0)
    ap.add_argument("--claim-blocks", type=int, default=0)
    ap.add_argument("--plate", type=float, nargs=3, default=(4.0, 2.0, 1.0),
                    help="plate size in mm (smaller plates with proportionally fewer grains "
                         "keep the grain density; used for profiling captures)")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="end-to-end steps (default: as many as --steps, on the same states)")
    ap.add_argument("--cpu-grains", type=int, default=100)
    ap.add_argument("--ref-grains", type=int, default=40)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the adjoint-cost and batched-ensemble measurements")
    args = ap.parse_args()
    rank, world, local_rank = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "native" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        dist.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world)
        return run_native(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            if dist.is_initialized():
                dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
