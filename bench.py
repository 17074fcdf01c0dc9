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
workload on the host cores: one oracle process per core, each on its own grains
of the fixture, timed together.

The line also reports, beside the fixture, the two workloads of the method's
applications at their stated sizes: competitive columnar growth in a slab
(configuration 2) and growth from the fusion line of the weld plate
(configuration 3 as the method runs it).

--ncu-digest CSV LOG turns a one-pass ncu capture (dram bytes and durations of
every launch of `bench.py ... --no-e2e --profile-warmup`) and that command's plain
JSON line into the per-unit DRAM bytes of every timed entry; the result is written
to profiles/ncu_traffic.json with the digest of the kernel sources it was taken on.
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


def ncu_record():
    """The committed per-unit DRAM figures (profiles/ncu_traffic.json), if they were
    taken on the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    return d if d.get("sources_digest") == kernel_sources_digest() else None


def step_dram_bytes(prof, psteps):
    """DRAM bytes per particle-step of a run: every timed entry's per-unit DRAM bytes
    (from the committed capture) times the units this run processed, summed, divided
    by the run's particle-steps.  None if the capture does not cover every entry."""
    d = ncu_record()
    if d is None or not prof or psteps <= 0:
        return None
    per = d.get("entries", {})
    tot = 0.0
    for k in prof:
        if k["total_ms"] <= 0:
            continue
        if k["name"] not in per:
            return None
        tot += per[k["name"]]["dram_bytes_per_unit"] * k["units"]
    return tot / psteps


# profile entry -> the kernels it times; k_scan_sums belongs to the entry of the kernel
# launched before it (group: k_scan_blocks; obstacle: k_obs_count)
ENTRY_KERNELS = {
    "group": ("k_group_count", "k_scan_blocks", "k_group_scatter"),
    "build": ("k_group_order", "k_group_gather", "k_act_list"),
    "advance": ("k_advance",),
    "emit": ("k_emit", "k_emit_check"),
    "obstacle": ("k_obs_count", "k_obs_list", "k_obs_split", "k_obs_merge", "k_obs_table"),
    "nucleate": ("k_nucleate",),
    "finalize": ("k_finalize",),
    "keys": ("k_keys",),
}


def ncu_digest(csv_path, log_path):
    """Per-unit DRAM bytes of every timed entry from an ncu capture of all launches of
    `bench.py ... --no-e2e --profile-warmup` and that command's plain JSON line."""
    import csv
    import re
    line = [json.loads(x) for x in open(log_path) if x.startswith('{"metric"')][-1]
    units = {k: v["units"] for k, v in line["kernels"].items()}
    launches = {}
    rows = [r for r in csv.reader(open(csv_path)) if len(r) > 10]
    head = rows[0]
    col = {n: head.index(n) for n in ("ID", "Kernel Name", "Metric Name", "Metric Value")}
    for r in rows[1:]:
        try:
            i = int(r[col["ID"]])
        except ValueError:
            continue
        m = re.search(r"\b(k_[a-z0-9_]+)", r[col["Kernel Name"]])
        rec = launches.setdefault(i, {"kernel": m.group(1) if m else "?", "bytes": 0.0,
                                      "ns": 0.0})
        v = float(r[col["Metric Value"]].replace(",", ""))
        name = r[col["Metric Name"]]
        if name.startswith("dram__bytes"):
            rec["bytes"] += v
        elif name == "gpu__time_duration.sum":
            rec["ns"] += v
    owner = {k: e for e, ks in ENTRY_KERNELS.items() for k in ks}
    per, prev = {}, None
    for i in sorted(launches):
        k = launches[i]["kernel"]
        e = owner.get(k)
        if k == "k_scan_sums":
            e = "obstacle" if prev == "k_obs_count" else "group"
        prev = k
        if e is None:
            continue
        agg = per.setdefault(e, {"bytes": 0.0, "ns": 0.0, "launches": 0})
        agg["bytes"] += launches[i]["bytes"]
        agg["ns"] += launches[i]["ns"]
        agg["launches"] += 1
    out = {"sources_digest": kernel_sources_digest(), "entries": {},
           "capture": line["config"], "profiled_particle_steps": line.get("profiled_particle_steps")}
    for e, agg in per.items():
        if units.get(e):
            out["entries"][e] = {"dram_bytes_per_unit": round(agg["bytes"] / units[e], 2),
                                 "units": units[e], "launches": agg["launches"],
                                 "ncu_ms": round(agg["ns"] / 1e6, 3)}
    tot = sum(a["bytes"] for a in per.values())
    if line.get("profiled_particle_steps"):
        out["dram_bytes_per_particle_step"] = round(tot / line["profiled_particle_steps"], 1)
    return out


# algorithmic bytes of one particle-step for the whole step: read and write the
# 16-byte record, write and read back the 8-byte (cell key, index) pair
B_ALG_STEP = 48


# ----------------------------------------------------------------------------------
# CPU oracle on a bounded sample (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------------
def oracle_sample(n_grains_sample: int, n0: int, first: int = 0):
    import oracle
    w = fixture(10000, n0)
    o = oracle.Oracle(w.lo, w.hi, w.h, w.dt, w.a, w.b, w.T_L)
    g = w.grid
    o.set_thermal_grid(g["T"], g["origin"], g["spacing"], g["vel"])
    sl = slice(first, first + n_grains_sample)
    o.add_grains(w.seeds[sl], w.quats[sl], nucleate=False)
    o.seed_shell(np.arange(n_grains_sample), n0)
    return o


def time_oracle(o, steps: int):
    before = o.stats()["particle_steps"]
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return (o.stats()["particle_steps"] - before) / dt, dt


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_worker(k, n_grains, n0, warm, steps, barrier, q):
    o = oracle_sample(n_grains, n0, first=k * n_grains)
    o.step(warm)
    before = o.stats()["particle_steps"]
    barrier.wait()
    t0 = time.perf_counter()
    o.step(steps)
    t1 = time.perf_counter()
    q.put((o.stats()["particle_steps"] - before, t0, t1, o.n_particles))


def oracle_all_cores(n_grains=60, n0=50, warm=1, steps=2, procs=None):
    """One oracle process per host core, each on its own n_grains grains of the
    fixture (disjoint), stepped together after a barrier: the particle-steps of all
    processes over the time from the first start to the last finish.  Processes are
    spawned (never forked from a process that holds a CUDA context)."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    procs = min(procs, 10000 // n_grains)
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(k, n_grains, n0, warm, steps, barrier, q))
          for k in range(procs)]
    for p in ps:
        p.start()
    res = [q.get() for _ in ps]
    for p in ps:
        p.join()
    units = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    return units / span, span, procs, sum(r[3] for r in res)


def _oracle_from(w, nucleate=True):
    """The oracle set up on workload w (thermal field, grains, nucleation sites, or the
    initial particles and lattice sites of a given state)."""
    import oracle
    o = oracle.Oracle(w.lo, w.hi, w.h, w.dt, w.a, w.b, w.T_L)
    if w.analytic:
        an = w.analytic
        o.set_thermal_analytic(an["T0"], an["G"], an["xref"], an["Tdot"])
    if w.grid:
        g = w.grid
        o.set_thermal_grid(g["T"], g["origin"], g["spacing"], g["vel"])
    init = w.extra.get("particles") if w.extra else None
    o.add_grains(w.seeds, w.quats, nucleate=nucleate and init is None)
    if init is not None:
        o.load_particles(init["grain"], init["site"], init["dir"],
                         init["ell"].astype(np.float64), init["state"])
        gr, sr = w.extra["reached"]
        o.add_reached(gr, sr)
        o.add_claimed(gr, sr)
        o.add_claimed(*w.extra["claimed"])
    if w.nuclei:
        o.nucleation_sites(w.nuclei["pos"], w.nuclei["dTn"], w.nuclei["quat"])
    return o


def _oracle_config_worker(name):
    from paper_2504_12858_gb300 import inputs
    if name == "cet_runs":
        # the eight smallest cubes of the ensemble (0.50-0.55 mm), all 400 steps of each
        runs = inputs.cet_runs()
        pick = sorted(range(len(runs)), key=lambda r: runs[r].hi[0])[:8]
        ps, t = 0, 0.0
        for r in pick:
            o = _oracle_from(runs[r])
            rate, dt = time_oracle(o, runs[r].steps)
            ps += int(o.stats()["particle_steps"])
            t += dt
        return name, {"steps": 400, "runs": [int(r) for r in pick]}, ps / t, t, ps
    if name == "weld_natural":
        w = inputs.weld_natural()
        o = _oracle_from(w)
        steps = 5    # its first 5 of 500 steps (7e5 ACTIVE particles)
    else:
        w = getattr(inputs, name)()
        o = _oracle_from(w)
        steps = w.steps
    rate, dt = time_oracle(o, steps)
    return name, {"steps": steps}, rate, dt, int(o.stats()["particle_steps"])


def oracle_configs():
    """The oracle, one process (one core) per configuration, run side by side: the single
    grain (400 steps) and the columnar slab (600 steps) at their stated sizes, the first
    5 steps of growth from the fusion line of the weld plate, and the eight smallest runs
    of the ensemble (400 steps each)."""
    import multiprocessing as mp
    jobs = ["single_grain", "columnar_slab", "weld_natural", "cet_runs"]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(_oracle_config_worker, jobs)
    return {n: dict(extra, value=r, unit=METRIC, cores=1, seconds=round(t, 2), particle_steps=ps)
            for n, extra, r, t, ps in res}


def cpu_baseline(n_grains_sample=60, n0=50, steps=4):
    rate, span, procs, npart = oracle_all_cores(n_grains_sample, n0, 1, steps)
    return {"value": rate, "unit": METRIC, "cores": procs, "kind": "oracle",
            "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "sample": (f"{procs} oracle processes, one per host core, each on {n_grains_sample} "
                       f"of the 1e4 grains of the same workload (disjoint, {npart:.2e} particles "
                       f"in all), {steps} steps after 1 untimed step, {span:.1f} s wall from the "
                       f"first start to the last finish"),
            "configs": oracle_configs()}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    rate, span, procs, npart = oracle_all_cores(args.ref_grains, args.n0, args.warmup,
                                                args.steps)
    cb = {"value": rate, "unit": METRIC, "cores": procs, "kind": "oracle",
          "nproc": os.cpu_count(), "cpu_model": cpu_model(),
          "sample": (f"{procs} oracle processes (one per core), each on {args.ref_grains} of "
                     f"the 1e4 grains of the same workload, {args.steps} timed steps after "
                     f"{args.warmup} warm-up steps")}
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": METRIC,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * span / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "sample_grains_per_process": args.ref_grains,
                       "processes": procs},
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
    reverse sweep) over the plain forward that gives the same outputs, on the 32-grain
    calibration cube (200 steps).  Both timings hold the same work around the steps:
    the context is created with the same capacities and seeded, and the particles are
    read back and reduced to the front outputs."""
    import torch
    from paper_2504_12858_gb300 import inputs, native
    from paper_2504_12858_gb300.adjoint import FrontAdjoint, front_outputs
    w = inputs.adjoint_cube()
    an = w.analytic
    cap = 400000

    def plain():
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        sim = native.Sim(w.lo, w.hi, w.h, w.dt, w.a, w.b, w.T_L, capacity=cap,
                         reached_capacity=10 * cap, max_grains=len(w.seeds) + 8, device=dev)
        sim.gp_set_thermal_analytic(an["T0"], an["G"], an["xref"], an["Tdot"])
        sim.gp_add_grains(w.seeds, w.quats)
        sim.gp_step(w.steps)
        front_outputs(sim.gp_get_particles(), w.h, len(w.seeds))
        torch.cuda.synchronize(dev)
        t = time.perf_counter() - t0
        sim.close()
        return t

    def with_gradient(every):
        th = torch.tensor([w.a[0], w.b[0], an["G"][2], -an["Tdot"]], dtype=torch.float64,
                          requires_grad=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        out = FrontAdjoint.apply(th, w, cap, every)
        out[1:].sum().backward()
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t0

    plain()
    with_gradient(1)
    tp = min(plain() for _ in range(3))
    tg = {k: min(with_gradient(k) for _ in range(3)) for k in (1, 10)}
    # tape bytes per particle of capacity and taped step: states, parents and directions
    # (6), plus the 16-byte records of every k-th step
    return {"case": "adjoint_cube: 200 um cube, 32 grains, 200 steps", "plain_forward_ms": tp * 1e3,
            "forward_with_tape_plus_backward_ms": tg[1] * 1e3, "cost_ratio": tg[1] / tp,
            "checkpoint_every_10": {"forward_with_tape_plus_backward_ms": tg[10] * 1e3,
                                    "cost_ratio": tg[10] / tp},
            "tape_bytes_per_particle_step": {"every_1": 6 + 16, "every_10": 6 + 16 / 10}}


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


def _batch_of_one(w, steps, capacity, dev, graph_steps=20, **kw):
    """The same workload as a batch context of one run: its steps sized on the device
    and replayed from CUDA graphs of graph_steps steps (set-up outside the timing)."""
    import torch
    from paper_2504_12858_gb300 import ensemble
    b = ensemble.batch_from([w], capacity, device=dev, **kw)
    b.gp_set_launch_config(graph_steps=graph_steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    st0 = b.gp_stats()
    e0.record(b.stream)
    b.gp_step(steps)
    e1.record(b.stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    st1 = b.gp_stats()
    b.close()
    torch.cuda.empty_cache()
    return {"ms_per_step": ms / steps,
            "particle_steps_per_s": (st1["particle_steps"] - st0["particle_steps"]) / (ms / 1e3),
            "particles_end": st1["n_live"], "graph_steps": graph_steps}


def _workload_run(w, steps, capacity, dev, **kw):
    """Steps workload w on the GPU (after its set-up) and measures the timed steps
    with CUDA events on the library's stream."""
    import torch
    from paper_2504_12858_gb300 import native
    an, g = w.analytic, w.grid
    s = native.Sim(w.lo, w.hi, w.h, w.dt, w.a, w.b, w.T_L, capacity=capacity,
                   max_grains=len(w.seeds) + 16, device=dev,
                   grid_nodes=int(np.prod(g["T"].shape)) if g else 0, **kw)
    if an:
        s.gp_set_thermal_analytic(an["T0"], an["G"], an["xref"], an["Tdot"])
    if g:
        s.gp_set_thermal_grid(g["T"], g["origin"], g["spacing"], g["vel"])
    init = w.extra.get("particles")
    s.gp_add_grains(w.seeds, w.quats, nucleate=init is None)
    if init is not None:
        s.gp_load_particles(init["grain"], init["site"], init["dir"], init["ell"], init["state"], 0)
        gr, sr = w.extra["reached"]
        s.gp_add_sites(gr, sr, reached=True, claimed=True)
        s.gp_add_sites(*w.extra["claimed"], reached=False, claimed=True)
    st0 = s.gp_stats()
    s.gp_profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(s.stream)
    s.gp_step(steps)
    e1.record(s.stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    st1 = s.gp_stats()
    prof = s.gp_profile_read()
    s.close()
    psteps = st1["particle_steps"] - st0["particle_steps"]
    cross = st1["n_reached"] - st0["n_reached"]
    peak, kind = measured_peak()
    rate = psteps / (ms / 1e3)
    return {"steps": steps, "ms_per_step": ms / steps, "particle_steps_per_s": rate,
            "particles_start": st0["n_live"], "particles_end": st1["n_live"],
            "frozen_end": st1["n_frozen"], "grains": st1["n_grains"],
            "crossings_per_particle_step": cross / max(psteps, 1),
            "algorithmic_frac": rate * B_ALG_STEP / 1e9 / peak, "peak_source": kind,
            "kernels_ms_per_step": {k["name"]: round(k["total_ms"] / steps, 4) for k in prof}}


APPLICATIONS = ("single_grain", "columnar_slab", "weld_natural")


def application_workloads(dev, only=None):
    """Configurations 1 to 3 at their stated sizes: the single grain (400 steps),
    competitive columnar growth in the 1 x 1 x 0.05 mm slab (600 steps) and growth from
    the fusion line of the weld plate (the base metal cut by the t = 0 liquidus, 500
    steps); only: one of APPLICATIONS.  Set-up (input generation, seeding, loading) is
    outside the timing."""
    import torch
    from paper_2504_12858_gb300 import native
    out = {}

    def guarded(name, fn):
        try:
            out[name].update(fn())
        except native.GPError as e:    # reported in the line, not fatal to the bench
            out[name]["error"] = str(e)
        torch.cuda.empty_cache()

    if only in (None, "single_grain"):
        _single_grain(out, guarded, dev)
    if only in (None, "columnar_slab"):
        _columnar_slab(out, guarded, dev)
    if only in (None, "weld_natural"):
        _weld_natural(out, guarded, dev)
    return out


def _single_grain(out, guarded, dev):
    from paper_2504_12858_gb300 import inputs
    w = inputs.single_grain()
    out["single_grain"] = dict(
        workload="single_grain: 200 um cube, one grain, uniform dT = 5 K, v = 1e-5 dT^2, "
                 "h = 2 um, dt = 2 ms, 400 steps")
    # the envelope reaches about 100 sites along each axis: 1.4e6 reached sites inside it
    guarded("single_grain", lambda: _workload_run(w, w.steps, 200000, dev,
                                                  reached_capacity=4000000))
    # a problem this small is bound by the launches and host round trip of each step: the
    # same run as a batch context of one replays its steps from CUDA graphs
    guarded("single_grain", lambda: {"as_batch_of_one": _batch_of_one(
        w, w.steps, 200000, dev, reached_capacity=4000000)})


def _columnar_slab(out, guarded, dev):
    from paper_2504_12858_gb300 import inputs
    w = inputs.columnar_slab()
    out["columnar_slab"] = dict(
        workload="columnar_slab: 1x1x0.05 mm, 50 bottom seeds, G = 1e4 K/m, Tdot = 10 K/s, "
                 "v = 1e-5 dT^2, h = 2 um, dt = 1 ms, 600 steps")
    guarded("columnar_slab",
            lambda: _workload_run(w, w.steps, 2000000, dev, reached_capacity=6000000))
    guarded("columnar_slab", lambda: {"as_batch_of_one": _batch_of_one(
        w, w.steps, 2000000, dev, reached_capacity=6000000)})


def _weld_natural(out, guarded, dev):
    from paper_2504_12858_gb300 import inputs
    t0 = time.perf_counter()
    w = inputs.weld_natural()
    out["weld_natural"] = dict(
        workload="weld_natural: the 4x2x1 mm weld plate, base-metal grains cut by the t = 0 "
                 "liquidus, particles on the fusion line heading into the melt, 500 steps "
                 "of 0.1 ms (the source moves 0.83 mm)",
        input_generation_s=round(time.perf_counter() - t0, 1))
    # the solid the grains leave behind the moving pool: at step 500 about 1.2e8 live
    # particles (1.17e8 of them FROZEN at grain contacts), 9.6e8 reached lattice sites and
    # 3.5e6 claim blocks
    guarded("weld_natural",
            lambda: _workload_run(w, w.steps, 160000000, dev, reached_capacity=1200000000,
                                  claim_blocks=5000000))


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
    stw = sim.gp_stats()
    if args.profile_warmup:       # capture mode: the profile covers the warm-up steps too
        sim.gp_profile(True)
    sim.gp_step(args.warmup)
    torch.cuda.synchronize(dev)
    st0 = sim.gp_stats()
    if not args.profile_warmup:
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
    Th = torch.from_numpy(np.ascontiguousarray(g["T"])).pin_memory()
    e2e_value = None
    if args.no_e2e:
        e2e_steps = 0
    else:
        sim = make_sim()
        sim.gp_step(args.warmup)
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
    rec = ncu_record()
    roof = None
    nsteps_prof = args.steps + (args.warmup if args.profile_warmup else 0)
    if dom:
        achieved = dom["units"] * dom["bytes_per_unit"] / (dom["total_ms"] / 1e3) / 1e9
        # each timed entry runs once per step (some entries hold several kernels)
        per_launch_units = dom["units"] / max(nsteps_prof, 1)
        ent = (rec or {}).get("entries", {}).get(dom["name"])
        roof = {"bound": "hbm", "kernel": dom["name"], "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": None if ent is None else ent["dram_bytes_per_unit"] * per_launch_units,
                "traffic_source": None if ent is None else
                "per-unit DRAM bytes of the 1 mm plate capture, scaled by this run's units",
                "algorithmic_bytes_per_launch": dom["bytes_per_unit"] * per_launch_units,
                "avg_launch_ms": dom["total_ms"] / max(nsteps_prof, 1)}
    # the whole step against the copy bandwidth: DRAM bytes per particle-step (per-unit
    # bytes of every entry from the committed small-plate capture, times this run's
    # units) and the algorithmic 48 B
    psteps_prof = float(st1["particle_steps"] - (stw if args.profile_warmup else st0)["particle_steps"])
    sb = step_dram_bytes(prof, psteps_prof)
    step_roof = {"peak": peak, "unit": "GB/s", "peak_source": peak_kind,
                 "algorithmic_bytes_per_particle_step": B_ALG_STEP,
                 "algorithmic_frac": value * B_ALG_STEP / 1e9 / peak,
                 "dram_bytes_per_particle_step": sb,
                 "dram_frac": None if sb is None else value * sb / 1e9 / peak,
                 "dram_source": None if sb is None else
                 "per-unit DRAM bytes of each timed entry from the 1 mm plate capture "
                 "(profiles/ncu_traffic.json), times this run's units"}
    launches = sum(k["launches"] for k in prof)
    kernels = {k["name"]: {"launches": k["launches"], "ms": round(k["total_ms"], 3),
                           "units": k["units"],
                           "share": round(k["total_ms"] / max(sum(x["total_ms"] for x in prof),
                                                               1e-9), 4)} for k in prof}
    cb = cpu_baseline(args.cpu_grains, args.n0, 4) if (world == 1 and not args.no_cpu) else None
    adj = adjoint_cost(dev) if not args.no_extras else None
    bat = batch_ensemble(dev, rank, world) if not args.no_extras else None
    apps = application_workloads(dev) if not args.no_extras else None
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
            "clocks": clk, "gpu_launches": launches, "adjoint": adj, "batch": bat,
            "applications": apps, "obstacles_at_end": st1["n_frozen"],
            "profiled_particle_steps": psteps_prof}
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
    ap.add_argument("--cpu-grains", type=int, default=60)
    ap.add_argument("--ref-grains", type=int, default=60)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the adjoint-cost, batched-ensemble and application measurements")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end context")
    ap.add_argument("--profile-warmup", action="store_true",
                    help="capture mode: the per-kernel profile covers the warm-up steps too")
    ap.add_argument("--application", choices=APPLICATIONS,
                    help="time one of configurations 1 to 3 alone and print its line")
    ap.add_argument("--ncu-digest", nargs=2, metavar=("CSV", "LOG"),
                    help="write profiles/ncu_traffic.json from an ncu capture and its plain log")
    args = ap.parse_args()
    if args.application:         # one of configurations 1 to 3 alone, on cuda:0
        import torch
        r = application_workloads(torch.device("cuda:0"), only=args.application)
        print(json.dumps({"application": args.application, **r[args.application]}))
        return 0 if "error" not in r[args.application] else 1
    if args.ncu_digest:
        d = ncu_digest(*args.ncu_digest)
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json"), "w") as f:
            json.dump(d, f, indent=1)
        print(json.dumps(d))
        return 0
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
