"""Host logic of bench.py on CPU: multi-rank aggregation over gloo (world size 2) and
the clock-log parser."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    assert (r, w, lr) == (rank, world, rank)
    bench.barrier(world)
    ms, units = bench.reduce_timing(10.0 + 5.0 * rank, 1000.0 * (rank + 1), world)
    out[rank] = (ms, units)
    dist.destroy_process_group()


def test_reduce_timing_takes_max_time_and_sums_work_over_ranks():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        ms, units = out[rank]
        assert ms == 15.0            # slowest rank
        assert units == 3000.0       # all ranks' particle steps


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_timing(3.5, 7.0, 1) == (3.5, 7.0)


def test_clock_parser(tmp_path):
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "c.csv")
    with open(c.path, "w") as f:
        f.write("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 210, 2070, 100.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")

    class _P:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            pass

    c.proc = _P()
    r = c.stop()
    assert r["sm_max_mhz"] == 2070.0
    assert r["sm_mhz"] == pytest.approx(2025.0)
    assert r["reasons"] == ["sw_power_cap"]


def test_ensemble_sharding_covers_every_run_once_and_balances_work():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2504_12858_gb300 import inputs
    runs = inputs.cet_runs()
    costs = [bench.run_cost(w) for w in runs]
    for world in (1, 2, 4, 8):
        parts = bench.shard_runs(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(len(runs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # greedy LPT: no rank exceeds the mean by more than the largest single run
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-9


def test_kernel_digest_ignores_comments_and_catches_code(tmp_path, monkeypatch):
    """The committed ncu figures are matched to the kernel sources by a digest that
    comment and blank-space edits leave unchanged and any code edit changes; on a
    mismatch the bench reports no traffic."""
    sys.path.insert(0, ROOT)
    import json
    import shutil
    import bench
    src = os.path.join(ROOT, "paper_2504_12858_gb300", "csrc")
    root = tmp_path / "r"
    shutil.copytree(src, root / "paper_2504_12858_gb300" / "csrc")
    (root / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(root))
    d0 = bench.kernel_sources_digest()
    f = root / "paper_2504_12858_gb300" / "csrc" / "gp_sort.cu"
    text = f.read_text()
    f.write_text("// a new comment line\n" + text.replace("\n", "\n\n", 3) + "\n/* block */\n")
    assert bench.kernel_sources_digest() == d0
    json.dump({"sources_digest": d0, "entries": {"advance": {"dram_bytes_per_unit": 7.0},
                                                 "emit": {"dram_bytes_per_unit": 3.0}}},
              open(root / "profiles" / "ncu_traffic.json", "w"))
    prof = [{"name": "advance", "units": 10.0, "total_ms": 1.0},
            {"name": "emit", "units": 20.0, "total_ms": 1.0}]
    assert bench.step_dram_bytes(prof, 10.0) == (7.0 * 10 + 3.0 * 20) / 10.0
    assert bench.step_dram_bytes(prof + [{"name": "group", "units": 1.0, "total_ms": 1.0}],
                                 10.0) is None          # an entry without a figure
    f.write_text(text.replace("kSortThreads", "kSortThreads ", 1).replace("return 0;", "return 1;", 1))
    assert bench.kernel_sources_digest() != d0
    assert bench.ncu_record() is None and bench.step_dram_bytes(prof, 10.0) is None


def test_ncu_digest_attributes_launches_to_timed_entries(tmp_path):
    """The digest sums each launch's DRAM bytes into the timed entry of its kernel
    (k_scan_sums goes to the entry of the kernel launched before it) and divides by
    the units that entry processed in the plain run."""
    sys.path.insert(0, ROOT)
    import json
    import bench
    rows = [["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream",
             "Block Size", "Grid Size", "Device", "CC", "Metric Name", "Metric Unit",
             "Metric Value"]]
    launches = [("k_seed_shell", 5), ("k_group_count", 10), ("k_scan_blocks", 1),
                ("k_scan_sums", 1), ("k_group_scatter", 20), ("k_obs_count", 2),
                ("k_scan_sums", 1), ("k_obs_merge", 40), ("k_advance", 100), ("k_emit", 50)]
    for i, (k, b) in enumerate(launches):
        name = f"void gp::(anonymous namespace)::{k}<false>(gp::Params, int)"
        for m, v in (("dram__bytes_read.sum", b / 2), ("dram__bytes_write.sum", b / 2),
                     ("gpu__time_duration.sum", 1000)):
            rows.append([str(i), "1", "python", "h", name, "1", "7", "(256,1,1)", "(1,1,1)", "0",
                         "10.3", m, "byte", str(v)])
    import csv
    with open(tmp_path / "c.csv", "w", newline="") as fh:
        csv.writer(fh).writerows(rows)
    line = {"metric": "particle-steps/s", "config": {}, "profiled_particle_steps": 10,
            "kernels": {"group": {"units": 4}, "obstacle": {"units": 2}, "advance": {"units": 10},
                        "emit": {"units": 5}}}
    (tmp_path / "p.log").write_text("noise\n" + json.dumps(line) + "\n")
    d = bench.ncu_digest(str(tmp_path / "c.csv"), str(tmp_path / "p.log"))
    e = d["entries"]
    assert e["group"]["dram_bytes_per_unit"] == (10 + 1 + 1 + 20) / 4
    assert e["obstacle"]["dram_bytes_per_unit"] == (2 + 1 + 40) / 2
    assert e["advance"]["dram_bytes_per_unit"] == 10.0 and e["emit"]["dram_bytes_per_unit"] == 10.0
    assert d["dram_bytes_per_particle_step"] == (32 + 43 + 100 + 50) / 10


def test_bench_oracle_setup_matches_the_tests():
    """The oracle that the cpu_baseline leg times is set up on a workload as the parity
    tests set it up (analytic field, grains, nucleation sites, or a given state of
    particles and reached and claimed sites): five steps give the same particles and
    counters."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from paper_2504_12858_gb300 import inputs
    from tests.helpers import oracle_from
    base = inputs.single_grain()
    o = oracle_from(base)
    o.step(20)
    state = inputs.Workload(**{**base.__dict__, "name": "state", "extra": dict(
        particles=o.particles(), reached=o.reached(), claimed=o.claimed())})
    for w in (base, inputs.cet_runs(n_runs=1)[0], state):
        a, b = bench._oracle_from(w), oracle_from(w)
        a.step(5)
        b.step(5)
        assert a.stats() == b.stats(), w.name
        pa, pb = a.particles(), b.particles()
        for f in pa:
            assert np.array_equal(pa[f], pb[f]), (w.name, f)


def test_application_option_names_every_timed_application():
    # `bench.py --application NAME` runs one of the applications the full bench times;
    # the option's choices and the timed sections name the same three configurations
    import inspect

    import bench
    assert bench.APPLICATIONS == ("single_grain", "columnar_slab", "weld_natural")
    src = inspect.getsource(bench.application_workloads)
    for name in bench.APPLICATIONS:
        assert f'only in (None, "{name}")' in src
        assert callable(getattr(bench, "_" + name))
