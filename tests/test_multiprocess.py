"""Host side of the multi-GPU path on CPU (gloo, world size 2).

Several GPUs run independent replicas of the index (every rank holds the
whole graph and labels and runs the whole step); the only collective is the
timing reduction: the job's time is the slowest rank's, and the whole-job
rate counts every rank's units.  The reference arm runs on rank 0 alone.
"""
import os
import socket
import subprocess
import sys

import torch.distributed as tdist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [3.0, 5.0][rank]
    slowest = bench.max_over_ranks(local_ms, world, tdist)
    rate = bench.whole_job_rate(1000.0, world, slowest)
    tdist.barrier()
    q.put((rank, slowest, rate))
    tdist.destroy_process_group()


def test_step_time_is_the_slowest_rank_and_rate_counts_every_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, slowest, rate in got:
        assert slowest == 5.0                       # every rank sees the slowest replica's time
        assert abs(rate - 2 * 1000.0 / 5e-3) < 1e-6  # units of both ranks over that time


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(4.0, 1, None) == 4.0
    assert bench.whole_job_rate(500.0, 1, 2.0) == 500.0 / 2e-3


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "tiny", "--steps", "1"],
                       cwd=ROOT, env=env, capture_output=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == b""


def test_rooflines_also_against_nominal_peaks():
    import bench
    line = {"roofline": {"achieved": 790.0, "unit": "GB/s", "frac": 0.1},
            "roofline_scorer": {"achieved": 450.0, "unit": "TFLOP/s", "frac": 0.2},
            "roofline_build": None}
    bench.add_nominal(line)
    assert abs(line["roofline"]["frac_of_nominal"] - 0.1) < 1e-12
    assert abs(line["roofline_scorer"]["frac_of_nominal"] - 0.2) < 1e-12
    assert line["roofline"]["frac"] == 0.1 and line["roofline_build"] is None


def test_cpu_baseline_reports_all_cores_and_one_thread():
    """The oracle as it stands on a sample of the step: all host cores (the
    paper's parallel DBL-P analogue) and one thread (its sequential DBL)."""
    import argparse

    import bench
    import dbl_inputs
    import oracle
    oracle.build()
    dbl_inputs.build()
    w = dbl_inputs.workload("tiny")
    r = bench.cpu_baseline(argparse.Namespace(k=64, kprime=64, batch=1000, ref_insertions=10_000,
                                              ref_queries=100_000), w)
    assert r["kind"] == "oracle" and r["cores"] >= 1 and r["value"] > 0 and r["cpu_model"]
    one = r["single_thread"]
    assert one["value"] > 0 and one["queries_per_s"] > 0 and one["inserted_edges_per_s"] > 0


def test_query_shards_cover_the_batch_once_in_order():
    import bench
    for world in range(1, 8):
        for q in (0, 1, 5, 7, 1003, 10_000_000):
            parts = [bench.shard_range(q, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == q
            for (a, b), (c, d) in zip(parts, parts[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1


def _shard_worker(rank, world, port, q):
    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    Q = 1003
    lo, hi = bench.shard_range(Q, rank, world)
    local = (torch.arange(lo, hi) * 7 % 251).to(torch.uint8)   # this rank's "answers"
    got = bench.gather_answers(local, Q, world, tdist)
    want = (torch.arange(Q) * 7 % 251).to(torch.uint8)
    q.put((rank, bool(torch.equal(got, want)), hi - lo))
    tdist.destroy_process_group()


def test_sharded_answers_gather_back_in_input_order():
    """Two gloo ranks answer their slices of a query batch; the gathered
    answers come back complete and in input order on every rank."""
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=10) for _ in range(world))
    assert all(ok for _, ok, _ in got)
    assert sum(n for _, _, n in got) == 1003


def test_build_roofline_arithmetic():
    """The build's roofline: algorithmic bytes over the propagation time, the
    preparation reported beside it, against the measured HBM peak."""
    import bench
    peaks, _ = bench.measured_peaks()
    form = {"build_kernel_ms": {"propagate": 10.0, "build_prep": 5.0}, "build_algorithmic_bytes": 20e9,
            "build_edges_relaxed": 700e6}
    r = bench.build_roofline(form)
    assert abs(r["achieved"] - 2000.0) < 1e-9                     # 20 GB in 10 ms
    assert abs(r["frac"] - 2000.0 / peaks["hbm_gbs"]) < 1e-12
    assert r["prep_ms"] == 5.0 and r["build_ms"] == 15.0
    assert abs(r["teps"] - 70e9) < 1e-3
    assert bench.build_roofline({"build_kernel_ms": {}}) is None


def test_learned_judge_keeps_only_what_searches_less_and_repairs_cheaply():
    import bench
    ref = {"searched": 1000, "relaxed_per_step": 100_000}
    assert not bench.learned_judge({"searched": 900, "relaxed_per_step": 120_000}, ref)    # kept
    assert bench.learned_judge({"searched": 1001, "relaxed_per_step": 100_000}, ref)       # more searches
    assert bench.learned_judge({"searched": 500, "relaxed_per_step": 10_000_000}, ref)     # repair much dearer


def test_ncu_traffic_keys_name_sources_that_exist():
    """Every stored traffic figure is keyed to a kernel source the bench can
    hash, so a changed kernel reports null instead of a stale figure."""
    import bench
    for kind in bench.NCU_TRAFFIC:
        assert len(bench.source_sha(kind)) == 12
    assert bench.NCU_TRAFFIC["propagate_grouped"][0] > bench.NCU_TRAFFIC["propagate_batch"][0]
