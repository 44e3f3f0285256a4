#!/usr/bin/env python3
"""Benchmark of the DBL reachability index on GB300.

Default workload "large" (the learned-landmark configuration): directed R-MAT
(a,b,c,d = .57,.19,.19,.05), n = 2^24, m = 2^28 (Graph500 edge factor 16),
seed 3; k = 64 landmarks and k' = 64 leaf buckets, with the same comparison
at k = 128.  One step = restore the built index, insert 1,000,000 new edges in
batches of 100,000 (label repair, Algorithm 3 and its mirrors) and answer
10,000,000 mixed queries (Algorithm 2: half uniform pairs, half (u, end of a
random forward walk from u)).  Inputs are resident in HBM before the timed
region; the labels (512 MB at k = 64), pair arrays (80 MB) and adjacency
(2 GB) exceed the 126 MB L2, so no flush is needed between steps.

Forms, all on the same graph and inputs (none of them with per-kernel timing):
  plain    degree landmarks; frontier levels driven from the host (one launch
           and one read-back per level)
  batched  degree landmarks; persistent cooperative kernels, no host round trip
  graph    batched, each step part (restore, insertions, queries) replayed as
           a captured CUDA graph
  learned  top-k learned landmarks (scorer trained on sampled query outcomes),
           batched + graph: the headline `value`
A separate pass of the learned form with per-kernel CUDA events gives the
roofline figures.  Extra forms on the social workload (n = 4,847,571,
m = 68,993,773): insertion batches of 1k, 10k and 100k edges, and the batched
configuration (k = 128, log-uniform batch sizes).
Output: one JSON line (rank 0).  `--impl reference` times the CPU oracle on
the same workload instead.
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

METRIC = "queries/s + inserted edges/s, learned+batched vs plain GPU form, 100% exact"
UNIT = "ops/s (queries + inserted edges)"

# DRAM traffic per launch from an ncu capture, valid only while the kernel's
# source is unchanged: {kernel class: (bytes per launch, sha1[:12] of the source file)}.
# query_label: 10M pairs on the 2^24-vertex graph (k = k' = 64, 32-byte L2
# fetch); propagate_grouped: one insertion launch of the workload's 1M edges;
# propagate_batch: one of 100,000 (bench.py --kernel-case label / insert).
NCU_TRAFFIC: dict[str, tuple[float, str]] = {"query_label": (636_424_192 + 22_371_584, "fb983a793219"),
                                             "propagate_grouped": (305_130_240 + 178_975_488, "74298b536cff"),
                                             "propagate_batch": (22_423_296 + 6_051_840, "74298b536cff")}
# Source a traffic figure was measured on: the kernel's own region of its file
# (None: the whole file) and the headers that file includes; an edit anywhere
# else does not invalidate the figure, any edit there does.
KERNEL_SOURCE = {
    "query_label": ("dbl_query.cu", "// ------------------------------------------------------------ label test",
                    "// The undecided pairs of a batch, from the answer array"),
    "propagate_grouped": ("dbl_insert.cu", None, None),
    "propagate_batch": ("dbl_insert.cu", None, None),
}
KERNEL_HEADERS = ("dbl_frontier.cuh", "dbl_internal.cuh", "dbl_kernels.cuh", "dbl_persistent.cuh")


def source_sha(kind: str) -> str:
    csrc = os.path.join(ROOT, "paper_2101_09441_gb300", "csrc")
    name, begin, end = KERNEL_SOURCE.get(kind, ("dbl_api.cu", None, None))
    text = open(os.path.join(csrc, name), "rb").read()
    if begin:
        i = text.find(begin.encode())
        j = text.find(end.encode(), i + 1)
        text = text[i:j] if i >= 0 and j > i else text
    h = hashlib.sha1(text)
    for hdr in KERNEL_HEADERS:
        h.update(open(os.path.join(csrc, hdr), "rb").read())
    return h.hexdigest()[:12]


def measured_peaks() -> tuple[dict, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(self.gpu)], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9 and parts[1].isdigit():
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "", 1).isdigit()]
        return {"sm_mhz": statistics.median(float(r[1]) for r in rows), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------------------ helpers
def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


NOMINAL = {"GB/s": 7900.0, "TFLOP/s": 2250.0}  # GB300 HBM3e and dense bf16 tensor rate, for context


def add_nominal(line: dict) -> dict:
    """Each roofline object also against the nominal peak of its unit (the
    fraction that counts is the one against the measured peak)."""
    for key in ("roofline", "roofline_label_test", "roofline_build", "roofline_scorer"):
        r = line.get(key)
        if r and r.get("achieved") is not None and r.get("unit") in NOMINAL:
            r["nominal_peak"] = NOMINAL[r["unit"]]
            r["frac_of_nominal"] = r["achieved"] / NOMINAL[r["unit"]]
    return line


def max_over_ranks(x: float, world: int, tdist, device="cpu") -> float:
    """The largest value over the ranks (the slowest replica's time); every
    rank gets it.  One process per GPU, replicas only: this reduction is the
    only collective of a run."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, total_ms: float) -> float:
    """Units all ranks processed per second over the slowest rank's time."""
    return world * units_per_rank / (total_ms * 1e-3)


def shard_range(q: int, rank: int, world: int) -> tuple[int, int]:
    """Rank `rank`'s contiguous slice of q queries: the slices of all ranks
    cover [0, q) once, in rank order, sizes differing by at most one."""
    base, extra = divmod(q, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def gather_answers(local, q: int, world: int, tdist):
    """Every rank's answers (uint8 tensor of its shard_range slice) back in
    input order on every rank: one all_gather of equal-length padded pieces
    (the only collective, and only after the timed region)."""
    import torch
    if world <= 1:
        return local
    width = q // world + 1
    buf = torch.zeros(width, dtype=torch.uint8, device=local.device)
    buf[:local.numel()] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    tdist.all_gather(parts, buf)
    out = [parts[r][:shard_range(q, r, world)[1] - shard_range(q, r, world)[0]] for r in range(world)]
    return torch.cat(out)


def step_batches(n_edges: int, batch: int):
    return [(b, min(b + batch, n_edges)) for b in range(0, n_edges, batch)]


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        outp = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in outp.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_oracle_step(ref, w, batches, nq, threads):
    ref.rewind()
    t0 = time.perf_counter()
    for a, b in batches:
        ref.insert_edges(w["ins_src"][a:b], w["ins_dst"][a:b])
    t1 = time.perf_counter()
    ref.query(w["q_u"][:nq], w["q_v"][:nq], nthreads=threads)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1


def workload_config(args, w, form="learned+batched (persistent kernels, CUDA graphs)", world=1):
    return {"workload": args.workload, "n": int(w["n"]), "m": int(w["m"]), "seed": int(w["seed"]), "k": args.k,
            "kprime": args.kprime, "k2": args.k2, "insert_batch": args.batch,
            "inserted_edges_per_step": int(w["ins_src"].shape[0]),
            "queries_per_step": int(w["q_u"].shape[0]), "form": form,
            "l2": "inputs larger than L2 (no flush)",
            "parallelism": "replicas" if world <= 1 else
            f"{world} replicas: every rank applies every insertion, rank r answers its 1/{world} slice of the queries"}


# ------------------------------------------------------------------ reference arm
def bench_reference(args):
    """The CPU oracle on the same workload: each step a bounded sample of the
    GPU step (its first 100,000 insertions, applied one by one with
    Algorithm 3, and its first 1,000,000 queries on every host core: the same
    1:10 mix), so that the whole run ends within minutes."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import dbl_inputs
    import oracle
    w = dbl_inputs.workload(args.workload)
    cores = cpu_cores()
    ref = oracle.OracleIndex(w["row_ptr"], w["col"], args.k, args.kprime).build(nthreads=cores)
    ref.mark()
    E = min(args.ref_insertions, int(w["ins_src"].shape[0]))
    Q = min(args.ref_queries, int(w["q_u"].shape[0]))
    batches = step_batches(E, args.batch)
    for _ in range(args.warmup):
        run_oracle_step(ref, w, batches, Q, cores)
    t_ins = t_q = 0.0
    for _ in range(args.steps):
        a, b = run_oracle_step(ref, w, batches, Q, cores)
        t_ins += a
        t_q += b
    total = t_ins + t_q
    value = args.steps * (E + Q) / total
    sample = (f"per step: the first {E} insertions of the GPU step (sequential, Algorithm 3) + its first {Q} "
              f"queries (Algorithm 2, {cores} threads)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(args, w, "CPU oracle (sequential insertion repair, threaded queries)"),
            "components": {"queries_per_s": args.steps * Q / t_q, "inserted_edges_per_s": args.steps * E / t_ins},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu_model": cpu_model(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(args, w):
    """The oracle, as it stands, on a bounded sample of the same step."""
    import oracle
    cores = cpu_cores()
    t0 = time.perf_counter()
    ref = oracle.OracleIndex(w["row_ptr"], w["col"], args.k, args.kprime).build(nthreads=cores)
    build_s = time.perf_counter() - t0
    ref.mark()
    e_s = min(args.ref_insertions, w["ins_src"].shape[0])
    q_s = min(args.ref_queries, w["q_u"].shape[0])
    t_ins, t_q = run_oracle_step(ref, w, step_batches(e_s, args.batch), q_s, cores)
    # the paper's sequential DBL: the same insertions, a tenth of the queries on one thread
    q_1 = max(1, q_s // 10)
    t_ins1, t_q1 = run_oracle_step(ref, w, step_batches(e_s, args.batch), q_1, 1)
    return {"value": (e_s + q_s) / (t_ins + t_q), "unit": UNIT, "cores": cores, "cpu_model": cpu_model(),
            "kind": "oracle",
            "sample": f"first {e_s} insertions (sequential, Algorithm 3) + first {q_s} queries "
                      f"(Algorithm 2, {cores} threads) of the step; same 1:10 mix",
            "inserted_edges_per_s": e_s / t_ins, "queries_per_s": q_s / t_q, "oracle_build_s": build_s,
            "single_thread": {"value": (e_s + 10 * q_1) / (t_ins1 + 10 * t_q1), "unit": UNIT,
                              "sample": f"first {e_s} insertions + first {q_1} queries on one thread, "
                                        f"queries scaled to the 1:10 mix",
                              "inserted_edges_per_s": e_s / t_ins1, "queries_per_s": q_1 / t_q1}}


# ------------------------------------------------------------------ GPU arm
def changed_bytes(ix, w, batches, deg_out0, deg_in0, rec_half_bytes, src_all, dst_all, group=False):
    """Algorithmic bytes of label repair for one step: per direction, over the
    vertices whose half-record changes in a batch (in the whole group of
    batches when they are applied together), offsets (8 B) + adjacency
    (4 B/edge) + neighbour record sectors (32 B/edge) + own write."""
    import torch
    ix.restore(0)
    ix.sync()
    deg_out = deg_out0.clone()
    deg_in = deg_in0.clone()
    total = 0.0
    prev = ix.labels()
    if group:
        batches = [(batches[0][0], batches[-1][1])] if batches else []
    for a, b in batches:
        ix.insert_edges(src_all[a:b], dst_all[a:b])
        cur = ix.labels()
        s, d = src_all[a:b].long(), dst_all[a:b].long()
        keep = s != d
        deg_out += torch.bincount(s[keep], minlength=deg_out.numel())
        deg_in += torch.bincount(d[keep], minlength=deg_in.numel())
        chf = (cur[0] != prev[0]).any(1) | (cur[2] != prev[2]).any(1)
        chb = (cur[1] != prev[1]).any(1) | (cur[3] != prev[3]).any(1)
        total += float((8 + 36 * deg_out[chf].double() + rec_half_bytes).sum())
        total += float((8 + 36 * deg_in[chb].double() + rec_half_bytes).sum())
        prev = cur
    ix.restore(0)
    ix.sync()
    return total


class Inputs:
    def __init__(self, w, dev):
        import torch
        self.rp = torch.from_numpy(w["row_ptr"]).to(dev)
        self.col = torch.from_numpy(w["col"]).to(dev)
        self.src = torch.from_numpy(w["ins_src"]).to(dev)
        self.dst = torch.from_numpy(w["ins_dst"]).to(dev)
        self.qu = torch.from_numpy(w["q_u"]).to(dev)
        self.qv = torch.from_numpy(w["q_v"]).to(dev)
        self.ans = torch.empty(w["q_u"].shape[0], dtype=torch.uint8, device=dev)
        self.code = torch.empty(w["q_u"].shape[0], dtype=torch.uint8, device=dev)


class Step:
    """One step of a form, in three parts: restore the built index, insert the
    step's edges batch by batch, answer the step's queries batch by batch.
    Eager (each part launched from the host) or replayed as three captured
    CUDA graphs; CUDA events on the current stream between the parts give the
    split of every step."""

    def __init__(self, ix, I, batches, qbatches, use_graph: bool, queries: bool = True, defer: bool = False):
        self.ix, self.I, self.batches, self.qbatches = ix, I, batches, qbatches
        self.use_graph, self.queries, self.defer = use_graph, queries, defer
        self.graphs = None
        self.launches_per_step = None

    def restore(self):
        self.ix.restore(0)

    def inserts(self):
        I = self.I
        for a, b in self.batches:
            self.ix.insert_edges(I.src[a:b], I.dst[a:b])

    def query(self):
        if not self.queries:
            return
        I = self.I
        for a, b in self.qbatches:
            self.ix.query(I.qu[a:b], I.qv[a:b], out=(I.ans[a:b], I.code[a:b]))

    def parts(self):
        return (self.restore, self.inserts, self.query)

    def capture(self):
        """Capture the three parts (after warm-up) and count their launches."""
        import torch
        if not self.use_graph:
            return
        l0 = self.ix.info()["launches"]
        self.graphs = []
        for i, part in enumerate(self.parts()):
            if i == 2 and not self.queries:
                self.graphs.append(None)  # nothing to capture
                continue
            if i == 1 and self.defer:
                # deferred insertions only queue on the host: queue them, and the
                # captured query part applies them (one launch) before answering
                part()
                self.graphs.append(None)
                continue
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                part()
            self.graphs.append(g)
        self.launches_per_step = self.ix.info()["launches"] - l0
        for g in self.graphs:
            if g is not None:
                g.replay()
        torch.cuda.synchronize()
        self.ix.sync()

    def __call__(self):
        import torch
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        run = ([g.replay if g is not None else (lambda: None) for g in self.graphs] if self.graphs
               else list(self.parts()))
        for i, f in enumerate(run):
            ev[i].record()
            f()
        ev[3].record()
        return ev


def time_steps(step, steps, world, tdist, sampler=None, profile=False):
    import torch
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    if profile:
        torch.cuda.profiler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    outs = [step() for _ in range(steps)]
    e1.record()
    torch.cuda.synchronize()
    if profile:
        torch.cuda.profiler.stop()
    if world > 1:
        tdist.barrier()
    clocks = sampler.stop() if sampler else None
    return e0.elapsed_time(e1), outs, clocks


FORM_FLAGS = {  # library flags of each form (FLAG_TIMING only in the separate timing passes)
    "plain": 0, "batched": "P|A", "graph": "P|A", "learned": "P|A", "learned_timing": "T|P|A",
    "deferred": "P|A|D", "deferred_timing": "T|P|A|D",
}


def form_flags(name, fine_l2=False):
    """The form's library flags; fine_l2 adds DBL_FLAG_FINE_L2 (a process-wide
    setting: the first index built with it sets it for every later kernel, so
    it is given to every form or to none)."""
    import paper_2101_09441_gb300 as dbl
    spec = FORM_FLAGS[name]
    f = dbl.FLAG_FINE_L2 if fine_l2 else 0
    for c in (spec.split("|") if spec else []):
        f |= {"P": dbl.FLAG_PERSISTENT, "A": dbl.FLAG_ASYNC, "T": dbl.FLAG_TIMING, "D": dbl.FLAG_DEFER}[c]
    return f


def decided_by(code_t):
    import torch
    code = torch.bincount(code_t.long(), minlength=8).cpu().numpy()
    return {n: int(code[i]) for i, n in enumerate(["undecided", "self", "dl", "bl", "thm1", "thm2", "bfs_pos",
                                                   "bfs_neg"])}


def run_form(name, args, w, I, k, kp, landmarks, leaves, batches, qbatches, world, tdist, local, steps,
             queries=True, autotune=True, sample_clocks=False, keep=False):
    """Build the form's index and time `steps` steps (restore, insertions,
    queries).  Returns a dict (with the index under "ix" when keep)."""
    import torch

    import paper_2101_09441_gb300 as dbl
    E = int(batches[-1][1]) if batches else 0
    Q = sum(int(b) - int(a) for a, b in qbatches) if (queries and qbatches) else 0  # this rank's queries
    flags = form_flags(name, args.fine_l2)
    kw = dict(flags=flags, team=args.team, edge_capacity=max(E, 1 << 20))
    if landmarks is not None:
        kw.update(landmarks=landmarks, leaf_buckets=leaves[0], leaf_roles=leaves[1])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ix = dbl.DBLIndex(I.rp, I.col, k, kp, **kw)
    ix.sync()
    build_s = time.perf_counter() - t0
    build_t = ix.timings() if flags & dbl.FLAG_TIMING else {}
    ix.snapshot(0)
    res = {"k": k, "kprime": kp, "landmarks": "learned" if landmarks is not None else "degree",
           "flags": FORM_FLAGS[name] or "0", "build_s": build_s}
    if build_t:
        res["build_kernel_ms"] = {kk: v[0] for kk, v in build_t.items() if v[1]}
        res["build_algorithmic_bytes"] = build_bytes(ix, I, ix.info()["record_bytes"] // 2)
        res["build_edges_relaxed"] = int(ix.stats()[10])
    if flags & dbl.FLAG_PERSISTENT and autotune and not args.no_autotune and E:
        # autotuned frontier schedule (sample: the step's insertions as one batch
        # and up to 1M queries); the persistent forms keep the fastest
        # persistent candidate
        nq = min(1_000_000, int(I.qu.numel()))
        tune = ix.autotune(I.src[:E], I.dst[:E], I.qu[:nq], I.qv[:nq], trials=3)
        team = min(tune["persistent_ms"], key=tune["persistent_ms"].get)
        ix.set_schedule(team, persistent=True)
        res["autotune"] = {"team": team, "persistent_ms": tune["persistent_ms"], "level_ms": tune["level_ms"]}
    use_graph = name in ("graph", "learned", "deferred")  # (timing passes launch each part eagerly)
    step = Step(ix, I, batches, qbatches, use_graph, queries, defer=bool(flags & dbl.FLAG_DEFER))
    for _ in range(args.warmup):
        for f in step.parts():
            f()
    torch.cuda.synchronize()
    ix.sync()
    step.capture()
    if not use_graph:
        ix.timings()
    l0 = ix.info()["launches"]
    sampler = ClockSampler(local) if sample_clocks else None
    total_ms, evs, clocks = time_steps(step, steps, world, tdist, sampler,
                                       profile=args.profile and name == args.profile_form)
    ix.sync()
    total_ms = max_over_ranks(total_ms, world, tdist, I.qu.device)
    split = [sum(ev[i].elapsed_time(ev[i + 1]) for ev in evs) / steps for i in range(3)]
    split = [max_over_ranks(x, world, tdist, I.qu.device) for x in split]
    ms = total_ms / steps
    res.update(ms_per_step=ms, value=whole_job_rate(steps * (E + Q), world, total_ms),
               restore_ms=split[0], insert_ms=split[1], query_ms=split[2],
               value_excl_restore=whole_job_rate(steps * (E + Q), world, steps * (ms - split[0])),
               inserted_edges_per_s=world * E / (split[1] * 1e-3) if E else None,
               queries_per_s=world * Q / (split[2] * 1e-3) if Q else None,
               gpu_launches=(step.launches_per_step * steps) if use_graph else ix.info()["launches"] - l0)
    if flags & dbl.FLAG_TIMING:
        res["kernels"] = {kk: {"ms_total": v[0], "launches": v[1]} for kk, v in ix.timings().items() if v[1]}
    # label-repair work of one step (edges relaxed), for the learned-vs-degree judge
    r0 = int(ix.stats()[10])
    ix.restore(0)
    step.inserts()
    ix.sync()
    res["relaxed_per_step"] = int(ix.stats()[10]) - r0
    if queries:
        step.query()
        ix.sync()
        res["decided_by"] = decided_by(I.code[qbatches[0][0]:qbatches[-1][1]])
        res["searched"] = res["decided_by"]["bfs_pos"] + res["decided_by"]["bfs_neg"]
    res["clocks"] = clocks
    if keep:
        res["ix"] = ix
    else:
        ix.close()
    return res


def build_bytes(ix, I, rec_half_bytes):
    """Algorithmic bytes of the label build (Algorithm 1 as one fixpoint):
    per direction, every vertex whose final half-record is non-zero pushes it
    once: offsets (8 B) + adjacency (4 B/edge) + neighbour record sectors
    (32 B/edge) + its own half-record."""
    import torch
    dl_in, dl_out, bl_in, bl_out = ix.labels()
    fwd = (dl_in != 0).any(1) | (bl_in != 0).any(1)
    bwd = (dl_out != 0).any(1) | (bl_out != 0).any(1)
    deg_out = torch.diff(I.rp).long()
    deg_in = torch.bincount(I.col.long(), minlength=deg_out.numel())
    return float((8 + 36 * deg_out[fwd].double() + rec_half_bytes).sum() +
                 (8 + 36 * deg_in[bwd].double() + rec_half_bytes).sum())


def insertion_bytes(ix, w, I):
    """Algorithmic bytes of appending and seeding one step's insertions (the
    persistent insertion kernel does both before it propagates): per edge its
    two ids (8 B), a read and a write of the segment word of each endpoint
    (4 x 32 B), the two label records read by the skip test (2 x 32 B), the two
    appended ids (2 x 32 B); applied edges also write back the two changed
    halves (2 x 32 B).  Self-loops: the ids only."""
    st = ix.stats()
    E = int(w["ins_src"].shape[0])
    loops = int((I.src == I.dst).sum().item())
    applied = int(st[11]) / max(1, int(st[11]) + int(st[12])) * (E - loops)
    return 8 * E + (E - loops) * (4 * 32 + 2 * 32 + 2 * 32) + applied * 2 * 32


MLP_FLOPS_PER_ROW = 2 * (16 * 128 + 128 * 128 + 128)  # the scorer's three layers


def scorer_roofline(ix, reps: int = 10):
    """Tensor-core roofline of the scorer's fused forward (k_mlp_forward) over
    every vertex's features, as at landmark selection: CUDA events around
    `reps` back-to-back launches on the current stream."""
    import torch

    import paper_2101_09441_gb300 as dbl
    peaks, src = measured_peaks()
    feats = ix.features()
    mlp = dbl.MLP(dbl.MLP.init_params(1))
    y = torch.empty(feats.shape[0], dtype=torch.float32, device=feats.device)
    for _ in range(3):
        mlp.forward(feats, out=y, sync=False)
    mlp.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        mlp.forward(feats, out=y, sync=False)
    e1.record()
    mlp.sync()
    ms = e0.elapsed_time(e1) / reps
    mlp.close()
    rows = int(feats.shape[0])
    ach = rows * MLP_FLOPS_PER_ROW / (ms * 1e-3) / 1e12
    return {"kernel": "k_mlp_forward (tcgen05, TMA)", "bound": "tensor", "achieved": ach,
            "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "frac": ach / peaks["bf16_tflops"], "traffic": None,
            "peak_source": f"bf16_tflops (burst) of {src}", "rows": rows, "flops_per_row": MLP_FLOPS_PER_ROW,
            "ms_per_launch": ms}


def build_roofline(form):
    """Achieved GB/s of the label build's propagation (CUDA events at build)."""
    peaks, src = measured_peaks()
    ms = form.get("build_kernel_ms", {}).get("propagate")
    alg = form.get("build_algorithmic_bytes")
    if not ms or not alg:
        return None
    ach = alg / (ms * 1e-3) / 1e9
    relaxed = form.get("build_edges_relaxed")
    prep = form.get("build_kernel_ms", {}).get("build_prep")
    return {"kernel": "propagate (label build)", "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "traffic": None, "peak_source": f"hbm_gbs of {src}",
            "algorithmic_bytes": alg, "ms": ms, "edges_relaxed": relaxed,
            "teps": relaxed / (ms * 1e-3) if relaxed else None,
            "prep_ms": prep, "build_ms": ms + prep if prep else None,
            "note": "ms: the propagation (seeds, frontier levels, record copies); prep_ms: the graph preparation "
                    "before it (CSR-in transpose, landmark and leaf selection, seeds, and on graphs whose records "
                    "exceed 256 MB the degree-grouped renumbering the propagation runs on)"}


def roofline(form, ix, steps, w, I, batches, persistent=True, group=False):
    """Achieved GB/s of the form's dominant kernel class (library CUDA events
    over the timed region) against the measured HBM copy peak.  In the
    persistent forms the `propagate` class is the insertion kernel (append,
    seeds and repair in one launch per batch); its fraction is given both
    with the append/seed bytes counted and with the repair bytes alone."""
    import torch
    peaks, src = measured_peaks()
    Q = int(w["q_u"].shape[0])
    info = ix.info()
    rec = info["record_bytes"]
    alg = {"query_label": steps * Q * (8 + 2 * rec + 2)}
    kern = form["kernels"]
    repair_only = None
    if "propagate" in kern:
        prop = changed_bytes(ix, w, batches, torch.diff(I.rp).long(), torch.bincount(I.col.long(), minlength=w["n"]),
                             rec // 2, I.src, I.dst, group=group)
        alg["propagate"] = steps * (prop + (insertion_bytes(ix, w, I) if persistent else 0))
        repair_only = steps * prop
    for kk, v in kern.items():
        v["ms_per_launch"] = v["ms_total"] / v["launches"]
        if kk in alg and v["ms_total"] > 0:
            v["algorithmic_bytes_per_launch"] = alg[kk] / v["launches"]
            v["achieved_gbs"] = alg[kk] / (v["ms_total"] * 1e-3) / 1e9
            v["frac_of_hbm"] = v["achieved_gbs"] / peaks["hbm_gbs"]
    dom = max(kern, key=lambda kk: kern[kk]["ms_total"])
    cand = dom if "achieved_gbs" in kern[dom] else max((kk for kk in kern if "achieved_gbs" in kern[kk]),
                                                       key=lambda kk: kern[kk]["ms_total"])

    def obj(kk):
        ach = kern[kk]["achieved_gbs"]
        tk = kk if kk != "propagate" else ("propagate_grouped" if group else "propagate_batch")
        traffic = NCU_TRAFFIC[tk][0] if tk in NCU_TRAFFIC and NCU_TRAFFIC[tk][1] == source_sha(tk) else None
        return {"kernel": kk, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": traffic, "peak_source": f"hbm_gbs of {src}",
                "algorithmic_bytes_per_launch": kern[kk]["algorithmic_bytes_per_launch"],
                "ms_per_launch": kern[kk]["ms_per_launch"]}
    out = obj(cand)
    out["dominant_kernel_by_time"] = dom
    if cand == "propagate":
        if repair_only is not None:
            ach_r = repair_only / (kern[cand]["ms_total"] * 1e-3) / 1e9
            out["repair_bytes_only"] = {"algorithmic_bytes_per_launch": repair_only / kern[cand]["launches"],
                                        "achieved": ach_r, "frac": ach_r / peaks["hbm_gbs"]}
        if form.get("relaxed_per_step") is not None:
            # repair traversal rate: edges relaxed per second of insertion-kernel time
            out["edges_relaxed_per_launch"] = form["relaxed_per_step"] * steps / kern[cand]["launches"]
            out["teps"] = form["relaxed_per_step"] * steps / (kern[cand]["ms_total"] * 1e-3)
    return out, (obj("query_label") if "achieved_gbs" in kern.get("query_label", {}) else None)


def public(f):
    return {kk: v for kk, v in f.items() if kk not in ("ix", "clocks")}


def train_learned(args, w, I, k, kp, batches, dev):
    """Train the scorer on the outcomes of a separate sample of queries on the
    plain index (degree landmarks) after the step's insertions; returns the
    learned landmark slots, the plain index's leaves, and the training facts."""
    import torch

    import dbl_inputs
    import paper_2101_09441_gb300 as dbl
    from paper_2101_09441_gb300 import learned as L
    E = int(batches[-1][1])
    t0 = time.perf_counter()
    tu, tv = dbl_inputs.queries(w["row_ptr"], w["col"], args.train_queries, w["seed"] + 300, False,
                                w["ins_src"], w["ins_dst"])
    tu, tv = torch.from_numpy(tu).to(dev), torch.from_numpy(tv).to(dev)
    plain_ix = dbl.DBLIndex(I.rp, I.col, k, kp, edge_capacity=max(E, 1 << 20))
    for a, b in batches:
        plain_ix.insert_edges(I.src[a:b], I.dst[a:b])
    base_slots = max(1, k // 8)
    if args.learn_rounds > 1:
        lm, tinfo = L.select_in_rounds(plain_ix, I.rp, I.col, (tu, tv), k, kp, base_slots, args.learn_rounds,
                                       idx_kw={"edge_capacity": max(E, 1 << 20)},
                                       inserts=[(I.src[a:b], I.dst[a:b]) for a, b in batches], steps=args.train_steps)
    else:
        scores, tinfo = L.train_scorer(plain_ix, tu, tv, base_slots, steps=args.train_steps)
        lm = L.select_landmarks(plain_ix, scores, k, base_slots)
    _, lb, lr_ = plain_ix.selection()
    torch.cuda.synchronize()
    info = {"train_s": time.perf_counter() - t0, "base_slots": base_slots, "rounds": args.learn_rounds,
            **{kk: v for kk, v in tinfo.items() if kk != "losses"}, "final_loss": tinfo["losses"][-1]}
    return lm, (lb, lr_), info, plain_ix


def learned_judge(learned, ref):
    """Keep the learned landmarks only if they send no more pairs to the
    search than the degree rule and keep the insertions' repair cheap."""
    from paper_2101_09441_gb300 import learned as L
    return not (learned["searched"] <= ref["searched"] and L.repair_ok(ref["relaxed_per_step"],
                                                                        learned["relaxed_per_step"]))


def gain(deg, lrn):
    """What the learned landmarks change against the degree rule, same k."""
    keys = ("ms_per_step", "value", "queries_per_s", "inserted_edges_per_s", "relaxed_per_step", "searched")
    out = {"degree": {kk: deg.get(kk) for kk in keys}, "learned": {kk: lrn.get(kk) for kk in keys}}
    out["degree"]["decided_by_dl"] = deg["decided_by"]["dl"]
    out["learned"]["decided_by_dl"] = lrn["decided_by"]["dl"]
    out["dl_decided_delta"] = lrn["decided_by"]["dl"] - deg["decided_by"]["dl"]
    out["searched_delta"] = lrn["searched"] - deg["searched"]
    out["value_ratio"] = lrn["value"] / deg["value"]
    return out


def restore_batches(sizes):
    out, a = [], 0
    for s in sizes:
        out.append((a, a + int(s)))
        a += int(s)
    return out


def bench_extras(args, world, tdist, local, dev):
    """Extra timed forms on the social workload (stand-in for LiveJournal's
    size): insertion throughput at batch sizes 1k, 10k and 100k (persistent +
    CUDA graph, and plain), and the batched configuration (k = 128,
    log-uniform insertion batches of 1..200k edges and query batches of
    1k..4M pairs) in the graph form against the plain form."""
    import dbl_inputs
    w = dbl_inputs.workload("social")
    I = Inputs(w, dev)
    E, Q = int(w["ins_src"].shape[0]), int(w["q_u"].shape[0])
    steps = args.extra_steps
    out = {"workload": "social", "n": int(w["n"]), "m": int(w["m"]), "steps": steps,
           "inserted_edges_per_step": E, "queries_per_step": Q}
    bs = {}
    for b in (1000, 10_000, 100_000):
        batches = step_batches(E, b)
        row = {}
        for name in ("graph", "plain"):
            r = run_form(name, args, w, I, 64, 64, None, None, batches, None, world, tdist, local, steps,
                         queries=False, autotune=False)
            row[name] = {kk: r[kk] for kk in ("insert_ms", "restore_ms", "inserted_edges_per_s", "gpu_launches",
                                              "relaxed_per_step")}
            row[name]["us_per_batch"] = 1e3 * r["insert_ms"] / len(batches)
        row["graph_vs_plain"] = row["graph"]["inserted_edges_per_s"] / row["plain"]["inserted_edges_per_s"]
        bs[str(b)] = row
    out["insert_batch_sizes"] = bs
    ins_sizes = dbl_inputs.loguniform_batches(E, 1, 200_000, 11)
    q_sizes = dbl_inputs.loguniform_batches(Q, 1000, 4_000_000, 12)
    ib, qb = restore_batches(ins_sizes), restore_batches(q_sizes)
    cfg = {"k": 128, "kprime": 64, "insert_batches": len(ib), "query_batches": len(qb),
           "insert_sizes": "floor(exp(U[0, ln 200001)))", "query_sizes": "floor(exp(U[ln 1000, ln 4000001)))"}
    for name in ("graph", "plain"):
        r = run_form(name, args, w, I, 128, 64, None, None, ib, qb, world, tdist, local, steps, autotune=False)
        cfg[name] = public(r)
    cfg["graph_vs_plain"] = cfg["graph"]["value"] / cfg["plain"]["value"]
    out["batched_config"] = cfg
    return out


def learned_gain_community(args, dev, reps=10):
    """What the learned landmarks gain on a graph with several strongly
    connected parts of real size (on R-MAT it gains nothing measurable):
    128 R-MAT communities of power-law sizes (community c holds a share
    proportional to 1/(c+1)) joined by 2% of the edges, always from an earlier
    to a later community (dbl_inputs.community_dag), n = 500,000, m = 5M.
    Degree landmarks against the learned selection in 7 rounds (k = k' = 64),
    trained on the outcomes of 100k sampled queries and judged on 100k
    others; then 1M further queries (label test + search, persistent kernels)
    are timed with each landmark set (CUDA events, mean of `reps`)."""
    import torch

    import dbl_inputs
    import paper_2101_09441_gb300 as dbl
    from paper_2101_09441_gb300 import learned as L
    t0 = time.perf_counter()
    n, m, comm = 500_000, 5_000_000, 128
    rp, col = dbl_inputs.community_dag(n, m, comm, 1.0, 0.02, 21)
    qu, qv = dbl_inputs.queries(rp, col, 1_200_000, 22, False)

    def dev_t(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    tq = (dev_t(qu[:100_000]), dev_t(qv[:100_000]))
    ev = (dev_t(qu[100_000:200_000]), dev_t(qv[100_000:200_000]))
    tu, tv = dev_t(qu[200_000:]), dev_t(qv[200_000:])
    flags = dbl.FLAG_PERSISTENT | dbl.FLAG_ASYNC | (dbl.FLAG_FINE_L2 if args.fine_l2 else 0)
    plain, chosen, learned, info = L.learned_index(dev_t(rp), dev_t(col), tq, ev, k=64, kprime=64, rounds=7,
                                                   steps=args.train_steps, flags=flags)
    out = {"graph": "community_dag", "n": n, "m": int(col.shape[0]), "communities": comm, "alpha": 1.0,
           "cross": 0.02, "k": 64, "kprime": 64, "rounds": 7, "timed_queries": int(tu.numel()),
           "setup_s": time.perf_counter() - t0, "judge_keeps_learned": not info["fallback"],
           "judge_pairs": {"degree": info["eval_plain"], "learned": info["eval_learned"]}}
    ans = torch.empty(tu.numel(), dtype=torch.uint8, device=dev)
    code = torch.empty_like(ans)
    ref = None
    for name, ix in (("degree", plain), ("learned", learned)):
        for _ in range(3):
            ix.query(tu, tv, out=(ans, code))
        ix.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            ix.query(tu, tv, out=(ans, code))
        e1.record()
        ix.sync()
        ms = e0.elapsed_time(e1) / reps
        c = code.long()
        out[name] = {"ms_per_batch": ms, "queries_per_s": tu.numel() / (ms * 1e-3),
                     "decided_by_dl": int((c == dbl.CODE_DL).sum()),
                     "searched": int(((c == dbl.CODE_BFS_POS) | (c == dbl.CODE_BFS_NEG)).sum())}
        if ref is None:
            ref = ans.clone()
        else:
            out["same_answers"] = bool(torch.equal(ref, ans))
    out["queries_per_s_ratio"] = out["learned"]["queries_per_s"] / out["degree"]["queries_per_s"]
    plain.close()
    learned.close()
    return out


def bench_gpu(args):
    import torch
    import torch.distributed as tdist

    import dbl_inputs
    import paper_2101_09441_gb300 as dbl

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=dev)
    dbl.build()
    w = dbl_inputs.workload(args.workload)
    E, Q = int(w["ins_src"].shape[0]), int(w["q_u"].shape[0])
    batches = step_batches(E, args.batch)
    # replicas: every rank applies every insertion batch; the query batch is
    # sharded, rank r answering its slice (no collective on the data path)
    q_lo, q_hi = shard_range(Q, rank, world)
    qbatches = [(q_lo, q_hi)]
    I = Inputs(w, dev)
    k, kp, k2 = args.k, args.kprime, args.k2
    S = args.steps
    common = (world, tdist, local)
    forms = {}
    for name in ("plain", "batched", "graph"):
        if name in args.forms:
            forms[name] = run_form(name, args, w, I, k, kp, None, None, batches, qbatches, *common, S)

    # ---- learned landmarks (top-k scored) against degree landmarks, same k
    lm, leaves, linfo, plain_ix = train_learned(args, w, I, k, kp, batches, dev)
    roof_scorer = scorer_roofline(plain_ix)
    plain_ix.close()
    learned = run_form("learned", args, w, I, k, kp, lm, leaves, batches, qbatches, *common, S,
                       sample_clocks=True, keep=True)
    learned_t = run_form("learned_timing", args, w, I, k, kp, lm, leaves, batches, qbatches, *common, S,
                         keep=True)
    # the headline: the same step with the insertion batches queued and applied
    # as one group by the query call that follows them (DBL_FLAG_DEFER: the
    # device work queue of uneven batches; each query observes exactly the
    # insertions queued before it); its split puts the insertions inside the
    # query part.  Its own timing pass gives the roofline figures.
    grouped = "deferred" in args.forms
    deferred = run_form("deferred", args, w, I, k, kp, lm, leaves, batches, qbatches, *common, S,
                        sample_clocks=True, keep=True) if grouped else None
    deferred_t = run_form("deferred_timing", args, w, I, k, kp, lm, leaves, batches, qbatches, *common, S,
                          keep=True) if grouped else None
    ref_form = forms.get("graph") or forms.get("batched") or forms.get("plain")
    fallback = learned_judge(learned, ref_form) if ref_form else False
    if fallback and "graph" in forms:
        head = forms["graph"]
    else:
        head = deferred if grouped else learned
    timing = deferred_t if grouped else learned_t
    roof, roof_label = roofline(timing, timing["ix"], S, w, I, batches, group=grouped)
    roof_per_batch = roofline(learned_t, learned_t["ix"], S, w, I, batches)[0] if grouped else None
    learned_t["ix"].close()
    if grouped:
        deferred_t["ix"].close()

    # ---- the same comparison at k2 landmarks (two words per direction at 128)
    k2_forms = {}
    if k2:
        for name in ("plain", "graph"):
            k2_forms[name] = run_form(name, args, w, I, k2, kp, None, None, batches, qbatches, *common, S)
        lm2, leaves2, linfo2, pix2 = train_learned(args, w, I, k2, kp, batches, dev)
        pix2.close()
        if not args.no_serve:
            # serving on the learned k2 index (the serving configuration of the workload)
            k2_forms["serving"] = serving_pass(w, I, k2, kp, lm2, leaves2, args.serve_requests)
        k2_forms["learned"] = run_form("learned", args, w, I, k2, kp, lm2, leaves2, batches, qbatches, *common, S)
        k2_forms["learned"]["training"] = linfo2
        k2_forms["fallback_to_degree_rule"] = learned_judge(k2_forms["learned"], k2_forms["graph"])
        k2_forms["learned_vs_plain"] = k2_forms["learned"]["value"] / k2_forms["plain"]["value"]

    # ---- end to end through the host-buffer C-ABI calls, on the headline's
    # index and form (grouped: the uploaded batches wait in the queue and the
    # query call applies them as one launch)
    e2e_form = deferred if head is deferred else learned
    for f in (learned, deferred):
        if f is not None and f is not e2e_form:
            f["ix"].close()
    ix = e2e_form["ix"]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    h_src, h_dst = pin(w["ins_src"]), pin(w["ins_dst"])
    h_qu, h_qv = pin(w["q_u"][q_lo:q_hi]), pin(w["q_v"][q_lo:q_hi])
    h_ans = torch.empty(q_hi - q_lo, dtype=torch.uint8).pin_memory().numpy()
    e2e_steps = 0 if args.no_e2e else S

    def e2e_step():
        ix.restore(0)
        for a, b in batches:
            ix.insert_edges_host(h_src[a:b], h_dst[a:b])
        ix.query_host(h_qu, h_qv, out=(h_ans, None))

    if e2e_steps:
        for _ in range(args.warmup):  # the host forms' staging buffers are allocated here
            e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        tdist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, tdist, dev)
    ix.close()

    extras = None if args.no_extras else bench_extras(args, *common, dev)
    gain_comm = None if args.no_extras or rank != 0 else learned_gain_community(args, dev)

    gain_k = gain(ref_form, learned) if ref_form else None
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": S,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(args, w, world=world, form=(
                "learned+batched (persistent kernels, CUDA graphs; the step's insertion batches queued and "
                "applied as one group before its queries)" if head is deferred else
                "learned+batched (persistent kernels, CUDA graphs; one launch per insertion batch)")),
            "forms": {**{kk: public(v) for kk, v in forms.items()}, "learned": public(learned),
                      "learned_timing_pass": public(learned_t),
                      **({"learned_grouped": public(deferred), "learned_grouped_timing_pass": public(deferred_t)}
                         if grouped else {})},
            "learned_vs_plain": head["value"] / forms["plain"]["value"] if "plain" in forms else None,
            "learned": {"fallback_to_degree_rule": bool(fallback), **linfo},
            "learned_gain": {f"k{k}": gain_k,
                             **({f"k{k2}": gain(k2_forms["graph"], k2_forms["learned"])} if k2 else {})},
            "learned_gain_community": gain_comm,
            f"forms_k{k2}": {kk: (public(v) if isinstance(v, dict) else v) for kk, v in k2_forms.items()
                             if kk != "serving"} if k2 else None,
            "restore": {"ms": head["restore_ms"], "share_of_step": head["restore_ms"] / head["ms_per_step"],
                        "value_excl_restore": head["value_excl_restore"],
                        "note": "dbl_restore returns the index to its built state at the start of every step "
                                "(labels and adjacency metadata copied back); it is not part of the method"},
            "roofline": roof,
            "roofline_per_batch_insertion": roof_per_batch,
            "roofline_label_test": roof_label,
            "roofline_build": build_roofline(timing),
            "roofline_scorer": roof_scorer,
            "e2e": {"value": world * e2e_steps * (E + q_hi - q_lo) / e2e_s if e2e_steps else None, "unit": UNIT,
                    "h2d_bytes_per_step": 8 * (E + q_hi - q_lo), "d2h_bytes_per_step": q_hi - q_lo},
            "serving": k2_forms.get("serving"),
            "extras": extras,
            "clocks": head["clocks"] or learned["clocks"],
            "gpu_launches": head["gpu_launches"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, w)
    add_nominal(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        tdist.destroy_process_group()


# ------------------------------------------------------------------ serving
def serve_requests(w, count, seed, q_off=0, e_off=0):
    """`count` requests: 90% query batches, 10% insertion batches, sizes
    floor(exp(U[0, ln 65537))) clamped to >= 1; queries and edges are taken in
    order from the workload's streams (queries wrap around, edges do not)."""
    rng = np.random.default_rng(seed)
    Q, E = w["q_u"].shape[0], w["ins_src"].shape[0]
    out = []
    for _ in range(count):
        size = max(1, int(np.exp(rng.uniform(0.0, np.log(65537.0)))))
        if rng.random() < 0.1:
            size = min(size, E - e_off)
            if size <= 0:
                continue
            out.append((1, w["ins_src"][e_off:e_off + size], w["ins_dst"][e_off:e_off + size]))
            e_off += size
        else:
            a = q_off % Q
            size = min(size, Q - a)
            out.append((0, w["q_u"][a:a + size], w["q_v"][a:a + size]))
            q_off += size
    return out, q_off, e_off


def run_serving(srv, reqs, rate=None, seed=0):
    """Submit the requests (Poisson arrivals at `rate` requests/s, or as fast
    as the engine admits them), wait for all, and return the engine's report."""
    import threading

    import paper_2101_09441_gb300 as dbl
    srv.reset_stats()
    tickets = []
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, len(reqs)) if rate else np.zeros(len(reqs))
    done = threading.Event()
    errors = []

    def waiter():
        i = 0
        while i < len(reqs):
            if i < len(tickets):
                try:
                    srv.wait(tickets[i])
                except Exception as e:  # noqa: BLE001 - reported below
                    errors.append(str(e))
                i += 1
            else:
                time.sleep(1e-5)
        done.set()

    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    t0 = time.perf_counter()
    t_next = t0
    for (kind, a, b), gap in zip(reqs, gaps):
        t_next += gap
        while True:
            now = time.perf_counter()
            if now >= t_next:
                break
            time.sleep(min(t_next - now, 1e-4))
        while True:
            try:
                tickets.append(srv.submit(kind, a, b))
                break
            except dbl.DblError as e:
                if e.status != dbl.DBL_ERR_BUSY:
                    raise
                time.sleep(1e-5)
    done.wait()
    wall = time.perf_counter() - t0
    rep = srv.report()
    rep["wall_s"] = wall
    rep["requests_per_s"] = len(reqs) / wall
    rep["pairs_per_s"] = rep["pairs"] / wall
    rep["edges_per_s"] = rep["edges"] / wall
    rep["errors"] = errors[:3]
    return rep


def serving_pass(w, I, k, kp, lm, leaves, n_req, slots=4):
    """Serving on a resident index with the given landmarks: a closed-loop run
    gives the peak request rate, then Poisson streams at 50% and 90% of it
    report p50/p99 latency per request kind and sustained pairs/s and
    edges/s.  Every run starts from the built index; one server serves all
    runs (a warm-up run first admits its slots)."""
    import paper_2101_09441_gb300 as dbl
    E = int(w["ins_src"].shape[0])
    ix = dbl.DBLIndex(I.rp, I.col, k, kp, landmarks=lm, leaf_buckets=leaves[0], leaf_roles=leaves[1],
                      edge_capacity=max(2 * E, 1 << 20), flags=dbl.FLAG_PERSISTENT)
    ix.sync()
    ix.snapshot(0)

    srv = dbl.Server(ix, slots=slots)

    def run(reqs, rate, seed):
        srv.drain()  # nothing in flight: the index goes back to its built state
        ix.restore(0)
        ix.sync()
        return run_serving(srv, reqs, rate, seed)

    try:
        # the warm-up run admits the slots (each set up once, when the free
        # memory allows and requests wait); the measured runs reuse them
        warm, _, _ = serve_requests(w, max(1, n_req // 2), 99)
        run(warm, None, 0)
        reqs, _, _ = serve_requests(w, n_req, 100)
        peak = run(reqs, None, 0)
        loads = {}
        for i, frac in enumerate((0.5, 0.9)):
            reqs, _, _ = serve_requests(w, n_req, 200 + i, q_off=(i + 1) * 3_000_000)
            loads[str(frac)] = run(reqs, frac * peak["requests_per_s"], 300 + i)
    finally:
        srv.close()
        ix.close()
    return {"k": k, "kprime": kp, "slots": slots, "requests_per_run": n_req,
            "mix": "90% query / 10% insertion requests, sizes floor(exp(U[0, ln 65537)))",
            "closed_loop_peak": peak, "poisson": loads}


def bench_serve(args):
    """Serving measurement: the learned index (k = 128, k' = 64) resident on
    the device behind dbl_server; a closed-loop run gives the peak request
    rate, then Poisson streams at 50% and 90% of it report p50/p99 latency and
    sustained throughput.  One JSON line."""
    import torch

    import dbl_inputs
    import paper_2101_09441_gb300 as dbl
    dbl.build()
    w = dbl_inputs.workload(args.serve_workload)
    dev = torch.device("cuda", 0)
    I = Inputs(w, dev)
    E = int(w["ins_src"].shape[0])
    k, kp = 128, 64
    t0 = time.perf_counter()
    lm, leaves, tinfo, plain = train_learned(args, w, I, k, kp, step_batches(E, args.batch), dev)
    plain.close()
    setup_s = time.perf_counter() - t0
    rep = serving_pass(w, I, k, kp, lm, leaves, args.serve_requests)
    line = {"metric": "serving: p50/p99 latency and sustained throughput under Poisson load", "impl": "dbl",
            "workload": args.serve_workload, "n": int(w["n"]), "m": int(w["m"]), "landmarks": "learned",
            "setup_s": setup_s, **rep, "learned": tinfo}
    print(json.dumps(line), flush=True)


def bench_sweep(args):
    """Label widths, leaf threshold and landmark ranking (Section 6, Table 5,
    Table 3 and "Label Node Selection"): the batched step (persistent kernels)
    at k, k' in {64, 128, 256} and at the small widths 16 and 32 (with each
    other and with 64) with M-ranked landmarks and zero-degree leaves;
    at k = k' = 64 with leaves M(u) <= r for r in {2, 16}, and with Table 3's
    rankings A, B, C.  One JSON line with a row per
    configuration: step time, throughput, per-kernel times (CUDA events), the
    label test's achieved HBM fraction and which rule decided each query."""
    import torch

    import dbl_inputs
    import paper_2101_09441_gb300 as dbl
    dbl.build()
    dbl_inputs.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = dbl_inputs.workload(args.workload)
    E, Q = int(w["ins_src"].shape[0]), int(w["q_u"].shape[0])
    I = Inputs(w, dev)
    batches = step_batches(E, args.batch)
    peaks, src = measured_peaks()
    configs = ([(k, kp, 0, "M", 0) for k in (64, 128, 256) for kp in (64, 128, 256)] +
               [(k, kp, 0, "M", 0) for k, kp in ((16, 16), (32, 32), (16, 64), (64, 16), (32, 64), (64, 32))] +
               [(64, 64, 2, "M", 0), (64, 64, 16, "M", 0), (64, 64, 0, "A", 0), (64, 64, 0, "B", 0),
                (64, 64, 0, "C", 0)] +
               [(128, 64, 0, "M", qpt) for qpt in (1, 4)] + [(256, 64, 0, "M", qpt) for qpt in (1, 4)])
    rows = []
    for k, kp, r, rule, qpt in configs:
        ix = dbl.DBLIndex(I.rp, I.col, k, kp, leaf_r=r, landmark_rule=rule, edge_capacity=max(E, 1 << 20),
                          query_unroll=qpt, flags=dbl.FLAG_PERSISTENT | dbl.FLAG_ASYNC | dbl.FLAG_TIMING |
                          (dbl.FLAG_FINE_L2 if args.fine_l2 else 0))
        ix.sync()
        ix.snapshot(0)
        step = Step(ix, I, batches, [(0, Q)], use_graph=False)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        ix.timings()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        t = ix.timings()
        rec = ix.info()["record_bytes"]
        code = torch.bincount(I.code.long(), minlength=8).cpu().numpy()
        lab_ms = t["query_label"][0] / max(1, t["query_label"][1])
        leaves = int((ix.selection()[2] > 0).sum().item())
        rows.append({"k": k, "kprime": kp, "leaf_r": r, "landmark_rule": rule,
                     "query_unroll": qpt or (2 if rec == 32 else 4),  # the library's default when 0
                     "record_bytes": rec, "leaves": leaves, "ms_per_step": ms,
                     "ops_per_s": (E + Q) / (ms * 1e-3),
                     "insert_ms_per_batch": t["propagate"][0] / max(1, t["propagate"][1]),
                     "label_test_ms": lab_ms,
                     "label_test_frac_of_hbm": Q * (8 + 2 * rec + 2) / (lab_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                     "search_ms": t["search_expand"][0] / max(1, t["search_expand"][1]),
                     "decided_by": {n: int(code[i]) for i, n in enumerate(
                         ["undecided", "self", "dl", "bl", "thm1", "thm2", "bfs_pos", "bfs_neg"])}})
        ix.close()
    print(json.dumps({"metric": "label width / leaf threshold sweep (batched step)", "unit": UNIT,
                      "workload": args.workload, "steps": args.steps, "warmup": args.warmup,
                      "peak_source": f"hbm_gbs of {src}", "sweep": rows}), flush=True)


def bench_kernel_case(args):
    """A small, single-index run of one kernel for an ncu capture: `label`
    builds the index (k, k'), applies the workload's insertions and answers
    its query batch `args.steps` times; `insert` applies the insertions in
    batches of `args.batch` (persistent kernels, asynchronous calls; with
    `args.defer` queued and applied as one group).  Prints
    per-kernel CUDA-event times (one JSON line)."""
    import torch

    import dbl_inputs
    import paper_2101_09441_gb300 as dbl
    dbl.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = dbl_inputs.workload(args.workload, with_queries=args.kernel_case == "label")
    I = Inputs(w, dev) if args.kernel_case == "label" else None
    if args.kernel_case == "scorer":
        # the scorer's fused forward over every vertex's features (tcgen05, TMA)
        rp = torch.from_numpy(w["row_ptr"]).to(dev)
        col = torch.from_numpy(w["col"]).to(dev)
        ix = dbl.DBLIndex(rp, col, args.k, args.kprime, flags=dbl.FLAG_PERSISTENT)
        r = scorer_roofline(ix, reps=max(1, args.steps))
        ix.close()
        print(json.dumps({"kernel_case": "scorer", "workload": args.workload, **r}), flush=True)
        return
    rp = torch.from_numpy(w["row_ptr"]).to(dev)
    col = torch.from_numpy(w["col"]).to(dev)
    src, dst = torch.from_numpy(w["ins_src"]).to(dev), torch.from_numpy(w["ins_dst"]).to(dev)
    E = int(src.numel())
    flags = dbl.FLAG_PERSISTENT | dbl.FLAG_TIMING | (dbl.FLAG_FINE_L2 if args.fine_l2 else 0)
    if args.kernel_case == "insert":
        flags |= dbl.FLAG_ASYNC | (dbl.FLAG_DEFER if args.defer else 0)
    ix = dbl.DBLIndex(rp, col, args.k, args.kprime, edge_capacity=max(E, 1 << 20), flags=flags,
                      build_order=args.build_order)
    ix.sync()
    ix.timings()
    for a, b in step_batches(E, args.batch):
        ix.insert_edges(src[a:b], dst[a:b])
    ix.sync()
    if args.kernel_case == "label":
        for _ in range(args.steps):
            ix.query(I.qu, I.qv, out=(I.ans, I.code))
        ix.sync()
    t = ix.timings()
    print(json.dumps({"kernel_case": args.kernel_case, "workload": args.workload, "k": args.k,
                      "kprime": args.kprime, "fine_l2": bool(args.fine_l2), "defer": bool(args.defer),
                      "ms_per_launch": {kk: v[0] / max(1, v[1]) for kk, v in t.items() if v[1]},
                      "launches": {kk: v[1] for kk, v in t.items() if v[1]}}), flush=True)
    ix.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["dbl", "reference"], default="dbl")
    ap.add_argument("--workload", default="large", choices=["large", "social", "tiny"])
    ap.add_argument("--batch", type=int, default=100_000)
    ap.add_argument("--k", type=int, default=64)
    ap.add_argument("--k2", type=int, default=128, help="second landmark count compared (0: none)")
    ap.add_argument("--kprime", type=int, default=64)
    ap.add_argument("--team", type=int, default=0, help="frontier team width; 0: library default (1)")
    ap.add_argument("--no-autotune", action="store_true", help="skip the autotuner in the persistent forms")
    ap.add_argument("--forms", default="plain,batched,graph,deferred",
                    help="comparison forms to time besides the headline")
    ap.add_argument("--train-queries", type=int, default=1_000_000)
    ap.add_argument("--train-steps", type=int, default=400)
    ap.add_argument("--learn-rounds", type=int, default=1,
                    help="learned selection in rounds (the index rebuilt with the picks so far before each)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-insertions", type=int, default=100_000, help="oracle sample: insertions per step")
    ap.add_argument("--ref-queries", type=int, default=1_000_000, help="oracle sample: queries per step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the extra forms on the social workload")
    ap.add_argument("--extra-steps", type=int, default=5, help="timed steps of each extra form")
    ap.add_argument("--profile", action="store_true",
                    help="bracket one form's timed region with cudaProfilerStart/Stop (ncu --profile-from-start off)")
    ap.add_argument("--profile-form", default="learned_timing")
    ap.add_argument("--serve", action="store_true", help="serving measurement instead of the step benchmark")
    ap.add_argument("--serve-workload", default="large", choices=["large", "social", "tiny"])
    ap.add_argument("--serve-requests", type=int, default=1500)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving pass of the step benchmark")
    ap.add_argument("--sweep", action="store_true", help="label width / leaf threshold sweep instead of the step")
    ap.add_argument("--kernel-case", choices=["label", "insert", "scorer"], default=None,
                    help="a small single-index run of one kernel (for an ncu capture) instead of the step")
    ap.add_argument("--build-order", type=int, default=0,
                    help="kernel cases: dbl_options.build_order (1 renumbered build, -1 id order, 0 by size)")
    ap.add_argument("--defer", action="store_true",
                    help="kernel case insert: queue the batches and apply them as one group (DBL_FLAG_DEFER)")
    ap.add_argument("--fine-l2", action=argparse.BooleanOptionalAction, default=True,
                    help="DBL_FLAG_FINE_L2 in every form: 32-byte L2 fetch granularity for the whole process "
                         "(default on; --no-fine-l2 keeps the driver's default)")
    args = ap.parse_args()
    args.forms = [f for f in args.forms.split(",") if f]
    if args.warmup < 3:
        args.warmup = 3
    if args.kernel_case:
        bench_kernel_case(args)
    elif args.serve:
        bench_serve(args)
    elif args.sweep:
        bench_sweep(args)
    elif args.impl == "reference":
        bench_reference(args)
    else:
        bench_gpu(args)


if __name__ == "__main__":
    main()
