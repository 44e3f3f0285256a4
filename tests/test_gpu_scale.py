"""GPU path vs the CPU oracle at the social-network scale (n = 4,847,571,
m = 68,993,773), in the launch configurations the benchmark times.

Every label word after 1,000,000 insertions and every answer and deciding
rule of the 10,000,000 queries are compared with the oracle, which inserts the
edges one at a time (Algorithm 3 and its mirrors) and answers each query with
Algorithm 2.  The labels are the unique least fixpoint, so incremental repair,
any batching and any GPU schedule must give the same words.
"""
import os

import numpy as np
import pytest
import torch

import dbl_inputs
import oracle
import paper_2101_09441_gb300 as dbl
from paper_2101_09441_gb300 import learned as L

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


def D(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def labels_np(ix):
    return [t.cpu().numpy().view(np.uint64) for t in ix.labels()]


def assert_same_labels(got, want, what):
    for a, b, name in zip(got, want, ("dl_in", "dl_out", "bl_in", "bl_out")):
        if not np.array_equal(a, b):
            bad = np.nonzero((a != b).any(axis=1))[0]
            raise AssertionError(f"{what}: {name} differs at {bad.size} vertices, first {bad[:8]}")


def assert_same_answers(ans, code, rans, rcode, what):
    a, c = ans.cpu().numpy(), code.cpu().numpy()
    bad = np.nonzero((a != rans) | (c != rcode))[0]
    assert bad.size == 0, f"{what}: {bad.size} of {a.size} queries differ, first {bad[:5]}"


@pytest.fixture(scope="module")
def social():
    dbl.build()
    dbl_inputs.build()
    oracle.build()
    w = dbl_inputs.workload("social")
    w["d"] = {k: D(w[k]) for k in ("row_ptr", "col", "ins_src", "ins_dst", "q_u", "q_v")}
    return w


@pytest.fixture(scope="module")
def oracle64(social):
    """Degree landmarks, k = k' = 64: labels after build, after all insertions,
    and the answers to every query."""
    w = social
    ref = oracle.OracleIndex(w["row_ptr"], w["col"], 64, 64).build(nthreads=THREADS)
    built = ref.labels()
    ref.insert_edges(w["ins_src"], w["ins_dst"])
    final = ref.labels()
    rans, rcode = ref.query(w["q_u"], w["q_v"], nthreads=THREADS)
    return dict(built=built, final=final, ans=rans, code=rcode)


def insert_batches(ix, w, sizes):
    src, dst = w["d"]["ins_src"], w["d"]["ins_dst"]
    a = 0
    for b in sizes:
        ix.insert_edges(src[a:a + b], dst[a:a + b])
        a += b
    assert a == src.numel()


def test_social_build_and_every_batch_size(social, oracle64):
    """Label build, then the 1M insertions in batches of 1k (host-driven
    levels), 10k (persistent, asynchronous) and 100k (persistent, captured in a
    CUDA graph), each from the same snapshot: all equal the oracle's labels."""
    w = social
    E = int(w["ins_src"].shape[0])
    ix = dbl.DBLIndex(w["d"]["row_ptr"], w["d"]["col"], 64, 64, edge_capacity=E, flags=dbl.FLAG_ASYNC)
    ix.sync()
    assert_same_labels(labels_np(ix), oracle64["built"], "social build")
    ix.snapshot(0)
    insert_batches(ix, w, [1000] * (E // 1000))
    assert_same_labels(labels_np(ix), oracle64["final"], "batches of 1k, level by level")

    ix.restore(0)
    ix.set_schedule(1, persistent=True)
    insert_batches(ix, w, [10_000] * (E // 10_000))
    ix.sync()
    assert_same_labels(labels_np(ix), oracle64["final"], "batches of 10k, persistent")

    ix.restore(0)
    ix.sync()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ix.restore(0)
        insert_batches(ix, w, [100_000] * (E // 100_000))
    g.replay()
    g.replay()  # a replay starts from the snapshot again: same result
    torch.cuda.synchronize()
    ix.sync()
    assert_same_labels(labels_np(ix), oracle64["final"], "batches of 100k, persistent, CUDA graph")
    ix.close()


def test_social_queries_every_form(social, oracle64):
    """All 10M queries after the insertions, host-driven and persistent
    search, against Algorithm 2 on the oracle: answers and deciding rules."""
    w = social
    E = int(w["ins_src"].shape[0])
    for persistent in (False, True):
        ix = dbl.DBLIndex(w["d"]["row_ptr"], w["d"]["col"], 64, 64, edge_capacity=E,
                          flags=(dbl.FLAG_PERSISTENT | dbl.FLAG_ASYNC) if persistent else 0)
        insert_batches(ix, w, [100_000] * (E // 100_000))
        ans, code = ix.query(w["d"]["q_u"], w["d"]["q_v"])
        ix.sync()
        assert_same_answers(ans, code, oracle64["ans"], oracle64["code"], f"queries, persistent={persistent}")
        ix.close()


def test_social_learned_headline_step(social):
    """The benchmark's headline configuration: learned landmarks (scorer
    trained on the GPU), persistent kernels, the whole step (restore, ten
    100k insertion batches, 10M queries) captured once as a CUDA graph and
    replayed.  The oracle is built with the same landmark and leaf sets."""
    w = social
    E = int(w["ins_src"].shape[0])
    d = w["d"]
    batches = [(a, a + 100_000) for a in range(0, E, 100_000)]
    plain = dbl.DBLIndex(d["row_ptr"], d["col"], 64, 64, edge_capacity=E)
    for a, b in batches:
        plain.insert_edges(d["ins_src"][a:b], d["ins_dst"][a:b])
    tu, tv = dbl_inputs.queries(w["row_ptr"], w["col"], 200_000, w["seed"] + 300, False, w["ins_src"], w["ins_dst"])
    scores, _ = L.train_scorer(plain, D(tu), D(tv), 8, steps=100)
    lm = L.select_landmarks(plain, scores, 64, 8)
    _, lb, lr = plain.selection()
    plain.close()
    ix = dbl.DBLIndex(d["row_ptr"], d["col"], 64, 64, landmarks=lm, leaf_buckets=lb, leaf_roles=lr,
                      edge_capacity=E, flags=dbl.FLAG_PERSISTENT | dbl.FLAG_ASYNC)
    ix.sync()
    ix.snapshot(0)
    Q = int(w["q_u"].shape[0])
    ans = torch.empty(Q, dtype=torch.uint8, device="cuda")
    code = torch.empty(Q, dtype=torch.uint8, device="cuda")

    def step():
        ix.restore(0)
        for a, b in batches:
            ix.insert_edges(d["ins_src"][a:b], d["ins_dst"][a:b])
        ix.query(d["q_u"], d["q_v"], out=(ans, code))

    step()
    torch.cuda.synchronize()
    ix.sync()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    ans.zero_()
    code.zero_()
    g.replay()
    torch.cuda.synchronize()
    ix.sync()

    lm_np, lb_np, lr_np = (t.cpu().numpy() for t in ix.selection())
    ref = oracle.OracleIndex(w["row_ptr"], w["col"], 64, 64).build(landmarks=lm_np, leaf_bucket=lb_np,
                                                                    leaf_role=lr_np, nthreads=THREADS)
    ref.insert_edges(w["ins_src"], w["ins_dst"])
    assert_same_labels(labels_np(ix), ref.labels(), "learned landmarks, graph replay")
    rans, rcode = ref.query(w["q_u"], w["q_v"], nthreads=THREADS)
    assert_same_answers(ans, code, rans, rcode, "learned landmarks, graph replay")
    ix.close()


def test_batched_config_uneven_batches(social):
    """k = 128 (two words per direction): insertion batches of log-uniform
    size in [1, 200k] and query batches of log-uniform size in [1k, 4M],
    through persistent kernels; every label word and every answer against the
    oracle (k = 128)."""
    w = social
    E, Q = int(w["ins_src"].shape[0]), int(w["q_u"].shape[0])
    d = w["d"]
    ins_sizes = dbl_inputs.loguniform_batches(E, 1, 200_000, 11)
    q_sizes = dbl_inputs.loguniform_batches(Q, 1000, 4_000_000, 12)
    ix = dbl.DBLIndex(d["row_ptr"], d["col"], 128, 64, edge_capacity=E,
                      flags=dbl.FLAG_PERSISTENT | dbl.FLAG_ASYNC)
    insert_batches(ix, w, [int(x) for x in ins_sizes])
    ans = torch.empty(Q, dtype=torch.uint8, device="cuda")
    code = torch.empty(Q, dtype=torch.uint8, device="cuda")
    a = 0
    for b in q_sizes:
        b = int(b)
        ix.query(d["q_u"][a:a + b], d["q_v"][a:a + b], out=(ans[a:a + b], code[a:a + b]))
        a += b
    assert a == Q
    ix.sync()
    ref = oracle.OracleIndex(w["row_ptr"], w["col"], 128, 64).build(nthreads=THREADS)
    ref.insert_edges(w["ins_src"], w["ins_dst"])
    assert_same_labels(labels_np(ix), ref.labels(), "k=128, uneven batches")
    rans, rcode = ref.query(w["q_u"], w["q_v"], nthreads=THREADS)
    assert_same_answers(ans, code, rans, rcode, "k=128, uneven query batches")
    ix.close()


def _merged_csr(rp, col, src, dst, n):
    """CSR of the base graph plus the inserted edges, on the device (rows sorted)."""
    deg = torch.diff(rp.long())
    s_all = torch.cat([torch.repeat_interleave(torch.arange(n, device=rp.device), deg), src.long()])
    d_all = torch.cat([col.long(), dst.long()])
    order = torch.argsort(s_all * n + d_all)
    s_all, d_all = s_all[order], d_all[order]
    rp2 = torch.zeros(n + 1, dtype=torch.int64, device=rp.device)
    rp2[1:] = torch.cumsum(torch.bincount(s_all, minlength=n), 0)
    return rp2.to(torch.int32), d_all.to(torch.int32)


def test_large_graph_incremental_equals_rebuild():
    """n = 2^24, m = 2^28 (the learned and serving workloads), k = 128,
    k' = 64: properties that hold at any size, checked without the oracle.
    (1) Labels after 1M insertions in batches of 100k through the persistent
    kernels equal the labels built from scratch on the final graph with the
    same landmark and leaf sets (the least fixpoint is unique).  (2) Every
    query whose v is the end of a forward walk from u (reachable by
    construction) is answered true, and the searches agree with the labels'
    verdicts on the rest (both indices answer identically)."""
    dbl.build()
    dbl_inputs.build()
    w = dbl_inputs.workload("large")
    n = int(w["n"])
    rp, col = D(w["row_ptr"]), D(w["col"])
    src, dst = D(w["ins_src"]), D(w["ins_dst"])
    E = int(src.numel())
    inc = dbl.DBLIndex(rp, col, 128, 64, edge_capacity=E, flags=dbl.FLAG_PERSISTENT | dbl.FLAG_ASYNC)
    for a in range(0, E, 100_000):
        inc.insert_edges(src[a:a + 100_000], dst[a:a + 100_000])
    inc.sync()
    lm, lb, lr = inc.selection()
    rp2, col2 = _merged_csr(rp, col, src, dst, n)
    del rp, col
    torch.cuda.empty_cache()
    full = dbl.DBLIndex(rp2, col2, 128, 64, landmarks=lm, leaf_buckets=lb, leaf_roles=lr)
    for a, b, name in zip(inc.labels(), full.labels(), ("dl_in", "dl_out", "bl_in", "bl_out")):
        assert torch.equal(a, b), f"large graph: {name} differs between incremental repair and rebuild"
    qu, qv = D(w["q_u"]), D(w["q_v"])
    a1, c1 = inc.query(qu, qv)
    inc.sync()
    a2, c2 = full.query(qu, qv)
    assert torch.equal(a1, a2) and torch.equal(c1, c2)
    assert bool((a1[1::2] == 1).all()), "a walk descendant was answered unreachable"
    inc.close()
    full.close()


def _large_learned(w, k, kp, E, train_pairs=200_000, steps=200):
    """The learned landmark slots of the large workload as the benchmark
    chooses them (plain degree index after the insertions, scorer trained on
    sampled query outcomes, k/8 degree landmarks kept), and the leaves."""
    rp, col = D(w["row_ptr"]), D(w["col"])
    src, dst = D(w["ins_src"]), D(w["ins_dst"])
    plain = dbl.DBLIndex(rp, col, k, kp, edge_capacity=E, flags=dbl.FLAG_PERSISTENT | dbl.FLAG_ASYNC)
    for a in range(0, E, 100_000):
        plain.insert_edges(src[a:a + 100_000], dst[a:a + 100_000])
    tu, tv = dbl_inputs.queries(w["row_ptr"], w["col"], train_pairs, int(w["seed"]) + 300, False,
                                w["ins_src"], w["ins_dst"])
    base = max(1, k // 8)
    scores, _ = L.train_scorer(plain, D(tu), D(tv), base, steps=steps)
    lm = L.select_landmarks(plain, scores, k, base)
    _, lb, lr = plain.selection()
    plain.close()
    return lm, lb, lr


@pytest.mark.parametrize("k,kp,grouped", [(64, 64, True), (128, 64, False)])
def test_large_graph_matches_oracle(k, kp, grouped):
    """n = 2^24, m = 2^28 with learned landmarks, in the benchmark's launch
    configurations: k = k' = 64 with the 1M insertions queued in batches of
    100k and applied as one group by the query call (the headline form), and
    k = 128, k' = 64 with one persistent launch per batch (the serving
    index).  Every label word against the oracle built with the same landmark
    and leaf sets (Algorithm 1, then Algorithm 3 and its mirrors edge by edge),
    and the answers and deciding rules of 1M of the 10M queries against
    Algorithm 2 on the oracle."""
    dbl.build()
    dbl_inputs.build()
    oracle.build()
    w = dbl_inputs.workload("large")
    E = int(w["ins_src"].shape[0])
    lm, lb, lr = _large_learned(w, k, kp, E)
    flags = dbl.FLAG_PERSISTENT | dbl.FLAG_ASYNC | (dbl.FLAG_DEFER if grouped else 0)
    ix = dbl.DBLIndex(D(w["row_ptr"]), D(w["col"]), k, kp, landmarks=lm, leaf_buckets=lb, leaf_roles=lr,
                      edge_capacity=E, flags=flags)
    src, dst = D(w["ins_src"]), D(w["ins_dst"])
    for a in range(0, E, 100_000):
        ix.insert_edges(src[a:a + 100_000], dst[a:a + 100_000])
    S = 1_000_000
    qu, qv = w["q_u"][-S:], w["q_v"][-S:]
    ans, code = ix.query(D(qu), D(qv))
    ix.sync()
    got = labels_np(ix)
    ans, code = ans.cpu().numpy(), code.cpu().numpy()
    ix.close()
    ref = oracle.OracleIndex(w["row_ptr"], w["col"], k, kp).build(
        landmarks=lm.cpu().numpy(), leaf_bucket=lb.cpu().numpy(), leaf_role=lr.cpu().numpy(), nthreads=THREADS)
    ref.insert_edges(w["ins_src"], w["ins_dst"])
    what = f"large graph, learned landmarks, k={k} k'={kp}, {'grouped' if grouped else 'per batch'}"
    assert_same_labels(got, ref.labels(), what)
    rans, rcode = ref.query(qu, qv, nthreads=THREADS)
    bad = np.nonzero((ans != rans) | (code != rcode))[0]
    assert bad.size == 0, f"{what}: {bad.size} of {S} queries differ, first {bad[:5]}"
