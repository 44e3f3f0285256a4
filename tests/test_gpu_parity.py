"""GPU path vs the CPU oracle, element by element, through the C ABI.

Integer work throughout: every label word, every answer and every deciding
rule must match bit for bit.
"""
import numpy as np
import pytest
import torch

import dbl_inputs
import oracle
import paper_2101_09441_gb300 as dbl
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    dbl.build()
    dbl_inputs.build()
    oracle.build()


def D(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def labels_np(ix):
    return [t.cpu().numpy().view(np.uint64) for t in ix.labels()]


def assert_labels(ix, ref, what=""):
    for a, b, name in zip(labels_np(ix), ref.labels(), ("dl_in", "dl_out", "bl_in", "bl_out")):
        if not np.array_equal(a, b):
            bad = np.nonzero((a != b).any(axis=1))[0]
            raise AssertionError(f"{what}: {name} differs at {bad.size} vertices, first {bad[:8]}")


def assert_queries(ix, ref, qu, qv, what=""):
    ans, code = ix.query(D(qu), D(qv))
    rans, rcode = ref.query(qu, qv, nthreads=8)
    a, c = ans.cpu().numpy(), code.cpu().numpy()
    bad = np.nonzero((a != rans) | (c != rcode))[0]
    assert bad.size == 0, f"{what}: {bad.size} queries differ, e.g. {[(int(qu[i]), int(qv[i]), int(a[i]), int(c[i]), int(rans[i]), int(rcode[i])) for i in bad[:5]]}"
    return rans, rcode


# ---------------------------------------------------------------- worked example
def test_running_example():
    ex = H.load_running_example()
    rp, col, lm, bucket, role = H.running_example_inputs(ex, 64, 64)
    ix = dbl.DBLIndex(D(rp), D(col), 64, 64, landmarks=D(lm), leaf_buckets=D(bucket), leaf_roles=D(role))
    ref = oracle.OracleIndex(rp, col, 64, 64).build(lm, bucket, role)
    assert_labels(ix, ref, "build")
    dl_in, dl_out, bl_in, bl_out = labels_np(ix)
    for v, (e_in, e_out) in ex["dl"].items():
        assert H.set_bits(dl_in[v]) == {ex["landmarks"].index(x) for x in e_in}
        assert H.set_bits(dl_out[v]) == {ex["landmarks"].index(x) for x in e_out}
    for v, (e_in, e_out) in ex["bl"].items():
        assert H.set_bits(bl_in[v]) == e_in and H.set_bits(bl_out[v]) == e_out
    u = np.array([q[0] for q in ex["queries"]], np.int32)
    v = np.array([q[1] for q in ex["queries"]], np.int32)
    ans, code = ix.query(D(u), D(v))
    assert list(ans.cpu().numpy()) == [q[2] for q in ex["queries"]]
    assert list(code.cpu().numpy()) == [H.CODES[q[3]] for q in ex["queries"]]
    s, d = zip(*ex["inserts"])
    ix.insert_edges(D(np.array(s, np.int32)), D(np.array(d, np.int32)))
    ref.insert_edges(s, d)
    assert_labels(ix, ref, "after (v9, v2)")
    dl_in = labels_np(ix)[0]
    for x, e in ex["dl_in_after"].items():
        assert H.set_bits(dl_in[x]) == {ex["landmarks"].index(y) for y in e}


# ---------------------------------------------------------------- tiny config
@pytest.fixture(scope="module")
def tiny():
    return dbl_inputs.workload("tiny")


def test_tiny_selection_matches_oracle(tiny):
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64)
    lm, lb, lr = [t.cpu().numpy() for t in ix.selection()]
    assert np.array_equal(lm, ref.degree_landmarks())
    rb, rr = ref.zero_degree_leaves()
    assert np.array_equal(lb, rb) and np.array_equal(lr, rr)


@pytest.mark.parametrize("rule,r", [("M", 2), ("A", 0), ("B", 8), ("C", 1000)])
@pytest.mark.parametrize("flags", [0, dbl.FLAG_PERSISTENT])
def test_selection_rules_match_oracle(tiny, rule, r, flags):
    """Section 6 (Label Node Selection): Table 3's landmark rankings and the
    M(u) <= r leaf rule chosen on the GPU equal the oracle's choice; labels
    after the 10k insertions and every answer follow the oracle with them."""
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64, landmark_rule=rule, leaf_r=r, flags=flags)
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64)
    lm, lb, lr = [t.cpu().numpy() for t in ix.selection()]
    assert np.array_equal(lm, ref.rank_landmarks(rule))
    rb, rr = ref.threshold_leaves(r)
    assert np.array_equal(lb, rb) and np.array_equal(lr, rr)
    if r > 0:
        assert (rr == 3).any()                            # the threshold adds two-sided leaves
    ref.build(lm, lb, lr)
    assert_labels(ix, ref, f"build, rule {rule}, r {r}")
    s, d = tiny["ins_src"], tiny["ins_dst"]
    for b in range(0, s.shape[0], 2500):
        ix.insert_edges(D(s[b:b + 2500]), D(d[b:b + 2500]))
    ref.insert_edges(s, d)
    ix.sync()
    assert_labels(ix, ref, f"insertions, rule {rule}, r {r}")
    assert_queries(ix, ref, tiny["q_u"], tiny["q_v"], f"queries, rule {rule}, r {r}")


@pytest.mark.parametrize("flags", [0, dbl.FLAG_PERSISTENT | dbl.FLAG_ASYNC])
def test_vertex_insertion_matches_oracle(tiny, flags):
    """Vertex insertion (Section 1): isolated new vertices with empty labels,
    then edges touching them; every label word and every answer against the
    oracle doing the same; capacity errors leave the index unchanged; a
    restore returns to the snapshot's vertices and re-added rows are clean."""
    n0, add = int(tiny["n"]), 3000
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64, vertex_capacity=n0 + add + 100, flags=flags)
    assert ix.info()["vertex_capacity"] == n0 + add + 100
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build()
    ix.sync()
    ix.snapshot(0)
    assert ix.add_vertices(add) == n0 and ix.n == n0 + add
    ref.add_vertices(add)
    assert_labels(ix, ref, "after adding vertices")
    rng = np.random.default_rng(17)
    n = n0 + add
    new_src = rng.integers(n0, n, 4000).astype(np.int32)          # edges out of, into and between new vertices
    new_dst = rng.integers(0, n, 4000).astype(np.int32)
    into_src = rng.integers(0, n0, 4000).astype(np.int32)
    into_dst = rng.integers(n0, n, 4000).astype(np.int32)
    es = np.concatenate([tiny["ins_src"], new_src, into_src])
    ed = np.concatenate([tiny["ins_dst"], new_dst, into_dst])
    perm = rng.permutation(es.shape[0])
    es, ed = es[perm], ed[perm]
    for b in range(0, es.shape[0], 1500):
        ix.insert_edges(D(es[b:b + 1500]), D(ed[b:b + 1500]))
    ref.insert_edges(es, ed)
    ix.sync()
    assert_labels(ix, ref, "after insertions touching new vertices")
    qu = np.concatenate([tiny["q_u"][:50_000], rng.integers(0, n, 50_000).astype(np.int32)])
    qv = np.concatenate([tiny["q_v"][:50_000], rng.integers(n0, n, 25_000).astype(np.int32),
                         rng.integers(0, n, 25_000).astype(np.int32)])
    assert_queries(ix, ref, qu, qv, "queries with new vertices")
    with pytest.raises(dbl.DblError):
        ix.add_vertices(101)                                      # capacity n0 + add + 100
    assert ix.n == n
    ix.restore(0)
    assert ix.n == n0
    fresh = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build()
    assert_labels(ix, fresh, "restored")
    assert ix.add_vertices(5) == n0
    assert all((t[n0:].cpu() == 0).all() for t in ix.labels())    # rows of the removed vertices are cleared
    ix.close()


def test_tiny_full_pipeline(tiny):
    """Plain DBL, tiny: build, 10k insertions in batches of 1k (labels after
    every batch), then 100k mixed queries (answers and deciding rules)."""
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build()
    assert_labels(ix, ref, "build")
    s, d = tiny["ins_src"], tiny["ins_dst"]
    for b in range(0, s.shape[0], 1000):
        ix.insert_edges(D(s[b:b + 1000]), D(d[b:b + 1000]))
        ref.insert_edges(s[b:b + 1000], d[b:b + 1000])
        assert_labels(ix, ref, f"after batch {b // 1000}")
    rans, rcode = assert_queries(ix, ref, tiny["q_u"], tiny["q_v"], "tiny queries")
    assert (rcode == oracle.BFS_POS).sum() > 100          # the search really runs
    st = ix.stats()
    assert st[oracle.BFS_POS] == (rcode == oracle.BFS_POS).sum()
    assert st[11] + st[12] == s.shape[0]                  # applied + skipped


# ---------------------------------------------------------------- label widths
@pytest.mark.parametrize("k,kprime", [(64, 64), (128, 64), (64, 128), (128, 128), (256, 64), (64, 256),
                                      (256, 256), (128, 256), (256, 128), (16, 16), (32, 32), (16, 32),
                                      (32, 16), (16, 64), (64, 16), (32, 256), (256, 32)])
def test_widths_random_selection(k, kprime):
    rp, col = dbl_inputs.rmat_csr(3000, 12_000, 31 + k + kprime)
    n = 3000
    lm = H.random_slots(n, k, k - 5, k * 7 + kprime)
    bucket, role = H.random_leaves(n, kprime, 0.25, kprime)
    ix = dbl.DBLIndex(D(rp), D(col), k, kprime, landmarks=D(lm), leaf_buckets=D(bucket), leaf_roles=D(role))
    ref = oracle.OracleIndex(rp, col, k, kprime).build(lm, bucket, role)
    assert_labels(ix, ref, f"k={k} k'={kprime} build")
    s, dd = dbl_inputs.insertions(rp, col, 500, 3)
    ix.insert_edges(D(s), D(dd))
    ref.insert_edges(s, dd)
    assert_labels(ix, ref, f"k={k} k'={kprime} insert")
    qu, qv = dbl_inputs.queries(rp, col, 20_000, 4, True, s, dd)
    assert_queries(ix, ref, qu, qv, f"k={k} k'={kprime}")


@pytest.mark.parametrize("team", [1, 4, 8, 16, 32])
def test_team_sizes(team, tiny):
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64, team=team)
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build()
    ix.insert_edges(D(tiny["ins_src"]), D(tiny["ins_dst"]))
    ref.insert_edges(tiny["ins_src"], tiny["ins_dst"])
    assert_labels(ix, ref, f"team {team}")
    assert_queries(ix, ref, tiny["q_u"][:20000], tiny["q_v"][:20000], f"team {team}")


# ---------------------------------------------------------------- closure shapes
@pytest.mark.parametrize("shape", ["path", "cycle", "two_cycles", "star_in", "star_out", "dense"])
def test_shapes_match_closure(shape):
    if shape == "path":
        n = 300
        s, d = H.path_graph(n)
    elif shape == "cycle":
        n = 257
        s, d = H.path_graph(n, cycle=True)
    elif shape == "two_cycles":
        n = 200
        s1, d1 = H.path_graph(100, cycle=True)
        s, d = np.concatenate([s1, s1 + 100, [5]]), np.concatenate([d1, d1 + 100, [150]])
    elif shape == "star_in":
        n = 5000
        s, d = np.arange(1, n, dtype=np.int32), np.zeros(n - 1, np.int32)
    elif shape == "star_out":
        n = 5000
        s, d = np.zeros(n - 1, np.int32), np.arange(1, n, dtype=np.int32)
    else:
        n = 200
        s, d = H.random_graph(n, 6000, 77)
    rp, col = H.csr_from_edges(n, s, d)
    ix = dbl.DBLIndex(D(rp), D(col), 64, 64)
    ref = oracle.OracleIndex(rp, col, 64, 64).build()
    assert_labels(ix, ref, shape)
    rng = np.random.default_rng(1)
    qu = rng.integers(0, n, 20000).astype(np.int32)
    qv = rng.integers(0, n, 20000).astype(np.int32)
    rans, _ = assert_queries(ix, ref, qu, qv, shape)
    if n <= 400:
        R = H.closure(n, s, d)
        assert np.array_equal(rans.astype(bool), R[qu, qv])


# ---------------------------------------------------------------- edge cases
def test_empty_and_single_vertex():
    for n in (1, 7):
        rp = np.zeros(n + 1, np.int32)
        ix = dbl.DBLIndex(D(rp), D(np.zeros(0, np.int32)), 64, 64)
        ref = oracle.OracleIndex(rp, np.zeros(0, np.int32), 64, 64).build()
        assert_labels(ix, ref, f"empty n={n}")
        qu = np.arange(n, dtype=np.int32)
        qv = np.roll(qu, 1)
        assert_queries(ix, ref, qu, qv, "empty")
        ix.insert_edges(D(np.zeros(0, np.int32)), D(np.zeros(0, np.int32)))  # b = 0
        a, c = ix.query(D(np.zeros(0, np.int32)), D(np.zeros(0, np.int32)))  # q = 0
        assert a.numel() == 0


def test_self_loops_and_duplicates():
    rp, col = dbl_inputs.rmat_csr(2000, 8000, 9)
    src, dst = H.edges_from_csr(rp, col)
    # a CSR with self-loops and duplicate edges is accepted; labels as without them
    s2 = np.concatenate([src, [3, 3, 10], src[:50]])
    d2 = np.concatenate([dst, [3, 3, 10], dst[:50]])
    rp2, col2 = H.csr_from_edges(2000, s2, d2)
    ref = oracle.OracleIndex(rp, col, 64, 64).build()
    ix = dbl.DBLIndex(D(rp2), D(col2), 64, 64, landmarks=D(ref.landmarks), leaf_buckets=D(ref.leaf_bucket),
                      leaf_roles=D(ref.leaf_role))
    assert_labels(ix, ref, "self-loops/duplicates")
    ix.insert_edges(D(np.array([5, 5, 7], np.int32)), D(np.array([5, 9, 9], np.int32)))
    ref.insert_edges([5, 5, 7], [5, 9, 9])
    assert_labels(ix, ref, "inserted self-loop")
    assert ix.stats()[13] == 1


def test_invalid_ids_leave_index_unchanged(tiny):
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    before = labels_np(ix)
    n = tiny["n"]
    with pytest.raises(dbl.DblError) as e:
        ix.insert_edges(D(np.array([1, 2], np.int32)), D(np.array([3, n], np.int32)))
    assert e.value.status == dbl.DBL_ERR_INVALID
    with pytest.raises(dbl.DblError):
        ix.insert_edges(D(np.array([-1], np.int32)), D(np.array([3], np.int32)))
    for a, b in zip(before, labels_np(ix)):
        assert np.array_equal(a, b)
    assert ix.info()["edges_stored"] == 0
    with pytest.raises(dbl.DblError) as e:
        ix.query(D(np.array([0], np.int32)), D(np.array([n], np.int32)))
    assert e.value.status == dbl.DBL_ERR_INVALID
    # still usable
    ix.insert_edges(D(np.array([1], np.int32)), D(np.array([2], np.int32)))


def test_invalid_build_inputs():
    rp = np.array([0, 2, 1], np.int32)  # decreasing
    with pytest.raises(dbl.DblError):
        dbl.DBLIndex(D(rp), D(np.array([1, 0], np.int32)), 64, 64)
    with pytest.raises(dbl.DblError):
        dbl.DBLIndex(D(np.array([0, 1], np.int32)), D(np.array([5], np.int32)), 64, 64)
    with pytest.raises(dbl.DblError):
        dbl.DBLIndex(D(np.array([0, 0], np.int32)), D(np.zeros(0, np.int32)), 96, 64)
    with pytest.raises(dbl.DblError):
        dbl.DBLIndex(D(np.array([0, 0, 0], np.int32)), D(np.zeros(0, np.int32)), 64, 64,
                     landmarks=D(np.full(64, 2, np.int32)))


def test_capacity_exhaustion(tiny):
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64, edge_capacity=1500)
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build()
    s, d = tiny["ins_src"], tiny["ins_dst"]
    ix.insert_edges(D(s[:1000]), D(d[:1000]))
    ref.insert_edges(s[:1000], d[:1000])
    with pytest.raises(dbl.DblError) as e:
        ix.insert_edges(D(s[1000:1600]), D(d[1000:1600]))
    assert e.value.status == dbl.DBL_ERR_CAPACITY
    assert_labels(ix, ref, "after refused batch")
    ix.insert_edges(D(s[1000:1500]), D(d[1000:1500]))
    ref.insert_edges(s[1000:1500], d[1000:1500])
    assert_labels(ix, ref, "after filling capacity")


def test_snapshot_restore(tiny):
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build()
    base = labels_np(ix)
    ix.snapshot(0)
    s, d = tiny["ins_src"], tiny["ins_dst"]
    ix.insert_edges(D(s), D(d))
    ix.restore(0)
    for a, b in zip(base, labels_np(ix)):
        assert np.array_equal(a, b)
    # the restored index behaves like the original: same insertions, same result
    ix.insert_edges(D(s[:4000]), D(d[:4000]))
    ref.insert_edges(s[:4000], d[:4000])
    assert_labels(ix, ref, "after restore + insert")
    assert_queries(ix, ref, tiny["q_u"][:30000], tiny["q_v"][:30000], "after restore")


@pytest.mark.parametrize("flags", [0, dbl.FLAG_PERSISTENT, dbl.FLAG_PERSISTENT | dbl.FLAG_ASYNC])
def test_restore_of_changed_vertices_only(tiny, flags):
    """A restore to the snapshot the index last equalled copies back only the
    vertices whose record or adjacency changed since; a restore to another
    slot copies everything.  The choice is made on the device, so a captured
    restore stays right when later snapshots change which slot the index last
    equalled.  A restore drops the snapshots taken after it.  Every case ends
    in the oracle's labels and answers."""
    rp, col = tiny["row_ptr"], tiny["col"]
    s, d = tiny["ins_src"], tiny["ins_dst"]
    A, B = (s[:5000], d[:5000]), (s[5000:], d[5000:])
    qu, qv = tiny["q_u"][:20000], tiny["q_v"][:20000]
    ix = dbl.DBLIndex(D(rp), D(col), 64, 64, flags=flags, edge_capacity=1 << 16, vertex_capacity=len(rp) + 63)
    refA = oracle.OracleIndex(rp, col, 64, 64).build()
    refA.insert_edges(*A)
    refAB = oracle.OracleIndex(rp, col, 64, 64).build()
    refAB.insert_edges(s, d)
    ix.sync()
    L0 = labels_np(ix)
    ix.snapshot(0)

    def same(want, what):
        ix.sync()
        for a, b in zip(labels_np(ix), want):
            assert np.array_equal(a, b), what

    ix.insert_edges(D(A[0]), D(A[1]))
    ix.restore(0)                              # changed vertices only
    same(L0, "restore of the changes")
    ix.insert_edges(D(A[0]), D(A[1]))
    ix.sync()
    assert_labels(ix, refA, "A after restore")
    ix.snapshot(1)                             # the index now equals slot 1
    ix.insert_edges(D(B[0]), D(B[1]))
    ix.restore(1)                              # changed vertices only
    ix.sync()
    assert_labels(ix, refA, "restore to slot 1")
    assert_queries(ix, refA, qu, qv, "after restore to slot 1")
    ix.restore(0)                              # another slot: everything; slot 1 is dropped
    same(L0, "full restore")
    with pytest.raises(dbl.DblError) as e:
        ix.restore(1)
    assert e.value.status == dbl.DBL_ERR_INVALID
    ix.insert_edges(D(s), D(d))
    ix.sync()
    assert_labels(ix, refAB, "A+B after full restore")
    assert_queries(ix, refAB, qu, qv, "A+B after full restore")
    ix.restore(0)
    ix.restore(0)                              # nothing changed in between
    same(L0, "restore with nothing changed")
    # vertices added after the snapshot go away; their rows return cleared
    first = ix.add_vertices(3)
    ix.insert_edges(D(np.array([first, first + 1], np.int32)), D(np.array([int(s[0]), first + 2], np.int32)))
    ix.restore(0)
    ix.sync()
    assert ix.n == first
    same(L0, "restore after vertex insertion")
    ix.insert_edges(D(A[0]), D(A[1]))
    ix.sync()
    assert_labels(ix, refA, "A after the vertex round trip")
    assert_queries(ix, refA, qu, qv, "A after the vertex round trip")
    if flags & dbl.FLAG_ASYNC:
        # a captured restore + insertion, replayed after a snapshot to another slot
        ix.restore(0)
        ix.sync()
        g = torch.cuda.CUDAGraph()
        dA0, dA1 = D(A[0]), D(A[1])
        with torch.cuda.graph(g):
            ix.restore(0)
            ix.insert_edges(dA0, dA1)
        for _ in range(2):
            g.replay()
            torch.cuda.synchronize()
            assert_labels(ix, refA, "captured restore + insert")
        ix.snapshot(2)                         # the index now equals slot 2
        g.replay()                             # the captured restore(0) must copy everything
        torch.cuda.synchronize()
        assert_labels(ix, refA, "captured restore after another snapshot")
        assert_queries(ix, refA, qu, qv, "captured restore after another snapshot")
    ix.close()


@pytest.mark.parametrize("slots", [-1, 2, 4, 64])
@pytest.mark.parametrize("flags", [0, dbl.FLAG_PERSISTENT, dbl.FLAG_PERSISTENT | dbl.FLAG_ASYNC])
def test_reserved_slots_and_segment_growth(tiny, slots, flags):
    """Inserted-edge slots reserved per vertex at build (dbl_options
    initial_slots): batches whose endpoints all have room take the
    one-phase append of the persistent insertion, a batch in which a hub
    gains 300 out-edges and 300 in-edges grows segments; with no reserved
    slots every first insertion grows one.  Labels and answers equal the
    oracle's after every batch."""
    rp, col = tiny["row_ptr"], tiny["col"]
    n = len(rp) - 1
    s, d = tiny["ins_src"], tiny["ins_dst"]
    hub = int(np.argmax(np.diff(rp)))
    have = set(col[rp[hub]:rp[hub + 1]].tolist())
    outs = np.array([t for t in range(n) if t != hub and t not in have][:300], np.int32)
    ins_from = np.array([t for t in range(n - 1, -1, -1) if t != hub and hub not in
                         set(col[rp[t]:rp[t + 1]].tolist())][:300], np.int32)
    batches = [(s[:2000], d[:2000]),
               (np.concatenate([np.full(300, hub, np.int32), ins_from, s[2000:3000]]),
                np.concatenate([outs, np.full(300, hub, np.int32), d[2000:3000]])),
               (s[3000:], d[3000:])]
    ix = dbl.DBLIndex(D(rp), D(col), 64, 64, flags=flags, initial_slots=slots, edge_capacity=1 << 16)
    ref = oracle.OracleIndex(rp, col, 64, 64).build()
    for k, (bs, bd) in enumerate(batches):
        ix.insert_edges(D(bs), D(bd))
        ref.insert_edges(bs, bd)
        ix.sync()
        assert_labels(ix, ref, f"slots={slots}, batch {k}")
    assert_queries(ix, ref, tiny["q_u"][:20000], tiny["q_v"][:20000], f"slots={slots}")
    ix.close()


@pytest.mark.parametrize("k,kp", [(64, 64), (128, 64), (256, 256)])
@pytest.mark.parametrize("flags", [0, dbl.FLAG_PERSISTENT])
def test_split_build_equals_joint_build(tiny, k, kp, flags):
    """The label build over each direction's halves in turn (dbl_options
    build_split = 1) gives the same least fixpoint as the joint build, and
    both equal the oracle's labels (Algorithm 1)."""
    rp, col = tiny["row_ptr"], tiny["col"]
    a = dbl.DBLIndex(D(rp), D(col), k, kp, flags=flags, build_split=1)
    b = dbl.DBLIndex(D(rp), D(col), k, kp, flags=flags, build_split=-1)
    ref = oracle.OracleIndex(rp, col, k, kp).build()
    assert_labels(a, ref, f"split build k={k} k'={kp}")
    assert_labels(b, ref, f"joint build k={k} k'={kp}")
    a.insert_edges(D(tiny["ins_src"]), D(tiny["ins_dst"]))
    ref.insert_edges(tiny["ins_src"], tiny["ins_dst"])
    a.sync()
    assert_labels(a, ref, "split build, after insertions")


def _with_hubs(rp, col, n_hubs=3, seed=9):
    """The graph plus n_hubs vertices joined to thousands of others in both
    directions (rows above the ordering's block-per-row threshold of 1024)."""
    n = rp.shape[0] - 1
    rng = np.random.default_rng(seed)
    src = np.repeat(np.arange(n), np.diff(rp)).astype(np.int64)
    dst = col.astype(np.int64)
    extra_s, extra_d = [src], [dst]
    for h in rng.choice(n, n_hubs, replace=False):
        outs = rng.choice(n, 3000, replace=False)
        ins = rng.choice(n, 2000, replace=False)
        extra_s += [np.full(3000, h), ins]
        extra_d += [outs, np.full(2000, h)]
    s_all, d_all = np.concatenate(extra_s), np.concatenate(extra_d)
    keep = s_all != d_all
    key = np.unique(s_all[keep] * n + d_all[keep])
    s_all, d_all = key // n, key % n
    rp2 = np.zeros(n + 1, np.int64)
    np.add.at(rp2, s_all + 1, 1)
    return np.cumsum(rp2).astype(np.int32), d_all.astype(np.int32)


@pytest.mark.parametrize("k,kp", [(16, 16), (64, 64), (128, 64)])
@pytest.mark.parametrize("split", [1, -1])
@pytest.mark.parametrize("flags", [0, dbl.FLAG_PERSISTENT])
def test_degree_ordered_build_equals_oracle(tiny, k, kp, split, flags):
    """The build over the degree-grouped renumbering of the graph
    (dbl_options build_order = 1) stores the same least fixpoint (Algorithm 1)
    as the oracle, with hub rows above and below the block-per-row threshold;
    insertions and queries afterwards run on the index's own numbering."""
    rp, col = _with_hubs(tiny["row_ptr"], tiny["col"])
    ix = dbl.DBLIndex(D(rp), D(col), k, kp, flags=flags, build_split=split, build_order=1,
                      vertex_capacity=rp.shape[0] + 100)
    ref = oracle.OracleIndex(rp, col, k, kp).build()
    assert_labels(ix, ref, f"ordered build k={k} k'={kp} split={split}")
    ix.insert_edges(D(tiny["ins_src"]), D(tiny["ins_dst"]))
    ref.insert_edges(tiny["ins_src"], tiny["ins_dst"])
    ix.sync()
    assert_labels(ix, ref, "ordered build, after insertions")
    assert_queries(ix, ref, tiny["q_u"][:20000], tiny["q_v"][:20000], "ordered build, queries")


@pytest.mark.parametrize("n,m", [(1, 0), (5, 0), (1500, 0), (3000, 9000)])
def test_degree_ordered_build_small_and_edgeless(n, m):
    """Degenerate graphs under the ordered build: one vertex, no edges, one
    ordering tile with a ragged tail."""
    rng = np.random.default_rng(n + m)
    if m:
        s = rng.integers(0, n, m)
        d = rng.integers(0, n, m)
        key = np.unique(s[s != d] * n + d[s != d])
        s, d = key // n, key % n
    else:
        s = d = np.zeros(0, np.int64)
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, s + 1, 1)
    rp, col = np.cumsum(rp).astype(np.int32), d.astype(np.int32)
    ix = dbl.DBLIndex(D(rp), D(col), 64, 64, build_order=1, build_split=1)
    ref = oracle.OracleIndex(rp, col, 64, 64).build()
    assert_labels(ix, ref, f"ordered build n={n} m={m}")


def test_deferred_insertions_apply_as_one_group(tiny):
    """DBL_FLAG_DEFER: insertion batches queue on the host and the next call
    that reads the index applies them in one launch.  A query sees exactly
    the batches queued before it; 40 small batches flush at 32; an invalid
    id in a queued batch rejects the whole group (nothing changes); a
    captured restore + queued batches + query replays correctly."""
    rp, col = tiny["row_ptr"], tiny["col"]
    s, d = tiny["ins_src"], tiny["ins_dst"]
    qu, qv = tiny["q_u"][:20000], tiny["q_v"][:20000]
    flags = dbl.FLAG_PERSISTENT | dbl.FLAG_ASYNC | dbl.FLAG_DEFER
    ix = dbl.DBLIndex(D(rp), D(col), 64, 64, flags=flags, edge_capacity=1 << 16)
    ix.snapshot(0)
    ref = oracle.OracleIndex(rp, col, 64, 64).build()
    dev_s, dev_d = D(s), D(d)
    for a in range(0, 3000, 1000):                      # three batches, then a query
        ix.insert_edges(dev_s[a:a + 1000], dev_d[a:a + 1000])
    ref.insert_edges(s[:3000], d[:3000])
    assert_queries(ix, ref, qu, qv, "after three queued batches")
    for a in range(3000, 7000, 100):                    # 40 batches: a flush at 32, the rest at labels()
        ix.insert_edges(dev_s[a:a + 100], dev_d[a:a + 100])
    ref.insert_edges(s[3000:7000], d[3000:7000])
    ix.sync()
    assert_labels(ix, ref, "after 40 queued batches")
    before = labels_np(ix)
    bad = D(np.array([0, len(rp) + 5], np.int32))      # an id out of range
    ix.insert_edges(dev_s[7000:8000], dev_d[7000:8000])
    ix.insert_edges(bad, bad)
    with pytest.raises(dbl.DblError) as e:
        ix.sync()
    assert e.value.status == dbl.DBL_ERR_INVALID
    for x, y in zip(labels_np(ix), before):
        assert np.array_equal(x, y)                     # the whole group was rejected
    # captured: restore, three queued batches, the query that applies them
    refB = oracle.OracleIndex(rp, col, 64, 64).build()
    refB.insert_edges(s[:6000], d[:6000])
    ix.restore(0)
    ix.sync()
    ans = torch.empty(len(qu), dtype=torch.uint8, device="cuda")
    code = torch.empty_like(ans)
    dqu, dqv = D(qu), D(qv)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ix.restore(0)
        for a in range(0, 6000, 2000):
            ix.insert_edges(dev_s[a:a + 2000], dev_d[a:a + 2000])
        ix.query(dqu, dqv, out=(ans, code))
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        rans, rcode = refB.query(qu, qv, nthreads=8)
        assert np.array_equal(ans.cpu().numpy(), rans) and np.array_equal(code.cpu().numpy(), rcode)
        assert_labels(ix, refB, "replayed deferred group")
    ix.close()


def test_batch_size_invariance(tiny):
    s, d = tiny["ins_src"], tiny["ins_dst"]
    results = []
    for bs in (1, 37, 1000, 10_000):
        ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
        lim = 400 if bs == 1 else 10_000
        for b in range(0, lim, bs):
            ix.insert_edges(D(s[b:min(b + bs, lim)]), D(d[b:min(b + bs, lim)]))
        results.append((lim, labels_np(ix)))
    full = [r for lim, r in results if lim == 10_000]
    for r in full[1:]:
        for a, b in zip(full[0], r):
            assert np.array_equal(a, b)
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build()
    ref.insert_edges(s[:400], d[:400])
    for a, b in zip(results[0][1], ref.labels()):
        assert np.array_equal(a, b)


def test_host_buffer_forms(tiny):
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    ix.insert_edges_host(tiny["ins_src"], tiny["ins_dst"])
    a1, c1 = ix.query(D(tiny["q_u"]), D(tiny["q_v"]))
    a2, c2 = ix.query_host(tiny["q_u"], tiny["q_v"], with_code=True)
    assert np.array_equal(a1.cpu().numpy(), a2) and np.array_equal(c1.cpu().numpy(), c2)


def test_host_buffer_forms_asynchronous(tiny):
    """With FLAG_ASYNC the host-buffer calls only queue their copies and
    kernels (pinned buffers, several insertion batches and query chunks in
    flight); with FLAG_DEFER the uploaded batches wait in the queue, holding
    their staging buffers (40 batches of 250 wrap the ring of 16 buffers and
    pass the group limit of 32); after a sync the answers equal the oracle's."""
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build()
    ref.insert_edges(tiny["ins_src"], tiny["ins_dst"])
    rans, rcode = ref.query(tiny["q_u"], tiny["q_v"], nthreads=8)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    src, dst, qu, qv = pin(tiny["ins_src"]), pin(tiny["ins_dst"]), pin(tiny["q_u"]), pin(tiny["q_v"])
    ans = torch.empty(qu.shape[0], dtype=torch.uint8).pin_memory().numpy()
    code = torch.empty(qu.shape[0], dtype=torch.uint8).pin_memory().numpy()
    for flags, bs in ((dbl.FLAG_ASYNC, 1000), (dbl.FLAG_ASYNC | dbl.FLAG_PERSISTENT, 1000),
                      (dbl.FLAG_ASYNC | dbl.FLAG_PERSISTENT | dbl.FLAG_DEFER, 1000),
                      (dbl.FLAG_ASYNC | dbl.FLAG_PERSISTENT | dbl.FLAG_DEFER, 250)):
        ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64, flags=flags)
        for a in range(0, src.shape[0], bs):
            ix.insert_edges_host(src[a:a + bs], dst[a:a + bs])
        ans[:] = 7
        ix.query_host(qu, qv, with_code=True, out=(ans, code))
        ix.sync()
        torch.cuda.synchronize()
        assert np.array_equal(ans, rans) and np.array_equal(code, rcode), f"flags {flags}, batches of {bs}"
        ix.close()


def test_torch_and_default_allocators_agree(tiny):
    a = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64, torch_allocator=False)
    b = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64, torch_allocator=True)
    for x, y in zip(labels_np(a), labels_np(b)):
        assert np.array_equal(x, y)
    a.close()
    b.close()


# ---------------------------------------------------------------- persistent / async forms
@pytest.mark.parametrize("flags", [dbl.FLAG_PERSISTENT, dbl.FLAG_PERSISTENT | dbl.FLAG_ASYNC])
@pytest.mark.parametrize("k", [64, 128])
@pytest.mark.parametrize("team", [1, 8])
def test_persistent_forms_match_oracle(tiny, flags, k, team):
    """One cooperative launch per propagation and per query batch; with
    FLAG_ASYNC no call waits for the device."""
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), k, 64, flags=flags, team=team)
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], k, 64).build()
    ix.sync()
    assert_labels(ix, ref, "persistent build")
    s, d = tiny["ins_src"], tiny["ins_dst"]
    sizes = [1, 7, 100, 1000, 2892, 6000]
    b = 0
    for sz in sizes:
        ix.insert_edges(D(s[b:b + sz]), D(d[b:b + sz]))
        ref.insert_edges(s[b:b + sz], d[b:b + sz])
        b += sz
        ix.sync()
        assert_labels(ix, ref, f"persistent after {b} edges")
    ans, code = ix.query(D(tiny["q_u"]), D(tiny["q_v"]))
    ix.sync()
    rans, rcode = ref.query(tiny["q_u"], tiny["q_v"], nthreads=8)
    assert np.array_equal(ans.cpu().numpy(), rans) and np.array_equal(code.cpu().numpy(), rcode)


def test_async_invalid_batch_is_latched(tiny):
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64, flags=dbl.FLAG_PERSISTENT | dbl.FLAG_ASYNC)
    ix.sync()
    before = labels_np(ix)
    ix.insert_edges(D(np.array([1, 2], np.int32)), D(np.array([3, tiny["n"] + 5], np.int32)))  # returns at once
    with pytest.raises(dbl.DblError) as e:
        ix.sync()
    assert e.value.status == dbl.DBL_ERR_INVALID
    for a, b in zip(before, labels_np(ix)):
        assert np.array_equal(a, b)
    ix.insert_edges(D(tiny["ins_src"][:500]), D(tiny["ins_dst"][:500]))
    ix.sync()
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build()
    ref.insert_edges(tiny["ins_src"][:500], tiny["ins_dst"][:500])
    assert_labels(ix, ref, "after the latched error was read")


# ---------------------------------------------------------------- autotuner
def test_autotune_restores_index_and_keeps_parity(tiny, tmp_path):
    """dbl_autotune times every schedule from one snapshot and restores the
    index: labels after tuning equal the labels before, the chosen schedule is
    one of the candidates, a cached result is applied without re-measuring,
    and the tuned index still matches the oracle."""
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build()
    s, d = tiny["ins_src"], tiny["ins_dst"]
    before = labels_np(ix)
    cache = str(tmp_path / "sched.json")
    out = ix.autotune(D(s[:1000]), D(d[:1000]), D(tiny["q_u"][:20000]), D(tiny["q_v"][:20000]), trials=1, cache=cache)
    assert out["team"] in (1, 4, 8, 16, 32) and out["best_ms"] > 0
    assert len(out["level_ms"]) == 5 and len(out["persistent_ms"]) == 5
    assert out["query_unroll"] in (1, 2, 4) and all(v > 0 for v in out["query_unroll_ms"].values())
    for a, b in zip(labels_np(ix), before):
        assert np.array_equal(a, b), "autotune changed the index"
    again = ix.autotune(D(s[:1000]), D(d[:1000]), D(tiny["q_u"][:100]), D(tiny["q_v"][:100]), cache=cache)
    assert again.get("cached") and again["team"] == out["team"] and again["query_unroll"] == out["query_unroll"]
    ix.insert_edges(D(s), D(d))
    ref.insert_edges(s, d)
    ix.sync()
    assert_labels(ix, ref, "after autotune")
    assert_queries(ix, ref, tiny["q_u"][:20000], tiny["q_v"][:20000], "after autotune")


def test_phase_trace_and_schedule(tiny):
    """dbl_phase_trace after a persistent insertion: start, one mark per grid
    barrier (validate + count, seed + grow, write + enqueue, each level) and
    the end, non-decreasing; dbl_set_schedule switches team width and
    persistence without changing results."""
    s, d = tiny["ins_src"], tiny["ins_dst"]
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64, flags=dbl.FLAG_TIMING | dbl.FLAG_PERSISTENT)
    ix.insert_edges(D(s[:1000]), D(d[:1000]))
    tr = ix.phase_trace()
    assert len(tr) >= 5 and tr[0] == 0 and all(b >= a for a, b in zip(tr, tr[1:])), tr
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build()
    ref.insert_edges(s[:1000], d[:1000])
    for team, persistent in ((8, False), (32, True), (1, True)):
        ix.set_schedule(team, persistent)
    ix.insert_edges(D(s[1000:]), D(d[1000:]))
    ref.insert_edges(s[1000:], d[1000:])
    ix.sync()
    assert_labels(ix, ref, "after set_schedule")
    with pytest.raises(dbl.DblError):
        ix.set_schedule(3, True)


@pytest.mark.parametrize("flags", [0, dbl.FLAG_PERSISTENT])
@pytest.mark.parametrize("table_log2", [0, 13])
def test_search_overflow_reruns(tiny, flags, table_log2):
    """A tiny first-attempt slice of the search table (2^6 slots) makes the
    waves overflow: they rerun over the whole table, and with a small table
    (2^13 states) split in halves there too; every answer and code still
    equals the oracle's."""
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64, flags=flags, search_first_log2=6,
                      search_table_log2=table_log2)
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build()
    ix.insert_edges(D(tiny["ins_src"]), D(tiny["ins_dst"]))
    ref.insert_edges(tiny["ins_src"], tiny["ins_dst"])
    ix.sync()
    w0 = int(ix.stats()[14])
    assert_queries(ix, ref, tiny["q_u"], tiny["q_v"], f"first slice 2^6, flags {flags}")
    ix.sync()
    assert int(ix.stats()[14]) - w0 > 1, "expected several search waves"


@pytest.mark.parametrize("k,kp", [(64, 64), (16, 16), (128, 64)])
def test_save_load_roundtrip(tiny, tmp_path, k, kp):
    """dbl_save / dbl_load: after half the insertions and 500 added vertices,
    the loaded index has the same sizes, labels and answers as the saved one,
    and takes the rest of the insertions (reserved slots, grown segments,
    edges at the new vertices) to the oracle's labels."""
    n0, add = int(tiny["n"]), 500
    s, d = tiny["ins_src"], tiny["ins_dst"]
    h = s.shape[0] // 2
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), k, kp, flags=dbl.FLAG_PERSISTENT,
                      vertex_capacity=n0 + add + 8, edge_capacity=1 << 16, initial_slots=2)
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], k, kp).build()
    ix.insert_edges(D(s[:h]), D(d[:h]))
    ref.insert_edges(s[:h], d[:h])
    ix.add_vertices(add)
    ref.add_vertices(add)
    rng = np.random.default_rng(23)
    es = np.concatenate([s[h:], rng.integers(n0, n0 + add, 2000).astype(np.int32)])
    ed = np.concatenate([d[h:], rng.integers(0, n0, 2000).astype(np.int32)])
    path = str(tmp_path / "index.dbl")
    ix.save(path)
    ld = dbl.DBLIndex.load(path, flags=dbl.FLAG_PERSISTENT)
    for key in ("n", "k", "kprime", "m", "edges_stored", "edge_capacity", "vertex_capacity", "record_bytes"):
        assert ld.info()[key] == ix.info()[key], key
    for a, b in zip(ix.labels(), ld.labels()):
        assert torch.equal(a, b)
    qu, qv = tiny["q_u"][:30_000], tiny["q_v"][:30_000]
    a1, c1 = ix.query(D(qu), D(qv))
    a2, c2 = ld.query(D(qu), D(qv))
    assert torch.equal(a1, a2) and torch.equal(c1, c2)
    for b in range(0, es.shape[0], 1000):
        ld.insert_edges(D(es[b:b + 1000]), D(ed[b:b + 1000]))
    ref.insert_edges(es, ed)
    ld.sync()
    assert_labels(ld, ref, f"loaded index after the rest of the insertions, k={k} k'={kp}")
    assert_queries(ld, ref, qu, qv, "loaded index, queries")


def test_load_rejects_bad_files(tmp_path):
    """A missing, foreign or truncated file is DBL_ERR_IO."""
    with pytest.raises(dbl.DblError) as e:
        dbl.DBLIndex.load(str(tmp_path / "missing.dbl"))
    assert e.value.status == dbl.DBL_ERR_IO
    junk = tmp_path / "junk.dbl"
    junk.write_bytes(b"not an index" * 100)
    with pytest.raises(dbl.DblError) as e:
        dbl.DBLIndex.load(str(junk))
    assert e.value.status == dbl.DBL_ERR_IO
    rp = np.array([0, 1, 2, 2], np.int32)
    col = np.array([1, 2], np.int32)
    ix = dbl.DBLIndex(D(rp), D(col), 64, 64)
    good = tmp_path / "good.dbl"
    ix.save(str(good))
    data = good.read_bytes()
    short = tmp_path / "short.dbl"
    short.write_bytes(data[: len(data) - 8])
    with pytest.raises(dbl.DblError) as e:
        dbl.DBLIndex.load(str(short))
    assert e.value.status == dbl.DBL_ERR_IO
    ok = dbl.DBLIndex.load(str(good))
    a, _ = ok.query(D(np.array([0, 2], np.int32)), D(np.array([2, 0], np.int32)))
    assert a.cpu().tolist() == [1, 0]
