"""Pins for the CPU oracle: checks against things other than itself.

* brute-force reflexive-transitive closure (boolean matrix squaring) fixes
  every label bit (Definitions 1-2) and every query answer;
* the paper's running example (Figures 1-2, Section 4 examples) fixes labels,
  leaf choice, four query decisions and one insertion;
* incremental insertion (Algorithm 3) must equal a rebuild (Algorithm 1) on the
  final graph with the same landmark and leaf sets;
* the landmark rule and the leaf hash are pinned to closed forms.
"""
import subprocess
import sys

import numpy as np
import pytest

import oracle
from oracle import OracleIndex
from tests import helpers as H


# ---------------------------------------------------------------- the pin's pin
def test_closure_helper_path_and_cycle():
    s, d = H.path_graph(6)
    R = H.closure(6, s, d)
    assert np.array_equal(R, np.triu(np.ones((6, 6), dtype=bool)))
    s, d = H.path_graph(6, cycle=True)
    assert H.closure(6, s, d).all()
    assert np.array_equal(H.closure(4, [], []), np.eye(4, dtype=bool))


# ---------------------------------------------------------- running example
@pytest.fixture(scope="module")
def example():
    return H.load_running_example()


def _example_index(ex, k, kprime):
    rp, col, lm, bucket, role = H.running_example_inputs(ex, k, kprime)
    o = OracleIndex(rp, col, k, kprime)
    o.build(lm, bucket, role)
    return o, lm


@pytest.mark.parametrize("k,kprime", [(2, 2), (64, 64), (128, 64)])
def test_running_example_labels(example, k, kprime):
    o, lm = _example_index(example, k, kprime)
    dl_in, dl_out, bl_in, bl_out = o.labels()
    slot_of = {int(v): i for i, v in enumerate(lm) if v >= 0}
    for v, (e_in, e_out) in example["dl"].items():
        assert H.set_bits(dl_in[v]) == {slot_of[x] for x in e_in}, f"DL_in(v{v+1})"
        assert H.set_bits(dl_out[v]) == {slot_of[x] for x in e_out}, f"DL_out(v{v+1})"
    for v, (e_in, e_out) in example["bl"].items():
        assert H.set_bits(bl_in[v]) == e_in, f"BL_in(v{v+1})"
        assert H.set_bits(bl_out[v]) == e_out, f"BL_out(v{v+1})"


def test_running_example_zero_degree_leaves(example):
    rp, col, *_ = H.running_example_inputs(example, 2, 2)
    o = OracleIndex(rp, col, 2, 2)
    bucket, role = o.zero_degree_leaves()
    sources = {v for v in range(example["n"]) if role[v] & 1}
    sinks = {v for v in range(example["n"]) if role[v] & 2}
    assert sources == {0, 1, 2}          # v1, v2, v3
    assert sinks == {9, 10}              # v10, v11
    assert all(bucket[v] == -1 for v in range(example["n"]) if role[v] == 0)


def test_running_example_queries(example):
    o, _ = _example_index(example, 2, 2)
    u = [q[0] for q in example["queries"]]
    v = [q[1] for q in example["queries"]]
    ans, code = o.query(u, v)
    for i, (_, _, a, rule) in enumerate(example["queries"]):
        assert ans[i] == a
        assert code[i] == H.CODES[rule]


def test_running_example_insertion(example):
    o, lm = _example_index(example, 2, 2)
    slot_of = {int(v): i for i, v in enumerate(lm) if v >= 0}
    before = o.labels()
    s, d = zip(*example["inserts"])
    o.insert_edges(s, d)
    dl_in, dl_out, bl_in, bl_out = o.labels()
    for v, e in example["dl_in_after"].items():
        assert H.set_bits(dl_in[v]) == {slot_of[x] for x in e}, f"DL_in(v{v+1}) after"
    for v, e in example["bl_in_after"].items():
        assert H.set_bits(bl_in[v]) == e, f"BL_in(v{v+1}) after"
    # Figure 2: nothing else changes (DL_out, BL_out of this example included)
    assert np.array_equal(dl_out, before[1])
    assert np.array_equal(bl_out, before[3])
    # v2 is now in the SCC {v2, v5, v6, v9} (Section 3)
    ans, code = o.query([1, 4], [4, 1])
    assert list(ans) == [1, 1]


# ------------------------------------------------------------ closure pins
def _shapes():
    out = []
    for seed in range(3):
        s, d = H.random_graph(120, 300 + 100 * seed, seed)
        out.append(("er%d" % seed, 120, s, d))
    s, d = H.path_graph(90)
    out.append(("path", 90, s, d))
    s, d = H.path_graph(70, cycle=True)
    out.append(("cycle", 70, s, d))
    s, d = H.random_graph(200, 180, 7)          # sparse, many leaves
    out.append(("sparse", 200, s, d))
    out.append(("empty", 10, np.zeros(0, np.int32), np.zeros(0, np.int32)))
    import dbl_inputs
    rp, col = dbl_inputs.rmat_csr(256, 900, 11)
    s, d = H.edges_from_csr(rp, col)
    out.append(("rmat", 256, s, d))
    return out


SHAPES = _shapes()


def _selections(n, k, kprime, o, mode, seed):
    if mode == "degree":
        lm = o.degree_landmarks()
        bucket, role = o.zero_degree_leaves()
    else:
        lm = H.random_slots(n, k, min(k, max(1, n // 4)), seed)
        bucket, role = H.random_leaves(n, kprime, 0.3, seed + 1)
    return lm, bucket, role


@pytest.mark.parametrize("shape", SHAPES, ids=[s[0] for s in SHAPES])
@pytest.mark.parametrize("k,kprime,mode", [(64, 64, "degree"), (128, 64, "random"),
                                           (64, 128, "random"), (3, 5, "random"), (16, 16, "degree"),
                                           (32, 16, "random"), (16, 32, "random"), (32, 32, "degree")])
def test_labels_and_answers_match_closure(shape, k, kprime, mode):
    name, n, s, d = shape
    rp, col = H.csr_from_edges(n, s, d)
    o = OracleIndex(rp, col, k, kprime)
    lm, bucket, role = _selections(n, k, kprime, o, mode, 5)
    o.build(lm, bucket, role)
    R = H.closure(n, s, d)
    exp = H.expected_labels(R, lm, bucket, role, k, kprime)
    got = o.labels()
    for e, g, nm in zip(exp, got, ["dl_in", "dl_out", "bl_in", "bl_out"]):
        assert np.array_equal(e, g), nm
    uu, vv = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ans, code = o.query(uu.ravel(), vv.ravel(), nthreads=4)
    assert np.array_equal(ans.astype(bool), R.ravel())
    _check_codes(R, exp, uu.ravel(), vv.ravel(), code)


def _check_codes(R, labels, u, v, code):
    """Expected deciding rule from closure-derived labels, in Algorithm 2's
    order (self, DL, BL, Theorem 1, Theorem 2, search)."""
    dl_in, dl_out, bl_in, bl_out = labels
    inter = lambda x, y: (dl_out[x] & dl_in[y]).any(axis=-1)
    contain = lambda x, y: (((bl_in[x] & ~bl_in[y]) == 0).all(axis=-1)
                            & ((bl_out[y] & ~bl_out[x]) == 0).all(axis=-1))
    exp = np.where(u == v, 1,
          np.where(inter(u, v), 2,
          np.where(~contain(u, v), 3,
          np.where(inter(v, u), 4,
          np.where(inter(u, u) | inter(v, v), 5,
          np.where(R[u, v], 6, 7))))))
    assert np.array_equal(code, exp)
    # soundness of every rule (Lemmas 1-2, Theorems 1-2)
    truth = R[u, v]
    assert truth[np.isin(code, [1, 2, 6])].all()
    assert not truth[np.isin(code, [3, 4, 5, 7])].any()


def test_two_hop_special_case():
    """With L = V the DL label is the full 2-hop cover (Section 4.1): every
    reachable pair is decided by DL, so the search never runs."""
    n = 60
    s, d = H.random_graph(n, 150, 3)
    rp, col = H.csr_from_edges(n, s, d)
    o = OracleIndex(rp, col, 64, 64)
    o.build(np.concatenate([np.arange(n), -np.ones(4)]).astype(np.int32),
            *o.zero_degree_leaves())
    uu, vv = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ans, code = o.query(uu.ravel(), vv.ravel())
    assert not np.isin(code, [6, 7]).any()
    assert np.array_equal(ans.astype(bool), H.closure(n, s, d).ravel())


# ------------------------------------------------------ incremental == rebuild
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_incremental_equals_rebuild(seed):
    n = 150
    s, d = H.random_graph(n, 220, 100 + seed)
    base, extra = slice(0, 160), slice(160, 220)
    rp, col = H.csr_from_edges(n, s[base], d[base])
    inc = OracleIndex(rp, col, 64, 64)
    lm = inc.degree_landmarks()
    bucket, role = inc.zero_degree_leaves()     # frozen at build
    inc.build(lm, bucket, role)
    prev = inc.labels()
    for i in range(160, 220):
        inc.insert_edges([s[i]], [d[i]])
        cur = inc.labels()
        for a, b in zip(prev, cur):             # monotone: labels only gain bits
            assert np.array_equal(a & b, a)
        prev = cur
    # plus a duplicate and a self-loop, which change nothing
    inc.insert_edges([s[0], 5], [d[0], 5])
    rp2, col2 = H.csr_from_edges(n, s, d)
    reb = OracleIndex(rp2, col2, 64, 64).build(lm, bucket, role)
    for a, b in zip(inc.labels(), reb.labels()):
        assert np.array_equal(a, b)
    R = H.closure(n, s, d)
    for a, b in zip(inc.labels(), H.expected_labels(R, lm, bucket, role, 64, 64)):
        assert np.array_equal(a, b)


def test_insert_order_and_batching_invariance():
    n = 120
    s, d = H.random_graph(n, 260, 9)
    rp, col = H.csr_from_edges(n, s[:150], d[:150])
    a = OracleIndex(rp, col, 64, 64).build()
    b = OracleIndex(rp, col, 64, 64).build(a.landmarks, a.leaf_bucket, a.leaf_role)
    a.insert_edges(s[150:], d[150:])
    b.insert_edges(s[150:][::-1], d[150:][::-1])
    for x, y in zip(a.labels(), b.labels()):
        assert np.array_equal(x, y)


# ------------------------------------------------------------- closed forms
def test_degree_landmark_rule():
    n = 300
    s, d = H.random_graph(n, 900, 4)
    rp, col = H.csr_from_edges(n, s, d)
    o = OracleIndex(rp, col, 64, 64)
    indeg = np.bincount(d, minlength=n).astype(np.int64)
    outdeg = np.bincount(s, minlength=n).astype(np.int64)
    M = indeg * outdeg
    order = np.lexsort((np.arange(n), -M))      # M desc, id asc
    assert np.array_equal(o.degree_landmarks(), order[:64])
    # k > n: trailing slots empty
    o2 = OracleIndex(*H.csr_from_edges(10, [0, 1], [1, 2]), 64, 64)
    lm = o2.degree_landmarks()
    assert lm[0] == 1 and (lm[10:] == -1).all() and sorted(lm[:10]) == list(range(10))


# Section 6, "Label Node Selection": Table 3's rankings and the M(u) <= r leaf rule,
# worked by hand on edges 0->1, 0->2, 0->3, 1->2, 2->3, 4->2, 5->4:
#   vertex (in, out):  0 (0,3)  1 (1,1)  2 (3,1)  3 (2,0)  4 (1,1)  5 (0,1)
#   M = in*out:        0        1        3        0        1        0
#   A = max:           3        1        3        2        1        1
#   B = min:           0        1        1        0        1        0
#   C = in+out:        3        2        4        2        2        1
HAND_EDGES = ([0, 0, 0, 1, 2, 4, 5], [1, 2, 3, 2, 3, 2, 4])
HAND_ORDER = {"M": [2, 1, 4, 0, 3, 5], "A": [0, 2, 3, 1, 4, 5], "B": [1, 2, 4, 0, 3, 5],
              "C": [2, 0, 1, 3, 4, 5]}
# roles: 1 = seeds BL_in (no in-edges), 2 = seeds BL_out (no out-edges), 3 = both (0 < M <= r)
HAND_ROLES = {0: [1, 0, 0, 2, 0, 1], 1: [1, 3, 0, 2, 3, 1], 2: [1, 3, 0, 2, 3, 1], 3: [1, 3, 3, 2, 3, 1]}


@pytest.mark.parametrize("rule", ["M", "A", "B", "C"])
def test_table3_rankings_hand_example(rule):
    o = OracleIndex(*H.csr_from_edges(6, *HAND_EDGES), 64, 64)
    lm = o.rank_landmarks(rule)
    assert lm[:6].tolist() == HAND_ORDER[rule] and (lm[6:] == -1).all()
    if rule == "M":
        assert np.array_equal(lm, o.degree_landmarks())


@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_threshold_leaves_hand_example(r):
    o = OracleIndex(*H.csr_from_edges(6, *HAND_EDGES), 64, 64)
    bucket, role = o.threshold_leaves(r)
    assert role.tolist() == HAND_ROLES[r]
    assert ((bucket >= 0) == (role > 0)).all()
    for v in np.nonzero(role)[0]:
        assert bucket[v] == oracle.leaf_hash(int(v), 64)
    if r == 0:
        zb, zr = o.zero_degree_leaves()
        assert np.array_equal(zb, bucket) and np.array_equal(zr, role)


@pytest.mark.parametrize("shape", SHAPES, ids=[s[0] for s in SHAPES])
@pytest.mark.parametrize("rule,r", [("A", 1), ("B", 4), ("C", 1000)])
def test_selection_rules_match_closure(shape, rule, r):
    """Labels and answers with Table 3 landmarks and M(u) <= r leaves equal the
    closure-derived definitions (Lemma 1, Lemma 2 hold for any fixed sets)."""
    name, n, s, d = shape
    rp, col = H.csr_from_edges(n, s, d)
    o = OracleIndex(rp, col, 64, 64)
    lm = o.rank_landmarks(rule)
    bucket, role = o.threshold_leaves(r)
    o.build(lm, bucket, role)
    R = H.closure(n, s, d)
    exp = H.expected_labels(R, lm, bucket, role, 64, 64)
    for e, g, nm in zip(exp, o.labels(), ["dl_in", "dl_out", "bl_in", "bl_out"]):
        assert np.array_equal(e, g), nm
    uu, vv = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ans, code = o.query(uu.ravel(), vv.ravel(), nthreads=4)
    assert np.array_equal(ans.astype(bool), R.ravel())
    _check_codes(R, exp, uu.ravel(), vv.ravel(), code)


# ------------------------------------------------------------ vertex insertion (Section 1)
@pytest.mark.parametrize("seed", range(3))
def test_vertex_insertion_matches_closure(seed):
    """New vertices start isolated (empty labels, not landmarks, not leaves);
    after edges touching them are inserted, every label and answer equals the
    closure-derived definition on the final graph with the build's landmark
    and leaf sets extended by non-leaves."""
    rng = np.random.default_rng(40 + seed)
    n0, add = 90, 30
    s, d = H.random_graph(n0, 260, seed)
    o = OracleIndex(*H.csr_from_edges(n0, s, d), 64, 64).build()
    lm = o.landmarks.copy()
    first = o.add_vertices(add)
    assert first == n0 and o.n == n0 + add
    lab = o.labels()
    assert all((x[n0:] == 0).all() for x in lab)                # isolated: empty labels
    ans, code = o.query(np.arange(n0, n0 + add), np.arange(n0, n0 + add))
    assert ans.all() and (code == oracle.SELF).all()
    ans, _ = o.query(np.full(n0, n0, np.int32), np.arange(n0))   # a new vertex reaches nothing else
    assert not ans.any()
    n = n0 + add
    es = rng.integers(0, n, 400).astype(np.int32)
    ed = rng.integers(0, n, 400).astype(np.int32)
    o.insert_edges(es, ed)
    fs, fd = np.concatenate([s, es]), np.concatenate([d, ed])
    R = H.closure(n, fs, fd)
    exp = H.expected_labels(R, lm, o.leaf_bucket, o.leaf_role, 64, 64)
    for e, g, nm in zip(exp, o.labels(), ["dl_in", "dl_out", "bl_in", "bl_out"]):
        assert np.array_equal(e, g), nm
    assert (o.leaf_bucket[n0:] == -1).all() and (o.leaf_role[n0:] == 0).all()
    uu, vv = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ans, code = o.query(uu.ravel(), vv.ravel(), nthreads=4)
    assert np.array_equal(ans.astype(bool), R.ravel())
    _check_codes(R, exp, uu.ravel(), vv.ravel(), code)


@pytest.mark.parametrize("rule,r", [("A", 1), ("C", 3)])
def test_vertex_insertion_with_selection_rules_equals_rebuild(rule, r):
    """Table 3 landmarks, M(u) <= r leaves, then new vertices and edges touching
    them: incremental labels equal a rebuild on the final graph with the same
    landmark and leaf sets (new vertices are not leaves), and the closure."""
    rng = np.random.default_rng(61)
    n0, add = 150, 40
    s, d = H.random_graph(n0, 420, 9)
    o = OracleIndex(*H.csr_from_edges(n0, s, d), 64, 64)
    lm = o.rank_landmarks(rule)
    lb, lr = o.threshold_leaves(r)
    o.build(lm, lb, lr)
    o.add_vertices(add)
    n = n0 + add
    es = rng.integers(0, n, 500).astype(np.int32)
    ed = rng.integers(0, n, 500).astype(np.int32)
    for b in range(0, 500, 125):
        o.insert_edges(es[b:b + 125], ed[b:b + 125])
    fs, fd = np.concatenate([s, es]), np.concatenate([d, ed])
    lb2 = np.concatenate([lb, np.full(add, -1, np.int32)])
    lr2 = np.concatenate([lr, np.zeros(add, np.uint8)])
    rebuilt = OracleIndex(*H.csr_from_edges(n, fs, fd), 64, 64).build(lm, lb2, lr2)
    R = H.closure(n, fs, fd)
    exp = H.expected_labels(R, lm, lb2, lr2, 64, 64)
    for e, g, b2, nm in zip(exp, o.labels(), rebuilt.labels(), ["dl_in", "dl_out", "bl_in", "bl_out"]):
        assert np.array_equal(e, g), nm
        assert np.array_equal(g, b2), nm


def test_vertex_insertion_rejects_bad_counts_and_ids():
    o = OracleIndex(*H.csr_from_edges(5, [0, 1], [1, 2]), 64, 64).build()
    with pytest.raises(ValueError):
        o.add_vertices(-1)
    with pytest.raises(Exception):
        o.insert_edges([0], [5])                                 # id 5 does not exist yet
    o.add_vertices(1)
    o.insert_edges([0], [5])
    ans, code = o.query([1], [5])
    assert not ans[0]
    ans, code = o.query([0], [5])
    assert ans[0]


@pytest.mark.parametrize("kprime", [1, 2, 64, 128, 256, 100])
def test_leaf_hash_fibonacci(kprime):
    phi = 0x9E3779B97F4A7C15
    for v in [0, 1, 2, 3, 1000, 123457, 2**31 - 1]:
        x = (v * phi) % 2**64
        exp = (x * kprime) >> 64
        if kprime & (kprime - 1) == 0 and kprime > 1:
            assert exp == x >> (64 - kprime.bit_length() + 1)
        assert oracle.leaf_hash(v, kprime) == exp


def test_parallel_build_and_query_match_sequential():
    import dbl_inputs
    rp, col = dbl_inputs.rmat_csr(4096, 20000, 21)
    a = OracleIndex(rp, col, 128, 64).build(nthreads=1)
    b = OracleIndex(rp, col, 128, 64).build(nthreads=6)
    for x, y in zip(a.labels(), b.labels()):
        assert np.array_equal(x, y)
    qu, qv = dbl_inputs.queries(rp, col, 5000, 3, True)
    a1, c1 = a.query(qu, qv, nthreads=1)
    a2, c2 = a.query(qu, qv, nthreads=6)
    assert np.array_equal(a1, a2) and np.array_equal(c1, c2)


def test_invalid_ids_rejected():
    rp, col = H.csr_from_edges(5, [0, 1], [1, 2])
    o = OracleIndex(rp, col, 64, 64).build()
    with pytest.raises(ValueError):
        o.query([0], [5])
    with pytest.raises(ValueError):
        o.insert_edges([-1], [2])
