"""The seeded input generators: exact sizes, validity, determinism."""
import os
import subprocess
import sys

import numpy as np

import dbl_inputs
from tests import helpers as H


def test_rmat_exact_simple_sorted():
    for n, m, seed in [(16384, 80_000, 1), (1000, 5000, 7), (3000, 1, 2)]:
        rp, col = dbl_inputs.rmat_csr(n, m, seed)
        assert rp[0] == 0 and rp[-1] == m and col.shape[0] == m
        assert (np.diff(rp) >= 0).all()
        src, dst = H.edges_from_csr(rp, col)
        assert (src != dst).all()
        assert ((0 <= dst) & (dst < n)).all()
        key = src.astype(np.int64) * n + dst
        assert (np.diff(key) > 0).all()            # rows sorted, no duplicates


def test_rmat_skew_and_permutation():
    rp, col = dbl_inputs.rmat_csr(1 << 14, 80_000, 1)
    outdeg = np.diff(rp)
    # power-law: the max degree is far above the mean, and hubs are not at id 0
    assert outdeg.max() > 20 * outdeg.mean()
    assert np.argmax(outdeg) != 0


def test_splitmix64_reference_values():
    # splitmix64 seeded with 1234567: published first outputs (Vigna's reference code)
    assert dbl_inputs.splitmix64_at(1234567, 0) == 6457827717110365317
    assert dbl_inputs.splitmix64_at(1234567, 1) == 3203168211198807973


def test_thread_count_independent():
    code = ("import dbl_inputs,hashlib;rp,c=dbl_inputs.rmat_csr(5000,40000,3);"
            "u,v=dbl_inputs.queries(rp,c,2000,4,True);"
            "print(hashlib.sha1(rp.tobytes()+c.tobytes()+u.tobytes()+v.tobytes()).hexdigest())")
    outs = []
    for t in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=t)
        outs.append(subprocess.check_output([sys.executable, "-c", code], env=env,
                                            cwd=H.GOLDEN + "/../..").strip())
    assert outs[0] == outs[1]


def test_insertions_new_and_distinct():
    rp, col = dbl_inputs.rmat_csr(2000, 8000, 5)
    s, d = dbl_inputs.insertions(rp, col, 3000, 6)
    assert (s != d).all()
    n = 2000
    existing = set((H.edges_from_csr(rp, col)[0].astype(np.int64) * n + col).tolist())
    keys = s.astype(np.int64) * n + d
    assert len(set(keys.tolist())) == 3000
    assert not (set(keys.tolist()) & existing)


def test_query_mix_descendants():
    n = 600
    rp, col = dbl_inputs.rmat_csr(n, 2500, 8)
    s, d = dbl_inputs.insertions(rp, col, 100, 9)
    es, ed = H.edges_from_csr(rp, col)
    R = H.closure(n, np.concatenate([es, s]), np.concatenate([ed, d]))
    for exact in (True, False):
        qu, qv = dbl_inputs.queries(rp, col, 4000, 10, exact, s, d)
        odd = np.arange(1, 4000, 2)
        assert R[qu[odd], qv[odd]].all()            # odd: descendants
        assert (qu[odd] != qv[odd]).all()
        even = np.arange(0, 4000, 2)
        assert R[qu[even], qv[even]].mean() < 0.9    # even: uniform pairs, mixed


def test_loguniform_batches():
    b = dbl_inputs.loguniform_batches(1_000_000, 1, 200_000, 5)
    assert b.sum() == 1_000_000 and b.min() >= 1 and b.max() <= 200_000
    assert len(set(b.tolist())) > 5


def test_community_dag_structure():
    """community_dag: sorted rows, no self-loops or duplicates, ids a
    permutation of [0, n); edges between communities only from the earlier to
    the later one, so the condensation of the communities is acyclic (no edge
    closes a cycle between two communities)."""
    n, m, C = 20_000, 150_000, 16
    rp, col = dbl_inputs.community_dag(n, m, C, 1.0, 0.05, 3)
    assert rp.shape == (n + 1,) and rp[0] == 0 and rp[-1] == col.shape[0] <= m
    assert np.all(np.diff(rp) >= 0)
    src = np.repeat(np.arange(n), np.diff(rp))
    assert not np.any(src == col)
    key = src.astype(np.int64) * n + col
    assert np.all(np.diff(key) > 0)                       # rows sorted, no duplicates
    # recover each vertex's community from the generator's recipe: the same
    # sizes and the same relabelling
    w = np.array([(c + 1.0) ** -1.0 for c in range(C)])
    sizes = np.maximum(64, np.floor(w / w.sum() * n)).astype(np.int64)
    sizes[0] += n - sizes.sum()
    comm_of_old = np.repeat(np.arange(C), sizes)
    perm = dbl_inputs.permutation(n, 4).astype(np.int64)  # seed + 1
    comm = np.empty(n, np.int64)
    comm[perm] = comm_of_old
    cs, cd = comm[src], comm[col]
    assert np.all(cs <= cd)                               # never from a later community to an earlier one
    cross = np.count_nonzero(cs < cd)
    assert 0.02 * m < cross < 0.08 * m                    # about 5% of the edges cross
    # the largest community holds the largest share of the edges
    per = np.bincount(cs, minlength=C)
    assert per.argmax() == 0
