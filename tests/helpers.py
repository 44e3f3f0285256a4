"""Shared test helpers: brute-force reachability, expected labels from it, the
golden running example, and small graph shapes.

The brute-force closure here is independent of the oracle and of the CUDA
library: it is boolean matrix squaring, R <- R or R*R, from R = I or A, which
reaches the reflexive-transitive closure (Des/Anc include the vertex itself,
Table 1 of the paper) after ceil(log2 n) squarings.
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

CODES = {"undecided": 0, "self": 1, "dl": 2, "bl": 3, "thm1": 4, "thm2": 5, "bfs_pos": 6, "bfs_neg": 7}


def csr_from_edges(n: int, src, dst):
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(row_ptr, src + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    return row_ptr, dst.astype(np.int32)


def edges_from_csr(row_ptr, col):
    n = row_ptr.shape[0] - 1
    src = np.repeat(np.arange(n, dtype=np.int32), np.diff(row_ptr).astype(np.int64))
    return src, np.asarray(col, dtype=np.int32)


def closure(n: int, src, dst) -> np.ndarray:
    """Reflexive-transitive closure R[u, v] = (u reaches v), bool [n, n]."""
    R = np.eye(n, dtype=np.float32)
    if len(src):
        R[np.asarray(src), np.asarray(dst)] = 1.0
    while True:
        R2 = ((R @ R) > 0).astype(np.float32)
        if np.array_equal(R2, R):
            return R.astype(bool)
        R = R2


def pack_bits(mask: np.ndarray, words: int) -> np.ndarray:
    """bool [n, nbits] -> uint64 [n, words] with bit i at word i//64, bit i%64."""
    n, nb = mask.shape
    out = np.zeros((n, words), dtype=np.uint64)
    for i in range(nb):
        if mask[:, i].any():
            out[:, i // 64] |= mask[:, i].astype(np.uint64) << np.uint64(i % 64)
    return out


def expected_labels(R: np.ndarray, landmarks, leaf_bucket, leaf_role, k: int, kprime: int):
    """Labels by definition (Definitions 1-2) from the closure R."""
    n = R.shape[0]
    wd, wb = (k + 63) // 64, (kprime + 63) // 64
    dl_in = np.zeros((n, k), dtype=bool)
    dl_out = np.zeros((n, k), dtype=bool)
    for i, l in enumerate(landmarks):
        if l >= 0:
            dl_in[:, i] = R[l, :]
            dl_out[:, i] = R[:, l]
    bl_in = np.zeros((n, kprime), dtype=bool)
    bl_out = np.zeros((n, kprime), dtype=bool)
    for s in range(n):
        b = leaf_bucket[s]
        if b < 0:
            continue
        if leaf_role[s] & 1:
            bl_in[:, b] |= R[s, :]
        if leaf_role[s] & 2:
            bl_out[:, b] |= R[:, s]
    return (pack_bits(dl_in, wd), pack_bits(dl_out, wd), pack_bits(bl_in, wb),
            pack_bits(bl_out, wb))


def set_bits(words_row) -> set:
    out = set()
    for w, x in enumerate(words_row):
        x = int(x)
        for b in range(64):
            if (x >> b) & 1:
                out.add(w * 64 + b)
    return out


def load_running_example():
    """Parse tests/golden/fig1_running_example.txt (ids converted to 0-based)."""
    ex = dict(edges=[], landmarks=[], leaves=[], dl={}, bl={}, queries=[], inserts=[],
              dl_in_after={}, bl_in_after={})

    def vs(tok):
        return set() if tok == "-" else {int(t) - 1 for t in tok.split(",")}

    def bs(tok):
        return set() if tok == "-" else {int(t) for t in tok.split(",")}

    with open(os.path.join(GOLDEN, "fig1_running_example.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            t = line.split()
            if t[0] == "n":
                ex["n"] = int(t[1])
            elif t[0] == "edge":
                ex["edges"].append((int(t[1]) - 1, int(t[2]) - 1))
            elif t[0] == "landmark":
                ex["landmarks"].append(int(t[1]) - 1)
            elif t[0] == "kprime":
                ex["kprime"] = int(t[1])
            elif t[0] == "leaf":
                ex["leaves"].append((int(t[1]) - 1, t[2], int(t[3])))
            elif t[0] == "dl":
                ex["dl"][int(t[1]) - 1] = (vs(t[2]), vs(t[3]))
            elif t[0] == "bl":
                ex["bl"][int(t[1]) - 1] = (bs(t[2]), bs(t[3]))
            elif t[0] == "query":
                ex["queries"].append((int(t[1]) - 1, int(t[2]) - 1, int(t[3]), t[4]))
            elif t[0] == "insert":
                ex["inserts"].append((int(t[1]) - 1, int(t[2]) - 1))
            elif t[0] == "dl_in_after":
                ex["dl_in_after"][int(t[1]) - 1] = vs(t[2])
            elif t[0] == "bl_in_after":
                ex["bl_in_after"][int(t[1]) - 1] = bs(t[2])
    return ex


def running_example_inputs(ex, k: int, kprime: int):
    """CSR, landmark slots (padded with -1 to k) and leaf arrays of the example."""
    n = ex["n"]
    src, dst = zip(*ex["edges"])
    row_ptr, col = csr_from_edges(n, src, dst)
    landmarks = np.full(k, -1, dtype=np.int32)
    landmarks[: len(ex["landmarks"])] = ex["landmarks"]
    bucket = np.full(n, -1, dtype=np.int32)
    role = np.zeros(n, dtype=np.uint8)
    for v, r, b in ex["leaves"]:
        bucket[v] = b
        role[v] |= 1 if r == "in" else 2
    return row_ptr, col, landmarks, bucket, role


# ---------------------------------------------------------------- graph shapes
def random_graph(n: int, m: int, seed: int):
    """Erdos-Renyi style directed multigraph-free edges with cycles (numpy)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = rng.integers(0, n, m * 2)
    d = rng.integers(0, n, m * 2)
    keep = s != d
    key = np.unique(s[keep].astype(np.int64) * n + d[keep])[:m]
    rng.shuffle(key)
    return (key // n).astype(np.int32), (key % n).astype(np.int32)


def path_graph(n: int, cycle: bool = False):
    s = np.arange(n - 1, dtype=np.int32)
    d = s + 1
    if cycle:
        s = np.append(s, n - 1)
        d = np.append(d, 0)
    return s.astype(np.int32), d.astype(np.int32)


def random_slots(n: int, k: int, used: int, seed: int):
    """k landmark slots, `used` of them distinct random vertices, rest -1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lm = np.full(k, -1, dtype=np.int32)
    pos = rng.choice(k, size=min(used, k, n), replace=False)
    lm[pos] = rng.choice(n, size=pos.shape[0], replace=False)
    return lm


def random_leaves(n: int, kprime: int, frac: float, seed: int):
    """An arbitrary fixed leaf set (Lemma 2 holds for any fixed set)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    role = (rng.random(n) < frac).astype(np.uint8) | ((rng.random(n) < frac).astype(np.uint8) << 1)
    bucket = np.where(role > 0, rng.integers(0, kprime, n), -1).astype(np.int32)
    return bucket, role.astype(np.uint8)
