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


# ---------------------------------------------------------------- scorer error bound
# The scorer's network computes with bf16 operands (features, weights, stored
# activations) and fp32 accumulation.  The oracle evaluates the same
# definition in fp64 with the same bf16 roundings (oracle.learned, q =
# bf16_round).  Two such evaluations differ only by (a) accumulation order and
# fp32 rounding in every sum of K terms, at most GAMMA_UNIT * K times the sum
# of the absolute terms; (b) a bf16 rounding whose input differs: rounding
# (and ReLU) are monotone, so if the input is known within e of v, the
# rounded value lies in [q(v - e), q(v + e)], and it equals q(v) unless a
# rounding boundary falls inside; (c) a ReLU mask that may differ where the
# pre-activation is within its own error of zero.  mlp_error_bound carries
# these as absolute error radii through the forward and backward pass (first
# order, every term by its absolute value), so every element of the result
# bounds |GPU - oracle| for that element.
FP32_U = 2.0 ** -23      # two fp32 units of roundoff
GAMMA_UNIT = 2.0 ** -22  # per accumulated term (4x fp32's worst case)


def _gamma(K):
    return GAMMA_UNIT * K


def _q():
    from oracle import learned as Lr
    return Lr.bf16_round


def _rounded_radius(v, e, relu=False):
    """Radius around q(v) (q(relu(v)) with relu) of the rounded value of any
    input within e of v."""
    q = _q()
    f = (lambda x: q(np.maximum(x, 0.0))) if relu else q
    c = f(v)
    return np.maximum(np.abs(f(v + e) - c), np.abs(f(v - e) - c))


def _masked_radius(D, eD, m, amb):
    """Radius of q(D' * m') around q(D * m), for D' within eD of D and a mask
    m' equal to m except where amb (there it may be 0 or 1)."""
    q = _q()
    c = q(D * m)
    hi = np.maximum(np.abs(q(D + eD)), np.abs(q(D - eD)))
    sure = np.where(m, _rounded_radius(D, eD), 0.0)
    return np.where(amb, hi + np.abs(c), sure)


def mlp_error_bound(P, X, t, eP=None):
    """Element-wise bounds on |g_gpu - g_oracle| for the gradients of the
    network with parameters P (W1, W2 already bf16), features X (bf16), targets
    t; eP: error radii of the parameters themselves (default zero).  Returns
    (bounds dict per parameter, bound on y, bound on the loss)."""
    q = _q()
    eP = eP or {}
    e = {k: np.asarray(eP.get(k, 0.0)) * np.ones_like(np.asarray(P[k], dtype=np.float64)) for k in P}
    A = {k: np.abs(np.asarray(P[k], dtype=np.float64)) for k in P}
    R = X.shape[0]
    aX = np.abs(X)
    Z1 = X @ P["W1"] + P["b1"]
    eZ1 = aX @ e["W1"] + e["b1"] + _gamma(17) * (aX @ A["W1"] + A["b1"])
    H1 = q(np.maximum(Z1, 0.0))
    eH1 = _rounded_radius(Z1, eZ1, relu=True)
    amb1 = (q(np.maximum(Z1 - eZ1, 0.0)) > 0) != (q(np.maximum(Z1 + eZ1, 0.0)) > 0)
    aH1 = np.abs(H1)
    Z2 = H1 @ P["W2"] + P["b2"]
    eZ2 = eH1 @ A["W2"] + (aH1 + eH1) @ e["W2"] + e["b2"] + _gamma(129) * (aH1 @ A["W2"] + A["b2"])
    H2 = q(np.maximum(Z2, 0.0))
    eH2 = _rounded_radius(Z2, eZ2, relu=True)
    amb2 = (q(np.maximum(Z2 - eZ2, 0.0)) > 0) != (q(np.maximum(Z2 + eZ2, 0.0)) > 0)
    aH2 = np.abs(H2)
    y = H2 @ P["w3"] + P["b3"]
    ey = eH2 @ A["w3"] + (aH2 + eH2) @ e["w3"] + e["b3"] + _gamma(129) * (aH2 @ A["w3"] + A["b3"])
    dy = (y - t) / R
    edy = ey / R + FP32_U * np.abs(dy)
    ady = np.abs(dy)
    out = {"w3": eH2.T @ ady + (aH2 + eH2).T @ edy + _gamma(R) * (aH2.T @ ady),
           "b3": edy.sum() + _gamma(R) * ady.sum()}
    D2 = np.outer(dy, P["w3"])
    eD2 = np.outer(edy, A["w3"]) + np.outer(ady + edy, e["w3"]) + FP32_U * np.abs(D2)
    m2 = H2 > 0
    dZ2 = q(D2 * m2)
    edZ2 = _masked_radius(D2, eD2, m2, amb2)
    adZ2 = np.abs(dZ2)
    out["b2"] = edZ2.sum(axis=0) + _gamma(R) * adZ2.sum(axis=0)
    out["W2"] = eH1.T @ adZ2 + (aH1 + eH1).T @ edZ2 + _gamma(R) * (aH1.T @ adZ2)
    D1 = dZ2 @ P["W2"].T
    eD1 = edZ2 @ A["W2"].T + (adZ2 + edZ2) @ e["W2"].T + _gamma(128) * (adZ2 @ A["W2"].T)
    m1 = H1 > 0
    dZ1 = q(D1 * m1)
    edZ1 = _masked_radius(D1, eD1, m1, amb1)
    adZ1 = np.abs(dZ1)
    out["b1"] = edZ1.sum(axis=0) + _gamma(R) * adZ1.sum(axis=0)
    out["W1"] = aX.T @ edZ1 + _gamma(R) * (aX.T @ adZ1)
    r = y - t
    eloss = (np.abs(r) * ey).sum() / R + _gamma(R) * (r * r).sum() / (2 * R)
    return out, ey, eloss


def bf16_weight_radius(p, e):
    """Radius of bf16(p') for any p' within e of p, around bf16(p): a weight
    whose fp32 value is only known within e may round to a neighbouring bf16
    value."""
    from oracle import learned as Lr
    b = Lr.bf16_round(p)
    return np.maximum(np.abs(Lr.bf16_round(p + e) - b), np.abs(Lr.bf16_round(p - e) - b))


MLP_BLOCKS = (("W1", 0, 2048, (16, 128)), ("b1", 2048, 2176, (128,)), ("W2", 2176, 18560, (128, 128)),
              ("b2", 18560, 18688, (128,)), ("w3", 18688, 18816, (128,)), ("b3", 18816, 18817, ()))


def mlp_unflat(p):
    """Flat parameter vector (the library's order) -> dict of float64 arrays."""
    q = np.asarray(p, dtype=np.float64)
    return {name: q[a:b].reshape(shape) for name, a, b, shape in MLP_BLOCKS}


def mlp_flat(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _, _, _ in MLP_BLOCKS])
