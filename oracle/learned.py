"""CPU oracle for the learned landmark scorer (not part of the paper).

TEST INFRASTRUCTURE ONLY (see the package docstring): plain numpy, float64.
The paper picks landmarks by M(u) = |Pre(u)|*|Suc(u)| (Section 4.1) and
notes that the optimal choice is NP-hard; the scorer replaces that ranking
with a small network trained on how many sampled reachable pairs each vertex
would decide as a landmark.  Answers stay exact whatever the ranking: only
which pairs the DL test decides changes (Lemma 1 holds for any landmark set).

* ``features``   16 per-vertex counts, log1p-scaled (definitions below).
* ``coverage``   for sampled reachable pairs (u_j, v_j): the number of j with
                 u_j reaching c and c reaching v_j -- exactly the pairs that
                 DL_out(u_j) and DL_in(v_j) would share if c were a landmark
                 (Lemma 1 with L = {c}).
* ``mlp_*``      16-128-128-1 ReLU network, squared loss, plain definitions;
                 optionally with the stored activations rounded to bf16, the
                 network's storage type.
* ``sgd_momentum`` the training step: momentum SGD on element-wise clipped
                 gradients.
"""
from __future__ import annotations

import numpy as np

FEATURE_NAMES = [
    "indeg", "outdeg", "indeg*outdeg", "indeg+outdeg",
    "sum_pre_indeg", "sum_suc_outdeg", "sum_pre_outdeg", "sum_suc_indeg",
    "popc_dl_in", "popc_dl_out", "popc_bl_in", "popc_bl_out",
    "popc_dl_in*popc_dl_out", "pre_source_leaves", "suc_sink_leaves", "is_landmark",
]


def _popc_rows(words: np.ndarray) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint64)
    b = w.view(np.uint8).reshape(w.shape[0], -1)
    return np.unpackbits(b, axis=1).sum(axis=1).astype(np.float64)


def feature_counts(row_ptr, col, labels, landmarks) -> np.ndarray:
    """Raw counts [n, 16] (before log1p) from the graph and a built index's
    labels (dl_in, dl_out, bl_in, bl_out) and landmark slots."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = row_ptr.shape[0] - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    outdeg = np.diff(row_ptr).astype(np.float64)
    indeg = np.bincount(col, minlength=n).astype(np.float64)
    F = np.zeros((n, 16), dtype=np.float64)
    F[:, 0] = indeg
    F[:, 1] = outdeg
    F[:, 2] = indeg * outdeg
    F[:, 3] = indeg + outdeg
    F[:, 4] = np.bincount(col, weights=indeg[src], minlength=n)      # over p in Pre(x): indeg(p)
    F[:, 5] = np.bincount(src, weights=outdeg[col], minlength=n)     # over s in Suc(x): outdeg(s)
    F[:, 6] = np.bincount(col, weights=outdeg[src], minlength=n)     # over p in Pre(x): outdeg(p)
    F[:, 7] = np.bincount(src, weights=indeg[col], minlength=n)      # over s in Suc(x): indeg(s)
    dl_in, dl_out, bl_in, bl_out = labels
    F[:, 8] = _popc_rows(dl_in)
    F[:, 9] = _popc_rows(dl_out)
    F[:, 10] = _popc_rows(bl_in)
    F[:, 11] = _popc_rows(bl_out)
    F[:, 12] = F[:, 8] * F[:, 9]
    F[:, 13] = np.bincount(col, weights=(indeg[src] == 0).astype(np.float64), minlength=n)
    F[:, 14] = np.bincount(src, weights=(outdeg[col] == 0).astype(np.float64), minlength=n)
    lm = np.asarray(landmarks)
    F[lm[lm >= 0], 15] = 1.0
    return F


def features(row_ptr, col, labels, landmarks) -> np.ndarray:
    """log1p of the counts, float64 [n, 16]."""
    return np.log1p(feature_counts(row_ptr, col, labels, landmarks))


def coverage(row_ptr, col, u, v) -> np.ndarray:
    """count[c] = #{j : u_j reaches c and c reaches v_j}, by one forward BFS
    from u_j and one backward BFS from v_j per pair (reachability is
    reflexive, Table 1)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = row_ptr.shape[0] - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    order = np.argsort(col, kind="stable")
    in_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(in_ptr, col + 1, 1)
    in_ptr = np.cumsum(in_ptr)
    in_col = src[order]

    def reach(start, ptr, adj):
        seen = np.zeros(n, dtype=bool)
        seen[start] = True
        stack = [start]
        while stack:
            x = stack.pop()
            for y in adj[ptr[x]:ptr[x + 1]]:
                if not seen[y]:
                    seen[y] = True
                    stack.append(int(y))
        return seen

    count = np.zeros(n, dtype=np.int64)
    for a, b in zip(u, v):
        count += reach(int(a), row_ptr, col) & reach(int(b), in_ptr, in_col)
    return count


# ------------------------------------------------------------------ the network
def _identity(a):
    return a


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64: the
    8-bit-significand storage type of the network's operands.  Written from
    the format's definition: keep the top 16 bits of the float32 pattern,
    rounding on the 16 bits dropped."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64)).reshape(np.shape(a))


def mlp_forward(X, P, q=_identity):
    """X [R,16]; P = dict(W1 [16,128], b1, W2 [128,128], b2, w3 [128], b3).
    Returns y [R] and the cache for mlp_backward.  `q` rounds the stored
    activations H1, H2 (identity: the plain definition; bf16_round: the
    network evaluated with bf16 activations, as its tensor-core kernels store
    them)."""
    Z1 = X @ P["W1"] + P["b1"]
    H1 = q(np.maximum(Z1, 0.0))
    Z2 = H1 @ P["W2"] + P["b2"]
    H2 = q(np.maximum(Z2, 0.0))
    y = H2 @ P["w3"] + P["b3"]
    return y, (X, Z1, H1, Z2, H2)


def mlp_loss(y, t):
    """Mean squared error / 2."""
    return 0.5 * np.mean((y - t) ** 2)


def mlp_backward(P, cache, y, t, q=_identity):
    """Gradients of mlp_loss with respect to every parameter (chain rule).
    `q` rounds the stored backward activations dZ2, dZ1 (as in mlp_forward)."""
    X, Z1, H1, Z2, H2 = cache
    R = X.shape[0]
    dy = (y - t) / R
    g = {"w3": H2.T @ dy, "b3": dy.sum()}
    dZ2 = q(np.outer(dy, P["w3"]) * (H2 > 0))
    g["W2"] = H1.T @ dZ2
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = q((dZ2 @ P["W2"].T) * (H1 > 0))
    g["W1"] = X.T @ dZ1
    g["b1"] = dZ1.sum(axis=0)
    return g


CLIP = 1.0  # element-wise gradient clip of the scorer's training step


def clip_grad(g, c=CLIP):
    """Each gradient element limited to [-c, c]; a non-finite element is 0."""
    g = np.asarray(g, dtype=np.float64)
    return np.where(np.isfinite(g), np.clip(g, -c, c), 0.0)


def sgd_momentum(P, g, V, lr, mu, clip=CLIP):
    """v <- mu*v + clip(g); p <- p - lr*v, for every parameter (clip=None:
    no clipping)."""
    for k in P:
        gk = g[k] if clip is None else clip_grad(g[k], clip)
        V[k] = mu * V[k] + gk
        P[k] = P[k] - lr * V[k]
