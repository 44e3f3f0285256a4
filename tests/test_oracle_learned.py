"""Pins for the learned-scorer oracle: features against hand counts, coverage
against brute-force closure, gradients against central finite differences."""
import numpy as np
import pytest

import oracle
from oracle import learned as Lr
from tests import helpers as H


def test_features_on_a_hand_graph():
    # 0 -> 1 -> 2, 0 -> 2, 3 -> 1 ; landmark slot 0 = vertex 1
    rp, col = H.csr_from_edges(4, [0, 1, 0, 3], [1, 2, 2, 1])
    o = oracle.OracleIndex(rp, col, 64, 64)
    lm = np.full(64, -1, np.int32)
    lm[0] = 1
    o.build(lm, *o.zero_degree_leaves())
    F = Lr.feature_counts(rp, col, o.labels(), lm)
    # vertex 1: Pre = {0, 3}, Suc = {2}
    assert list(F[1, :4]) == [2, 1, 2, 3]
    assert F[1, 4] == 0 + 0          # indeg(0) + indeg(3)
    assert F[1, 5] == 0              # outdeg(2)
    assert F[1, 6] == 2 + 1          # outdeg(0) + outdeg(3)
    assert F[1, 7] == 2              # indeg(2)
    assert F[1, 8] == 1 and F[1, 9] == 1 and F[1, 12] == 1   # landmark labels itself
    assert F[2, 8] == 1 and F[2, 9] == 0                     # 1 reaches 2
    assert F[1, 13] == 2             # both in-neighbours are sources
    assert F[0, 14] == 1             # out-neighbour 2 is a sink
    assert F[1, 15] == 1 and F[:, 15].sum() == 1
    assert np.allclose(Lr.features(rp, col, o.labels(), lm), np.log1p(F))


def test_coverage_against_closure():
    n = 150
    s, d = H.random_graph(n, 330, 5)
    rp, col = H.csr_from_edges(n, s, d)
    R = H.closure(n, s, d)
    rng = np.random.default_rng(0)
    pu, pv = np.nonzero(R)
    pick = rng.choice(pu.shape[0], 300, replace=False)
    u, v = pu[pick], pv[pick]
    cnt = Lr.coverage(rp, col, u, v)
    exp = (R[u, :] & R[:, v].T).sum(axis=0)
    assert np.array_equal(cnt, exp)


def _params(seed):
    rng = np.random.default_rng(seed)
    return {"W1": rng.normal(0, 0.5, (16, 128)), "b1": rng.normal(0, 0.1, 128),
            "W2": rng.normal(0, 0.2, (128, 128)), "b2": rng.normal(0, 0.1, 128),
            "w3": rng.normal(0, 0.2, 128), "b3": np.array(0.3)}


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    X = rng.normal(0, 1, (40, 16))
    t = rng.normal(0, 1, 40)
    P = _params(2)
    y, cache = Lr.mlp_forward(X, P)
    g = Lr.mlp_backward(P, cache, y, t)
    eps = 1e-6
    for name, idx in [("W1", (3, 7)), ("W1", (15, 100)), ("b1", (5,)), ("W2", (10, 20)), ("W2", (127, 0)),
                      ("b2", (64,)), ("w3", (9,)), ("b3", ())]:
        Pp = {k: np.array(v, dtype=np.float64, copy=True) for k, v in P.items()}
        Pm = {k: np.array(v, dtype=np.float64, copy=True) for k, v in P.items()}
        Pp[name][idx] += eps
        Pm[name][idx] -= eps
        num = (Lr.mlp_loss(Lr.mlp_forward(X, Pp)[0], t) - Lr.mlp_loss(Lr.mlp_forward(X, Pm)[0], t)) / (2 * eps)
        assert abs(num - np.asarray(g[name])[idx]) <= 1e-6 * max(1.0, abs(num)), name


def test_mlp_closed_forms():
    P = {k: np.zeros_like(v) for k, v in _params(0).items()}
    P["b3"] = np.array(1.5)
    X = np.random.default_rng(3).normal(size=(7, 16))
    y, _ = Lr.mlp_forward(X, P)
    assert np.allclose(y, 1.5)
    # a single active path: y = w3[0] * relu(W2[0,0] * relu(W1[0,0] x0))
    P["b3"] = np.array(0.0)
    P["W1"][0, 0], P["W2"][0, 0], P["w3"][0] = 2.0, 3.0, 0.5
    X = np.zeros((3, 16))
    X[:, 0] = [1.0, -1.0, 0.25]
    y, _ = Lr.mlp_forward(X, P)
    assert np.allclose(y, [3.0, 0.0, 0.75])


def test_sgd_momentum_step():
    P = {"a": np.array([1.0, 2.0])}
    V = {"a": np.array([0.5, 0.0])}
    Lr.sgd_momentum(P, {"a": np.array([1.0, -1.0])}, V, lr=0.1, mu=0.9)
    assert np.allclose(V["a"], [1.45, -1.0]) and np.allclose(P["a"], [0.855, 2.1])
