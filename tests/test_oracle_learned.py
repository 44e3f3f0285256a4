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


def test_sgd_step_clips_each_gradient_element():
    """The training step limits each gradient element to [-1, 1] and drops
    non-finite ones before the momentum update (worked by hand)."""
    P = {"a": np.zeros(6)}
    V = {"a": np.zeros(6)}
    Lr.sgd_momentum(P, {"a": np.array([2.5, -3.0, 0.5, np.nan, np.inf, -np.inf])}, V, lr=0.1, mu=0.9)
    assert np.array_equal(V["a"], [1.0, -1.0, 0.5, 0.0, 0.0, 0.0])
    assert np.allclose(P["a"], [-0.1, 0.1, -0.05, 0.0, 0.0, 0.0])
    Lr.sgd_momentum(P, {"a": np.array([0.2, 7.0, -0.5, 1.0, -1.0, 0.0])}, V, lr=0.1, mu=0.9)
    assert np.allclose(V["a"], [1.1, 0.1, -0.05, 1.0, -1.0, 0.0])
    assert np.allclose(P["a"], [-0.21, 0.09, -0.045, -0.1, 0.1, 0.0])
    # clip=None is the plain momentum step
    P2, V2 = {"a": np.zeros(1)}, {"a": np.zeros(1)}
    Lr.sgd_momentum(P2, {"a": np.array([3.0])}, V2, lr=0.1, mu=0.9, clip=None)
    assert np.allclose(P2["a"], [-0.3])


def test_bf16_round_by_the_format():
    """Round to nearest, ties to even, on an 8-bit significand (7 stored bits)."""
    u = 2.0 ** -7
    x = np.array([1.0, 1 + u / 2, 1 + 3 * u / 2, 1 + u / 2 + 2 ** -20, -(1 + 3 * u / 2), 2 ** -130, 0.0, 3.0e38],
                 dtype=np.float64)
    want = [1.0, 1.0, 1 + 2 * u, 1 + u, -(1 + 2 * u), 2 ** -130, 0.0, None]
    got = Lr.bf16_round(x)
    for g, w_ in zip(got[:-1], want[:-1]):
        assert g == w_
    assert np.isfinite(got[-1]) or np.isinf(got[-1])
    # agrees with torch's bfloat16 conversion (an independent implementation)
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(3).normal(0, 5, 20000).astype(np.float32)
    assert np.array_equal(Lr.bf16_round(r), torch.from_numpy(r).to(torch.bfloat16).float().numpy())


def _f32_grads(P, X, t):
    """The same network and gradients evaluated in float32 arithmetic with the
    same bf16 storage roundings (a second, independent evaluation order)."""
    f = np.float32
    q = lambda a: Lr.bf16_round(a).astype(f)
    W1, b1, W2, b2, w3, b3 = (np.asarray(P[k], f) for k in ("W1", "b1", "W2", "b2", "w3", "b3"))
    X = X.astype(f)
    H1 = q(np.maximum(X @ W1 + b1, 0))
    H2 = q(np.maximum(H1 @ W2 + b2, 0))
    y = H2 @ w3 + b3
    R = X.shape[0]
    dy = ((y - t.astype(f)) / f(R)).astype(f)
    dZ2 = q(np.outer(dy, w3) * (H2 > 0))
    dZ1 = q((dZ2 @ W2.T) * (H1 > 0))
    return {"W1": X.T @ dZ1, "b1": dZ1.sum(0), "W2": H1.T @ dZ2, "b2": dZ2.sum(0), "w3": H2.T @ dy,
            "b3": dy.sum()}


def _bound_case(seed, R=600):
    rng = np.random.default_rng(seed)
    P = _params(seed)
    for k in ("W1", "W2"):
        P[k] = Lr.bf16_round(P[k])
    X = Lr.bf16_round(rng.normal(0.5, 1.0, (R, 16)))
    t = rng.normal(3.0, 0.5, R)  # residuals bounded away from zero
    y, cache = Lr.mlp_forward(X, P, Lr.bf16_round)
    g = Lr.mlp_backward(P, cache, y, t, Lr.bf16_round)
    bound, _, _ = H.mlp_error_bound(P, X, t)
    return P, X, t, g, bound


def test_mlp_error_bound_admits_a_float32_evaluation():
    """The element-wise bound used to compare the tensor-core gradients with
    the oracle holds for another evaluation at the network's precision
    (float32 accumulation, same bf16 roundings), and is tight: far below the
    gradients themselves."""
    for seed in (11, 12):
        P, X, t, g, bound = _bound_case(seed)
        g32 = _f32_grads(P, X, t)
        for k in g:
            d = np.abs(np.asarray(g32[k], np.float64) - g[k])
            assert np.all(d <= bound[k]), (k, float((d - bound[k]).max()))
        rel = np.concatenate([(bound[k] / (np.abs(g[k]) + 1e-30)).ravel() for k in ("W1", "W2", "w3")])
        assert np.median(rel) < 0.05, np.median(rel)


@pytest.mark.parametrize("mistake", ["transposed_W2", "dropped_W1_column", "b1_sign", "no_H2_mask", "sum_not_mean",
                                     "no_b2", "unclipped"])
def test_mlp_error_bound_rejects_planted_mistakes(mistake):
    """A gradient computed with a plausible mistake (planted here, in a copy of
    the oracle's result) falls outside the bound somewhere."""
    P, X, t, g, bound = _bound_case(21)
    bad = {k: np.array(v, dtype=np.float64, copy=True) for k, v in g.items()}
    if mistake == "transposed_W2":
        bad["W2"] = bad["W2"].T
    elif mistake == "dropped_W1_column":
        bad["W1"][:, 17] = 0.0
    elif mistake == "b1_sign":
        bad["b1"] = -bad["b1"]
    elif mistake == "no_H2_mask":
        y, cache = Lr.mlp_forward(X, P, Lr.bf16_round)
        dy = (y - t) / X.shape[0]
        bad["b2"] = np.outer(dy, P["w3"]).sum(0)
    elif mistake == "sum_not_mean":
        bad = {k: v * X.shape[0] for k, v in bad.items()}
    elif mistake == "no_b2":
        P2 = dict(P, b2=np.zeros_like(P["b2"]))
        y, cache = Lr.mlp_forward(X, P2, Lr.bf16_round)
        bad = Lr.mlp_backward(P2, cache, y, t, Lr.bf16_round)
    elif mistake == "unclipped":
        # one SGD step from the same start: clipped (the oracle) vs not
        Pa = {k: np.array(v, dtype=np.float64, copy=True) for k, v in P.items()}
        Pb = {k: np.array(v, dtype=np.float64, copy=True) for k, v in P.items()}
        Va = {k: np.zeros_like(np.asarray(v, dtype=np.float64)) for k, v in P.items()}
        Vb = {k: np.zeros_like(np.asarray(v, dtype=np.float64)) for k, v in P.items()}
        Lr.sgd_momentum(Pa, g, Va, 0.05, 0.9)
        Lr.sgd_momentum(Pb, g, Vb, 0.05, 0.9, clip=None)
        assert any(np.any(np.abs(Pa[k] - Pb[k]) > 0.05 * bound[k] + 1e-12) for k in P)
        return
    assert any(np.any(np.abs(np.asarray(bad[k]) - g[k]) > bound[k]) for k in g), mistake
