"""Learned landmark scorer on the GPU vs its fp64 oracle (oracle/learned.py).

Integer outputs (coverage counts, selections) must match exactly; bf16
features within one bf16 rounding; network outputs, gradients, losses and
the parameters after training steps element by element, within a bound
carried through the network from its arithmetic (bf16 storage, fp32
accumulation; tests/helpers.py mlp_error_bound) against the oracle evaluated
at the same storage precision.
"""
import numpy as np
import pytest
import torch

import dbl_inputs
import oracle
import paper_2101_09441_gb300 as dbl
from oracle import learned as Lr
from paper_2101_09441_gb300 import learned as L
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    dbl.build()


def D(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def tiny():
    return dbl_inputs.workload("tiny")


def test_features_match_oracle(tiny):
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build()
    got = ix.features().float().cpu().numpy()
    exp = Lr.features(tiny["row_ptr"], tiny["col"], ref.labels(), ref.landmarks)
    assert np.allclose(got, exp, rtol=2 ** -7, atol=1e-6), np.abs(got - exp).max()


def test_coverage_matches_oracle(tiny):
    rp, col = tiny["row_ptr"], tiny["col"]
    ix = dbl.DBLIndex(D(rp), D(col), 64, 64)
    ref = oracle.OracleIndex(rp, col, 64, 64).build()
    qu, qv = tiny["q_u"][:1200], tiny["q_v"][:1200]
    ans, _ = ref.query(qu, qv)
    # all reachable pairs (u != v), several passes of 256
    keep = (ans == 1) & (qu != qv)
    cnt, tgt, kept = ix.coverage(D(qu), D(qv), reach=D(keep.astype(np.uint8)), base_slots=0)
    exp = Lr.coverage(rp, col, qu[keep], qv[keep])
    assert kept == int(keep.sum())
    assert np.array_equal(cnt.cpu().numpy(), exp)
    t = tgt.cpu().numpy()
    assert np.allclose(t, np.log1p(exp) / np.log1p(exp.max()), rtol=1e-6, atol=1e-6)
    # pairs the first 8 landmark slots already decide are left out
    dl_in, dl_out, _, _ = ref.labels()
    mask = np.uint64(0xFF)
    decided = ((dl_out[qu, 0] & dl_in[qv, 0] & mask) != 0)
    keep2 = keep & ~decided
    cnt2, _, kept2 = ix.coverage(D(qu), D(qv), reach=D(keep.astype(np.uint8)), base_slots=8)
    assert kept2 == int(keep2.sum())
    assert np.array_equal(cnt2.cpu().numpy(), Lr.coverage(rp, col, qu[keep2], qv[keep2]))


def test_select_by_score_ties_by_id(tiny):
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    rng = np.random.default_rng(4)
    sc = rng.integers(-50, 50, ix.n).astype(np.float32) / 4   # many ties, negatives
    got = ix.select_by_score(D(sc), 100).cpu().numpy()
    exp = np.lexsort((np.arange(ix.n), -sc))[:100]
    assert np.array_equal(got, exp)


def _spread_reference(rp, col, sc, k):
    """The greedy spread selection written out: k times, the untaken,
    unexcluded vertex of largest score (smaller id on ties; -inf and NaN never),
    then its in- and out-neighbours are excluded."""
    n = rp.shape[0] - 1
    ok = np.isfinite(sc) | (sc == np.inf)
    order = np.lexsort((np.arange(n), -np.where(ok, sc, 0)))
    order = order[ok[order]]
    ins = [[] for _ in range(n)]
    for u in range(n):
        for x in col[rp[u]:rp[u + 1]]:
            ins[x].append(u)
    gone = np.zeros(n, bool)
    out, pos = [], 0
    while len(out) < k:
        while pos < len(order) and gone[order[pos]]:
            pos += 1
        if pos == len(order):
            out.append(-1)
            continue
        x = int(order[pos])
        out.append(x)
        gone[x] = True
        gone[col[rp[x]:rp[x + 1]]] = True
        gone[ins[x]] = True
    return np.array(out, dtype=np.int32)


def test_select_spread_matches_greedy(tiny):
    rp, col = tiny["row_ptr"], tiny["col"]
    ix = dbl.DBLIndex(D(rp), D(col), 64, 64)
    rng = np.random.default_rng(6)
    sc = rng.integers(-40, 40, ix.n).astype(np.float32) / 4   # ties
    sc[rng.integers(0, ix.n, 500)] = -np.inf
    sc[rng.integers(0, ix.n, 50)] = np.nan
    got = ix.select_spread(D(sc), 60).cpu().numpy()
    assert np.array_equal(got, _spread_reference(rp, col, sc, 60))
    # fewer candidates than slots: the rest are -1
    sc2 = np.full(ix.n, -np.inf, np.float32)
    sc2[[5, 77, 1000]] = [1.0, 3.0, 2.0]
    got2 = ix.select_spread(D(sc2), 6).cpu().numpy()
    assert np.array_equal(got2, _spread_reference(rp, col, sc2, 6))
    assert (got2[3:] == -1).all()


@pytest.mark.parametrize("spread", [False, True])
def test_select_uncovered_matches_greedy(tiny, spread):
    """dbl_select_uncovered: the greedy selection over the vertices outside the
    strongly connected components of the first 8 landmarks (DL_in and DL_out
    sharing one of their bits), written out here from the labels."""
    rp, col = tiny["row_ptr"], tiny["col"]
    ix = dbl.DBLIndex(D(rp), D(col), 64, 64)
    rng = np.random.default_rng(8)
    sc = rng.integers(-40, 40, ix.n).astype(np.float32) / 4
    sc[rng.integers(0, ix.n, 300)] = -np.inf
    dl_in, dl_out = (t.cpu().numpy().view(np.uint64)[:, 0] for t in ix.labels()[:2])
    slots = 8
    covered = (dl_in & dl_out & np.uint64((1 << slots) - 1)) != 0
    lm = ix.selection()[0].cpu().numpy()
    assert covered[lm[:slots]].all()                 # a landmark is in its own component
    assert covered.sum() > slots                      # the giant component is covered
    ref_sc = np.where(covered, -np.inf, sc).astype(np.float32)
    if spread:
        exp = _spread_reference(rp, col, ref_sc, 60)
    else:
        cand = np.flatnonzero(np.isfinite(ref_sc))
        order = cand[np.lexsort((cand, -ref_sc[cand]))][:60]
        exp = np.concatenate([order, -np.ones(60 - len(order), np.int64)]).astype(np.int32)
    got = ix.select_uncovered(D(sc), 60, slots, spread=spread).cpu().numpy()
    assert np.array_equal(got, exp)
    assert not covered[got[got >= 0]].any()


def test_learned_rounds_gain_on_community_graph():
    """Communities of power-law sizes joined by edges from earlier to later
    ones: the degree rule's landmarks all sit in the largest community's
    strongly connected component.  The learned selection (8 degree landmarks
    kept, 56 scored vertices outside the kept landmarks' components, in 7
    rounds) decides more held-out pairs by the DL test and sends fewer to the
    search than the degree rule, is kept by the judge, and answers the same."""
    rp, col = dbl_inputs.community_dag(200_000, 2_000_000, 64, 1.0, 0.02, 5)
    qu, qv = dbl_inputs.queries(rp, col, 200_000, 11, False)
    tq, ev = (D(qu[:100_000]), D(qv[:100_000])), (D(qu[100_000:]), D(qv[100_000:]))
    plain, chosen, learned, info = L.learned_index(D(rp), D(col), tq, ev, k=64, kprime=64, rounds=7, steps=300)
    dp, dl = info["eval_plain"], info["eval_learned"]
    assert not info["fallback"], info
    # (training uses fp32 atomics, so the picks vary a little from run to run:
    # 45,700-47,700 decided by DL against 42,275, 17,300-17,800 searched against 23,592)
    assert dl["dl"] > 1.05 * dp["dl"] and dl["search"] < 0.9 * dp["search"], info
    a_p, _ = plain.query(*ev)
    a_l, _ = learned.query(*ev)
    assert torch.equal(a_p, a_l)


def _quantised_params(seed):
    p = dbl.MLP.init_params(seed)
    p[2048:2176] = np.random.default_rng(seed).normal(0, 0.05, 128)     # non-zero biases
    p[18560:18688] = np.random.default_rng(seed + 1).normal(0, 0.05, 128)
    p[18816] = 0.1
    return p


def _split(p):
    q = p.astype(np.float64)
    return {"W1": q[0:2048].reshape(16, 128), "b1": q[2048:2176], "W2": q[2176:18560].reshape(128, 128),
            "b2": q[18560:18688], "w3": q[18688:18816], "b3": np.array(q[18816])}


def test_mlp_forward_matches_oracle():
    p = _quantised_params(3)
    m = dbl.MLP(p)
    rng = np.random.default_rng(5)
    X = rng.normal(0.5, 1.0, (1000, 16)).astype(np.float32)
    Xb = torch.from_numpy(X).to(torch.bfloat16).cuda()
    y = m.forward(Xb).cpu().numpy()
    P = _split(p)
    for k in ("W1", "W2"):
        P[k] = bf16_round(P[k])
    Xq = bf16_round(X)
    yo, _ = Lr.mlp_forward(Xq, P, Lr.bf16_round)
    _, ey, _ = H.mlp_error_bound(P, Xq, np.zeros(Xq.shape[0]))
    assert np.all(np.abs(y - yo) <= ey), float((np.abs(y - yo) - ey).max())
    # row gather gives the same rows
    idx = torch.from_numpy(np.array([5, 999, 0, 5], np.int32)).cuda()
    yi = m.forward(Xb, rows_idx=idx).cpu().numpy()
    assert np.allclose(yi, y[[5, 999, 0, 5]], rtol=0, atol=0)


def _oracle_grads(P, X, t):
    """Oracle gradients and loss of the network at its storage precision
    (bf16 weights, features and activations; fp64 otherwise), with the
    element-wise bound on the tensor-core result (tests/helpers.py)."""
    y, cache = Lr.mlp_forward(X, P, Lr.bf16_round)
    g = Lr.mlp_backward(P, cache, y, t, Lr.bf16_round)
    return g, Lr.mlp_loss(y, t)


def _bf16_weights(P):
    Q = {k: np.array(v, dtype=np.float64, copy=True) for k, v in P.items()}
    for k in ("W1", "W2"):
        Q[k] = bf16_round(Q[k])
    return Q


def _check_elementwise(got_flat, want, bound, what):
    got = H.mlp_unflat(got_flat)
    for name, _, _, _ in H.MLP_BLOCKS:
        d = np.abs(np.asarray(got[name]) - np.asarray(want[name]))
        bad = d > bound[name]
        assert not np.any(bad), (what, name, int(bad.sum()), float((d - bound[name]).max()))


@pytest.mark.parametrize("gather", [False, True])
def test_mlp_gradients_match_oracle(gather):
    """Every gradient element of the tensor-core backward pass against the
    fp64 oracle at the network's precision, within the element-wise bound
    carried through the pass from fp32 accumulation and bf16 rounding
    (tests/helpers.py); the loss likewise.  Targets sit away from the outputs
    so that the residuals are not cancellations."""
    p = _quantised_params(6)
    m = dbl.MLP(p)
    rng = np.random.default_rng(7)
    R = 3000
    X = bf16_round(rng.normal(0.5, 1.0, (R, 16)))
    t = rng.normal(3.0, 0.5, R).astype(np.float32)
    Xb = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).cuda()
    idx = rng.integers(0, R, 2500).astype(np.int32) if gather else None
    rows = idx if gather else np.arange(R)
    g, loss = m.gradients(Xb, D(t), rows_idx=D(idx) if gather else None)
    P = _bf16_weights(H.mlp_unflat(p))
    want, loss_ref = _oracle_grads(P, X[rows], t[rows].astype(np.float64))
    bound, _, eloss = H.mlp_error_bound(P, X[rows], t[rows].astype(np.float64))
    _check_elementwise(g.cpu().numpy().astype(np.float64), want, bound, "gradients")
    assert abs(float(loss.item()) - loss_ref) <= eloss + 1e-6 * loss_ref


def test_mlp_train_step_matches_oracle():
    """Two training steps (momentum SGD on element-wise clipped gradients):
    every parameter after each step against the oracle's step, within the
    bound the gradient bound gives (lr times it, plus fp32 rounding of the
    update; for the second step the weights' bf16 copies may round to a
    neighbouring value where the first step left them within its bound of a
    rounding boundary)."""
    p0 = _quantised_params(11)
    m = dbl.MLP(p0)
    rng = np.random.default_rng(12)
    R, lr, mu = 4000, 0.05, 0.9
    X = bf16_round(rng.normal(0.5, 1.0, (R, 16)))
    t = rng.normal(3.0, 0.5, R).astype(np.float32)
    Xb = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).cuda()
    td = D(t)
    P = H.mlp_unflat(p0.astype(np.float32))
    V = {k: np.zeros_like(v) for k, v in P.items()}
    eP = {k: np.zeros_like(v) for k, v in P.items()}
    eV = {k: np.zeros_like(v) for k, v in P.items()}
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    clipped = 0
    for step in range(2):
        idx = rng.integers(0, R, 3000).astype(np.int32)
        m.train_step(Xb, td, D(idx), lr=lr, momentum=mu, loss=loss)
        got = m.params().astype(np.float64)
        # oracle step from its own parameters; the GPU's bf16 weight copies are
        # within bf16_weight_radius of the oracle's
        Pq = _bf16_weights(P)
        eq = {k: (H.bf16_weight_radius(P[k], eP[k]) if k in ("W1", "W2") else eP[k]) for k in P}
        g, loss_ref = _oracle_grads(Pq, X[idx], t[idx].astype(np.float64))
        bound, _, eloss = H.mlp_error_bound(Pq, X[idx], t[idx].astype(np.float64), eq)
        assert abs(float(loss.item()) - loss_ref) <= eloss + 1e-6 * loss_ref, step
        clipped += sum(int((np.abs(np.asarray(g[k])) > Lr.CLIP).sum()) for k in g)
        Lr.sgd_momentum(P, g, V, lr, mu)
        for k in P:
            eV[k] = mu * eV[k] + bound[k] + H.FP32_U * np.abs(V[k])
            eP[k] = eP[k] + lr * eV[k] + H.FP32_U * (np.abs(P[k]) + lr * np.abs(V[k]))
        _check_elementwise(got, P, eP, f"parameters after step {step + 1}")
    assert clipped > 0  # the clip is exercised
    m.close()


def test_mlp_training_reduces_loss():
    rng = np.random.default_rng(8)
    R = 20000
    X = rng.normal(0, 1, (R, 16)).astype(np.float32)
    t = (np.maximum(X[:, 0], 0) + 0.5 * X[:, 3] * X[:, 4] > 0.3).astype(np.float32)
    Xb = torch.from_numpy(X).to(torch.bfloat16).cuda()
    td = D(t)
    m = dbl.MLP(dbl.MLP.init_params(9))
    _, l0 = m.gradients(Xb, td)
    l0 = float(l0.item())
    loss = torch.zeros(1, device="cuda")
    for _ in range(300):
        idx = torch.randint(0, R, (4096,), device="cuda", dtype=torch.int32)
        m.train_step(Xb, td, idx, lr=0.05, momentum=0.9, loss=loss)
    _, l1 = m.gradients(Xb, td)
    assert float(l1.item()) < 0.5 * l0


def test_learned_landmarks_exact_and_better_or_fallback(tiny):
    """Learned landmarks (trained on the index after the 10k insertions) give
    exact answers, and the chosen set decides at least as many held-out pairs
    by the DL test as the degree rule (else the degree rule is kept)."""
    rp, col = D(tiny["row_ptr"]), D(tiny["col"])
    qu, qv = D(tiny["q_u"]), D(tiny["q_v"])
    ins = [(D(tiny["ins_src"]), D(tiny["ins_dst"]))]
    plain, chosen, learned, info = L.learned_index(rp, col, (qu[:50_000], qv[:50_000]), (qu[50_000:], qv[50_000:]),
                                                   k=64, kprime=64, inserts=ins, steps=300)
    print("learned scorer:", info)
    assert all(np.isfinite(info["losses"]))
    lm = learned.selection()[0].cpu().numpy()
    assert len(set(lm[lm >= 0].tolist())) == int((lm >= 0).sum())          # distinct landmarks
    # exact: answers equal the oracle's with the learned landmark set
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build(
        lm, *[t.cpu().numpy() for t in plain.selection()[1:]])
    ref.insert_edges(tiny["ins_src"], tiny["ins_dst"])
    a, c = learned.query(qu, qv)
    ra, rc = ref.query(tiny["q_u"], tiny["q_v"], nthreads=8)
    assert np.array_equal(a.cpu().numpy(), ra) and np.array_equal(c.cpu().numpy(), rc)
    assert np.array_equal(a.cpu().numpy(), plain.query(qu, qv)[0].cpu().numpy())
    dl_p, dl_c = L.decided(plain, qu[50_000:], qv[50_000:]), L.decided(chosen, qu[50_000:], qv[50_000:])
    assert dl_c["dl"] >= dl_p["dl"]
    # a kept learned set does not make the insertions' label repair much dearer
    assert info["fallback"] or L.repair_ok(info["repair_plain"], info["repair_learned"])
