"""Learned landmark selection on top of the C ABI (orchestration only).

The degree rule of the paper (Section 4.1) puts every landmark of an R-MAT or
social graph into its giant strongly connected component, where one landmark
already decides every pair routed through that component (Theorem 2's
argument): the others add little to the DL test.  Here the first
`base_slots` degree landmarks are kept and the remaining slots go to the
vertices a network scores highest; the network is trained on how many of the
sampled reachable pairs the kept landmarks leave undecided each vertex would
decide (dbl_coverage).  No pick lies in the strongly connected component of
a kept landmark (such a vertex decides nothing the landmark does not).  In
rounds (select_in_rounds) the landmarks taken so far join the kept ones
before the next round's training, so that a round's picks are scored on the
pairs the earlier picks leave undecided.  The learned
set is compared with the degree rule on held-out pairs and the degree rule is
kept when the learned set is not better (the fallback).  Answers are exact for
any landmark set.

Every computation runs in the library's kernels (queries, coverage, features,
tensor-core training, selection); this module only draws the random
mini-batch indices (seeded) and moves tensors between calls.
"""
from __future__ import annotations

import time

import numpy as np

from . import CODE_BFS_NEG, CODE_BFS_POS, CODE_DL, MLP, DBLIndex


def train_scorer(ix: DBLIndex, qu, qv, base_slots: int, steps: int = 400, batch: int = 8192, lr: float = 0.01,
                 momentum: float = 0.9, seed: int = 7, mlp: MLP | None = None):
    """Train the scorer on the index's outcomes for the sampled pairs (qu, qv)
    (a new network, or `mlp` trained further).

    Returns (scores float32 [n], info)."""
    import torch
    t0 = time.perf_counter()
    ans, _ = ix.query(qu, qv)                                     # outcomes of the plain index
    count, target, kept = ix.coverage(qu, qv, reach=ans, base_slots=base_slots)
    feats = ix.features()
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    gen = torch.Generator(device=feats.device)
    gen.manual_seed(seed)
    pos = torch.nonzero(count > 0).flatten().to(torch.int32)
    n = ix.n
    own = mlp is None
    if own:
        mlp = MLP(MLP.init_params(seed))
    loss = torch.zeros(1, dtype=torch.float32, device=feats.device)
    losses = []
    half = batch // 2
    for step in range(steps):
        if pos.numel():
            a = pos[torch.randint(0, pos.numel(), (half,), device=feats.device, generator=gen)]
        else:
            a = torch.randint(0, n, (half,), device=feats.device, generator=gen, dtype=torch.int32)
        b = torch.randint(0, n, (batch - half,), device=feats.device, generator=gen, dtype=torch.int32)
        idx = torch.cat([a, b]).to(torch.int32)
        mlp.train_step(feats, target, idx, lr=lr, momentum=momentum, loss=loss)
        if step % 50 == 0 or step == steps - 1:
            losses.append(float(loss.item()))
    scores = mlp.forward(feats)
    torch.cuda.synchronize()
    info = dict(pairs=int(qu.numel()), pairs_kept=kept, positive_vertices=int(pos.numel()), losses=losses,
                data_s=t_data, train_s=time.perf_counter() - t0 - t_data)
    if own:
        mlp.close()
    return scores, info


def _pick(ix: DBLIndex, scores, exclude, take: int, spread: bool, covered_slots: int = 0):
    """`take` vertices by score (spread: each excludes its neighbours from later
    picks), none of `exclude` and none in the strongly connected component of
    one of ix's first `covered_slots` landmarks (dbl_select_uncovered)."""
    import torch
    sc = torch.nan_to_num(scores.clone(), nan=float("-inf"))
    ex = exclude[exclude >= 0].long()
    sc[ex] = float("-inf")
    out = ix.select_uncovered(sc, take, covered_slots, spread=spread)
    return out[out >= 0]


def select_landmarks(ix: DBLIndex, scores, k: int, base_slots: int, spread: bool = False):
    """First `base_slots` degree landmarks of ix, then the best-scored others
    (spread: each pick excludes its in- and out-neighbours from later picks,
    dbl_select_spread)."""
    import torch
    lm_deg = ix.selection()[0]
    base = lm_deg[:base_slots]
    rest = _pick(ix, scores, base, k - base_slots, spread, covered_slots=base_slots)
    return _fill(torch.cat([base, rest]).to(torch.int32), lm_deg, k)


def _fill(chosen, lm_deg, k: int):
    """chosen, then degree landmarks not in it, up to k slots."""
    import torch
    if chosen.numel() >= k:
        return chosen[:k].to(torch.int32)
    taken = torch.isin(lm_deg, chosen)
    return torch.cat([chosen, lm_deg[~taken][: k - chosen.numel()]]).to(torch.int32)


def select_in_rounds(plain: DBLIndex, row_ptr, col, train_q, k: int, kprime: int, base_slots: int, rounds: int,
                     spread: bool = False, idx_kw: dict | None = None, inserts=None, **train_kw):
    """Greedy learned selection: after the first `base_slots` degree landmarks,
    `rounds` rounds each take about (k - base_slots) / rounds vertices by the
    scorer's output, and before every round but the first the index is rebuilt
    with the landmarks taken so far in its first slots, so that the coverage
    the scorer is trained on counts only the pairs those landmarks leave
    undecided (a set of top-scored vertices from one strongly connected
    component decides what one of them would).  One network is trained
    further in every round.  A rebuilt index applies `inserts` (the batches
    plain has applied).  Returns (landmarks int32 [k], info)."""
    import torch
    idx_kw = idx_kw or {}
    lm_deg, lb, lr_ = plain.selection()
    chosen = lm_deg[:base_slots]
    per = -(-(k - base_slots) // rounds)
    steps = int(train_kw.pop("steps", 400))
    seed = int(train_kw.get("seed", 7))
    mlp = MLP(MLP.init_params(seed))
    cur, infos = plain, []
    try:
        for r in range(rounds):
            scores, info = train_scorer(cur, train_q[0], train_q[1], int(chosen.numel()), mlp=mlp,
                                        steps=steps if r == 0 else max(1, steps // 2), **train_kw)
            infos.append(info)
            take = min(per, k - int(chosen.numel()))
            chosen = torch.cat([chosen, _pick(cur, scores, chosen, take, spread,
                                              covered_slots=int(chosen.numel()))]).to(torch.int32)
            if cur is not plain:
                cur.close()
            cur = plain
            if chosen.numel() >= k or r == rounds - 1:
                break
            cur = DBLIndex(row_ptr, col, k, kprime, landmarks=_fill(chosen, lm_deg, k), leaf_buckets=lb,
                           leaf_roles=lr_, **idx_kw)
            for s_, d_ in inserts or []:
                cur.insert_edges(s_, d_)
    finally:
        if cur is not plain:
            cur.close()
        mlp.close()
    info = dict(rounds=len(infos), pairs=infos[0]["pairs"], pairs_kept=[i["pairs_kept"] for i in infos],
                positive_vertices=[i["positive_vertices"] for i in infos], losses=infos[-1]["losses"],
                data_s=sum(i["data_s"] for i in infos), train_s=sum(i["train_s"] for i in infos))
    return _fill(chosen, lm_deg, k), info


def decided(ix: DBLIndex, qu, qv) -> dict:
    """How the index decides the pairs: counts of DL, search and other rules."""
    _, code = ix.query(qu, qv)
    c = code.long()
    return dict(dl=int((c == CODE_DL).sum()), search=int(((c == CODE_BFS_POS) | (c == CODE_BFS_NEG)).sum()),
                total=int(c.numel()))


REPAIR_SLACK = 1.5


def repair_ok(repair_plain: int, repair_learned: int) -> bool:
    """The learned landmarks' insertion repair (edges relaxed) stays within
    REPAIR_SLACK of the degree rule's (plus a small absolute allowance)."""
    return repair_learned <= REPAIR_SLACK * repair_plain + 10_000


def learned_index(row_ptr, col, train_q, eval_q, k: int = 64, kprime: int = 64, base_slots: int | None = None,
                  inserts=None, spread: bool = False, rounds: int = 1, **kw):
    """Build the plain index (after `inserts`, a list of (src, dst) batches),
    train the scorer on the plain index's outcomes for train_q = (u, v) (in
    `rounds` rounds: select_in_rounds), build the learned index with the same
    leaves and insertions, and keep the learned set only if it decides more of
    eval_q = (u, v) by the DL test, sends no more of them to the search, and
    does not make the insertions' label repair much dearer (edges relaxed at
    most REPAIR_SLACK times the degree rule's): landmarks whose reach grows
    under insertions make every batch push their bits to millions of
    vertices.  Otherwise the degree rule is kept.  Returns (plain, chosen,
    learned, info)."""
    idx_kw = {a: b for a, b in kw.items() if a in ("flags", "team", "edge_capacity")}
    train_kw = {a: b for a, b in kw.items() if a in ("steps", "batch", "lr", "momentum", "seed")}
    plain = DBLIndex(row_ptr, col, k, kprime, **idx_kw)
    r0 = int(plain.stats()[10])
    for s, d in inserts or []:
        plain.insert_edges(s, d)
    repair_plain = int(plain.stats()[10]) - r0
    if base_slots is None:
        base_slots = max(1, k // 8)
    if rounds > 1:
        lm, info = select_in_rounds(plain, row_ptr, col, train_q, k, kprime, base_slots, rounds, spread=spread,
                                    idx_kw=idx_kw, inserts=inserts, **train_kw)
    else:
        scores, info = train_scorer(plain, train_q[0], train_q[1], base_slots, **train_kw)
        lm = select_landmarks(plain, scores, k, base_slots, spread=spread)
    _, lb, lr_ = plain.selection()
    learned = DBLIndex(row_ptr, col, k, kprime, landmarks=lm, leaf_buckets=lb, leaf_roles=lr_, **idx_kw)
    r0 = int(learned.stats()[10])
    for s, d in inserts or []:
        learned.insert_edges(s, d)
    repair_learned = int(learned.stats()[10]) - r0
    dp = decided(plain, *eval_q)
    dlrn = decided(learned, *eval_q)
    info.update(base_slots=base_slots, eval_plain=dp, eval_learned=dlrn, repair_plain=repair_plain,
                repair_learned=repair_learned,
                fallback=not (dlrn["dl"] > dp["dl"] and dlrn["search"] <= dp["search"]
                              and repair_ok(repair_plain, repair_learned)))
    return plain, (plain if info["fallback"] else learned), learned, info
