"""Concurrent query contexts and the serving engine.

The serving engine admits requests in arrival order, packs consecutive
queries into device batches on several slots at once, and makes insertions
epoch barriers.  Its defining property is tested here: every request's
result is the same as when the requests are replayed one by one.
"""
import threading

import numpy as np
import pytest
import torch

import dbl_inputs
import oracle
import paper_2101_09441_gb300 as dbl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    dbl.build()


def D(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def tiny():
    return dbl_inputs.workload("tiny")


def test_concurrent_contexts(tiny):
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    ix.insert_edges(D(tiny["ins_src"]), D(tiny["ins_dst"]))
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build()
    ref.insert_edges(tiny["ins_src"], tiny["ins_dst"])
    rans, rcode = ref.query(tiny["q_u"], tiny["q_v"], nthreads=8)
    results = {}

    def run(i):
        torch.cuda.set_device(0)
        s = torch.cuda.Stream()
        ctx = dbl.QueryContext(ix, stream=s)
        lo, hi = i * 25_000, (i + 1) * 25_000
        with torch.cuda.stream(s):
            for _ in range(3):
                a, c = ctx.query(D(tiny["q_u"][lo:hi]), D(tiny["q_v"][lo:hi]), stream=s)
            s.synchronize()
            results[i] = (a.cpu().numpy(), c.cpu().numpy())
        ctx.close(stream=s)

    threads = [threading.Thread(target=run, args=(i,)) for i in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for i in range(4):
        lo, hi = i * 25_000, (i + 1) * 25_000
        assert np.array_equal(results[i][0], rans[lo:hi]) and np.array_equal(results[i][1], rcode[lo:hi])


def _request_stream(tiny, n_req, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    e = q = 0
    for _ in range(n_req):
        if rng.random() < 0.1 and e < tiny["ins_src"].shape[0]:
            sz = int(np.exp(rng.uniform(0, np.log(301))))
            reqs.append((1, tiny["ins_src"][e:e + sz], tiny["ins_dst"][e:e + sz]))
            e += sz
        else:
            sz = int(np.exp(rng.uniform(0, np.log(3001))))
            lo = q % 90_000
            reqs.append((0, tiny["q_u"][lo:lo + sz], tiny["q_v"][lo:lo + sz]))
            q += sz
    return reqs


def test_server_mix_equals_serial_replay(tiny):
    reqs = _request_stream(tiny, 400, 11)
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    srv = dbl.Server(ix, slots=4, max_batch=1 << 14)
    tickets = [srv.submit(k, a, b) for k, a, b in reqs]   # all queued at once: maximal overlap
    got = [srv.wait(t)[0] for t in tickets]
    rep = srv.report()
    srv.close()
    assert rep["query_requests"] + rep["insert_requests"] == len(reqs)
    assert rep["device_batches"] < rep["query_requests"]    # requests were packed together
    # the same requests one by one, alone
    alone = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    ref = oracle.OracleIndex(tiny["row_ptr"], tiny["col"], 64, 64).build()
    for (k, a, b), g in zip(reqs, got):
        if k == 1:
            alone.insert_edges(D(a), D(b))
            ref.insert_edges(a, b)
        else:
            exp = alone.query(D(a), D(b))[0].cpu().numpy()
            assert np.array_equal(g, exp)
            assert np.array_equal(g, ref.query(a, b)[0])
    for x, y in zip(ix.labels(), alone.labels()):
        assert torch.equal(x, y)


def test_server_backpressure_and_report(tiny):
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    srv = dbl.Server(ix, slots=2, max_batch=1 << 12, max_pending=8)
    a = tiny["q_u"][:4000]
    b = tiny["q_v"][:4000]
    tickets, busy = [], 0
    for _ in range(200):
        try:
            tickets.append(srv.submit(0, a, b))
        except dbl.DblError as e:
            assert e.status == dbl.DBL_ERR_BUSY
            busy += 1
    for t in tickets:
        srv.wait(t)
    rep = srv.report()
    srv.close()
    assert busy > 0
    assert rep["query_p50_s"] <= rep["query_p99_s"]
    assert rep["pairs"] == 4000 * len(tickets)
    with pytest.raises(dbl.DblError):
        dbl.Server(ix, slots=2, max_batch=1 << 12).submit(0, np.zeros(5000, np.int32), np.zeros(5000, np.int32))


def test_server_cancel_drops_queued_requests(tiny):
    """Requests cancelled before a slot takes them are dropped: their waits
    report DBL_ERR_CANCELLED, a cancelled insertion is never applied, and
    every other result equals a serial replay of the requests that were not
    cancelled."""
    reqs = _request_stream(tiny, 300, 13)
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    srv = dbl.Server(ix, slots=2, max_batch=1 << 12)
    tickets = [srv.submit(k, a, b) for k, a, b in reqs]
    cancelled = {i for i in range(len(reqs) - 1, 0, -3) if srv.cancel(tickets[i])}
    got = {}
    for i, t in enumerate(tickets):
        if i in cancelled:
            with pytest.raises(dbl.DblError) as e:
                srv.wait(t)
            assert e.value.status == dbl.DBL_ERR_CANCELLED
        else:
            got[i] = srv.wait(t)[0]
    with pytest.raises(dbl.DblError) as e:
        srv.cancel(tickets[0])                 # waited for already: an unknown ticket
    assert e.value.status == dbl.DBL_ERR_INVALID
    rep = srv.report()
    srv.close()
    assert cancelled and rep["cancelled"] == len(cancelled)
    assert any(reqs[i][0] == 1 for i in cancelled) or len(cancelled) > 5
    alone = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    for i, (k, a, b) in enumerate(reqs):
        if i in cancelled:
            continue
        if k == 1:
            alone.insert_edges(D(a), D(b))
        else:
            assert np.array_equal(got[i], alone.query(D(a), D(b))[0].cpu().numpy())
    for x, y in zip(ix.labels(), alone.labels()):
        assert torch.equal(x, y)


def test_server_admits_slots_by_free_memory(tiny):
    """A slot's scratch is allocated only when it then fits the device's free
    memory (mem_fraction) and the server's byte budget (max_memory): with a
    budget of one slot the server runs on that slot alone, with a generous
    one more slots are admitted under load.  Results equal a serial replay."""
    reqs = _request_stream(tiny, 200, 17)
    ix = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    probe = dbl.Server(ix, slots=1, max_batch=1 << 14)
    per_slot = int(probe.report()["bytes_per_slot"])
    probe.close()
    with pytest.raises(dbl.DblError) as e:
        dbl.Server(ix, slots=2, max_batch=1 << 14, max_memory=per_slot // 2)   # not even one slot
    assert e.value.status == dbl.DBL_ERR_OOM
    got = {}
    for name, budget in (("one", per_slot * 3 // 2), ("many", 0)):
        ix2 = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
        srv = dbl.Server(ix2, slots=4, max_batch=1 << 14, mem_fraction=0.9, max_memory=budget)
        tickets = [srv.submit(k, a, b) for k, a, b in reqs]
        got[name] = [srv.wait(t)[0] for t in tickets]
        rep = srv.report()
        srv.close()
        ix2.close()
        if name == "one":
            assert rep["slots_admitted"] == 1
        else:
            assert rep["slots_admitted"] >= 2
    alone = dbl.DBLIndex(D(tiny["row_ptr"]), D(tiny["col"]), 64, 64)
    for i, (k, a, b) in enumerate(reqs):
        if k == 1:
            alone.insert_edges(D(a), D(b))
        else:
            exp = alone.query(D(a), D(b))[0].cpu().numpy()
            assert np.array_equal(got["one"][i], exp) and np.array_equal(got["many"][i], exp)
