"""dbl_insert_edges_noalloc: insertion for callers that cannot allocate device
memory (their memory is fully handed to their own pool, or they must not wait
on an allocator).  Called through the C ABI and compared with the allocating
dbl_insert_edges on two calls in a row; labels are integer bitsets, so the
comparison is exact.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import dbl_inputs
import paper_2101_09441_gb300 as dbl

pytestmark = pytest.mark.gpu

MAX_BATCH = 1 << 20


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _labels(ix):
    return [t.cpu().numpy().view(np.uint64) for t in ix.labels()]


@pytest.mark.parametrize("flags", [0, dbl.FLAG_PERSISTENT, dbl.FLAG_PERSISTENT | dbl.FLAG_ASYNC])
def test_noalloc_insert_matches_allocating_insert(flags):
    """Level-by-level kernels, and the persistent insertion kernel (which keeps
    its per-edge slot words in the same scratch), synchronous and not."""
    dbl.build()
    w = dbl_inputs.workload("tiny", with_queries=False)
    rp, col = _dev(w["row_ptr"]), _dev(w["col"])
    a = dbl.DBLIndex(rp, col, 64, 64, flags=flags)   # allocating entry point
    b = dbl.DBLIndex(rp, col, 64, 64, flags=flags)   # allocation-free entry point
    L = dbl.lib()
    s = torch.cuda.current_stream().cuda_stream
    src, dst = _dev(w["ins_src"]), _dev(w["ins_dst"])
    for lo, hi in ((0, 4000), (4000, 10_000)):            # two calls in a row
        a.insert_edges(src[lo:hi], dst[lo:hi])
        st = L.dbl_insert_edges_noalloc(ctypes.c_void_p(b._h.value), ctypes.c_void_p(src[lo:hi].data_ptr()),
                                        ctypes.c_void_p(dst[lo:hi].data_ptr()), hi - lo, ctypes.c_void_p(s))
        assert st == dbl.DBL_OK, L.dbl_last_error(b._h).decode()
        a.sync()
        b.sync()
        torch.cuda.synchronize()
        for x, y in zip(_labels(a), _labels(b)):
            assert np.array_equal(x, y)
        assert a.info()["edges_stored"] == b.info()["edges_stored"] == hi
    qu = _dev(np.arange(0, 16380, 3, dtype=np.int32))
    qv = _dev(np.arange(1, 16381, 3, dtype=np.int32))
    ra, ca = a.query(qu, qv)
    rb, cb = b.query(qu, qv)
    a.sync()
    b.sync()
    assert torch.equal(ra, rb) and torch.equal(ca, cb)


def test_noalloc_rejects_oversized_batch():
    dbl.build()
    w = dbl_inputs.workload("tiny", with_queries=False)
    ix = dbl.DBLIndex(_dev(w["row_ptr"]), _dev(w["col"]), 64, 64, edge_capacity=MAX_BATCH + 16)
    big = torch.zeros(MAX_BATCH + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(dbl.DblError) as e:
        ix.insert_edges_noalloc(big, big)
    assert e.value.status == dbl.DBL_ERR_INVALID
    assert "maximum" in str(e.value)
    assert ix.info()["edges_stored"] == 0
