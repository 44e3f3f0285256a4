"""Failure detection without a GPU fault.

Every failure here is made on the host or by a bounded wait that runs out:
- a grid barrier whose wait gives up because one block never arrives (a
  short, run-time poll limit): DBL_ERR_TIMEOUT, the index poisoned until
  dbl_restore, and the barrier words usable again afterwards;
- an allocator callback that returns NULL: DBL_ERR_OOM with the index
  unchanged, and the same call succeeding once memory is given again.
Labels and answers are checked against the oracle after each recovery.
"""
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
    dbl_inputs.build()
    oracle.build()


@pytest.fixture(scope="module")
def tiny():
    return dbl_inputs.workload("tiny")


def D(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def labels_np(ix):
    return [t.cpu().numpy().view(np.uint64) for t in ix.labels()]


def same_as_oracle(ix, ref, qu, qv, what):
    for a, b, name in zip(labels_np(ix), ref.labels(), ("dl_in", "dl_out", "bl_in", "bl_out")):
        assert np.array_equal(a, b), f"{what}: {name}"
    ans, code = ix.query(D(qu), D(qv))
    rans, rcode = ref.query(qu, qv, nthreads=8)
    assert np.array_equal(ans.cpu().numpy(), rans) and np.array_equal(code.cpu().numpy(), rcode), what


def test_barrier_wait_runs_out_then_restore_recovers(tiny):
    rp, col = tiny["row_ptr"], tiny["col"]
    s, d = tiny["ins_src"], tiny["ins_dst"]
    ix = dbl.DBLIndex(D(rp), D(col), 64, 64, flags=dbl.FLAG_PERSISTENT)
    ix.snapshot(0)
    ix.barrier_probe(spin_limit=1 << 20, absent_block=-1)      # every block arrives: no error
    with pytest.raises(dbl.DblError) as e:
        ix.barrier_probe(spin_limit=2000, absent_block=3)       # block 3 never arrives
    assert e.value.status == dbl.DBL_ERR_TIMEOUT
    with pytest.raises(dbl.DblError) as e:
        ix.insert_edges(D(s[:100]), D(d[:100]))
    assert e.value.status == dbl.DBL_ERR_POISONED
    ix.restore(0)
    # the persistent insertion uses the same barrier words: they were reset
    ix.insert_edges(D(s), D(d))
    ref = oracle.OracleIndex(rp, col, 64, 64).build()
    ref.insert_edges(s, d)
    same_as_oracle(ix, ref, tiny["q_u"][:20000], tiny["q_v"][:20000], "after the timeout and restore")
    with pytest.raises(dbl.DblError) as e:
        ix.barrier_probe(spin_limit=0)
    assert e.value.status == dbl.DBL_ERR_INVALID
    ix.close()


@pytest.mark.parametrize("flags", [0, dbl.FLAG_PERSISTENT])
def test_allocator_failure_leaves_the_index_unchanged(tiny, flags):
    rp, col = tiny["row_ptr"], tiny["col"]
    s, d = dbl_inputs.insertions(rp, col, 90_000, 77)   # larger than the first scratch size (2^16 edges)
    ix = dbl.DBLIndex(D(rp), D(col), 64, 64, flags=flags, edge_capacity=1 << 18)
    ref = oracle.OracleIndex(rp, col, 64, 64).build()
    ix.insert_edges(D(s[:1000]), D(d[:1000]))
    ref.insert_edges(s[:1000], d[:1000])
    before = labels_np(ix)
    ix.fail_allocations(1)                               # the scratch for the larger batch is refused
    with pytest.raises(dbl.DblError) as e:
        ix.insert_edges(D(s[1000:]), D(d[1000:]))
    assert e.value.status == dbl.DBL_ERR_OOM
    for a, b in zip(labels_np(ix), before):
        assert np.array_equal(a, b)
    ix.insert_edges(D(s[1000:2000]), D(d[1000:2000]))    # smaller batches still run after the failure
    ref.insert_edges(s[1000:2000], d[1000:2000])
    ix.insert_edges(D(s[2000:]), D(d[2000:]))            # and the large one once memory is given
    ref.insert_edges(s[2000:], d[2000:])
    same_as_oracle(ix, ref, tiny["q_u"][:20000], tiny["q_v"][:20000], "after the refused allocation")
    # a snapshot into a new slot that gets only part of its memory (the
    # labels' copy, not the metadata's): nothing is kept, the next one works
    ix.fail_allocations(1, after=1)
    with pytest.raises(dbl.DblError) as e:
        ix.snapshot(2)
    assert e.value.status == dbl.DBL_ERR_OOM
    with pytest.raises(dbl.DblError):
        ix.restore(2)                                     # no snapshot was made
    ix.snapshot(2)
    ix.insert_edges(D(s[:10]), D(d[:10]))                # duplicates: labels unchanged
    ix.restore(2)
    same_as_oracle(ix, ref, tiny["q_u"][:5000], tiny["q_v"][:5000], "after a refused snapshot")
    ix.close()
