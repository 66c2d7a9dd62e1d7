"""Pipelined counts reads (GPU): a caller that steps, queues the read of that
step's counts and collects the previous step's gets, at every step, exactly
the counts a synchronous read gives; the oracle's at the end.  Misuse of the
slots is refused without failing the handle."""
import numpy as np
import pytest

import workloads as W
from gpu_common import engine, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    require_gpu()
    return engine()


def test_pipelined_counts_equal_synchronous_reads(A, oracle_mod):
    m, seed, steps = W.mapk(30_000), 5, 40
    a, b = A.Sim(m, seed), A.Sim(m, seed)
    got, want = [], []
    for k in range(steps):
        a.step(1)
        a.counts_begin(k % 2)
        if k:
            got.append(a.counts_finish((k - 1) % 2))
        b.step(1)
        want.append(b.counts())
    got.append(a.counts_finish((steps - 1) % 2))
    assert len(got) == steps
    for k in range(steps):
        assert np.array_equal(got[k], want[k]), f"step {k + 1}"
    o = oracle_mod.OracleSim(m, seed)
    o.step(steps)
    assert np.array_equal(got[-1], o.counts())
    o.close()
    a.close()
    b.close()


def test_pipelined_counts_in_a_batch(A):
    sims = [(W.mapk(9_000), 3), (W.toy(700, 600, edge_um=0.45), 4), (W.nuclear(8_000, boost=50.0, n_genes=8,
                                                                             genes_on=4), 5)]
    cap_a, cap_c = A.batch_capacity([m for m, _ in sims])
    bt = A.Batch(cap_a, cap_c, len(sims))
    ids = [bt.add(m, s) for m, s in sims]
    bt.step(7)
    for slot, sid in enumerate(ids):
        bt.counts_begin(sid, slot)
    got = [bt.counts_finish(slot) for slot in range(len(ids))]
    for sid, g in zip(ids, got):
        assert np.array_equal(g, bt.counts(sid))
    bt.close()


def test_slot_misuse_is_refused_and_the_handle_keeps_working(A):
    s = A.Sim(W.toy(300, 300, edge_um=0.3), 2)
    s.step(3)
    with pytest.raises(A.AbmError):
        s.counts_finish(0)                  # nothing queued
    s.counts_begin(3)
    with pytest.raises(A.AbmError):
        s.counts_begin(3)                   # still pending
    first = s.counts_finish(3)
    with pytest.raises(A.AbmError):
        s.counts_begin(A.READ_SLOTS)        # no such slot
    assert np.array_equal(first, s.counts())
    s.step(2)
    s.counts_begin(0)
    assert np.array_equal(s.counts_finish(0), s.counts())
    s.close()
