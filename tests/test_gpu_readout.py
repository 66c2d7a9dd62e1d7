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


def _live_models():
    import dataclasses
    from test_oracle_p5 import _model
    dense = _model()
    dense = dataclasses.replace(
        dense, species=[dataclasses.replace(sp, D=d) for sp, d in zip(dense.species, [2.0, 1.0, 1.5, 0.5])],
        reactions=[dataclasses.replace(r, p_release=0.2) if r.kind == W.BIND else r for r in dense.reactions])
    return {"toy": (W.toy(700, 600, edge_um=0.45), 3, 60),
            "mapk": (W.mapk(30_000), 4, 40),
            "nuclear": (W.nuclear(20_000, boost=100.0, n_genes=16, genes_on=8), 5, 40),
            "dense": (dense, 6, 40)}


@pytest.mark.parametrize("name", ["toy", "mapk", "nuclear", "dense"])
def test_live_counts_equal_the_counting_pass_and_the_oracle(A, oracle_mod, name):
    """With live counts on, the step itself keeps the counts of its result
    (moves and P1 changes counted by the move pass, reactions and complexes
    by the acceptance walk, births by the bookkeeping): equal, at every step,
    to the pass over all agents and to the oracle.  Read pipelined, one step
    in flight, then after an 8-step graph."""
    m, seed, steps = _live_models()[name]
    s = A.Sim(m, seed, births_per_step=4096)
    s.live_counts(True)
    o = oracle_mod.OracleSim(m, seed)
    want = []
    for k in range(steps):
        s.step(1)
        s.counts_begin(k % 2)
        o.step(1)
        want.append(o.counts())
        if k:
            assert np.array_equal(s.counts_finish((k - 1) % 2), want[k - 1]), (name, k)
    assert np.array_equal(s.counts_finish((steps - 1) % 2), want[-1]), name
    s.step(8)
    o.step(8)
    s.counts_begin(0)
    live = s.counts_finish(0)
    assert np.array_equal(live, s.counts()) and np.array_equal(live, o.counts()), name
    o.close()
    s.close()


def test_live_counts_across_admissions_and_removals(A):
    """A batch whose members change: a read right after an admission or a
    removal counts the agents (the live counts lack the change until a step
    has run), later reads use the live counts; all equal the counting pass."""
    sims = [(W.mapk(9_000), 3), (W.toy(700, 600, edge_um=0.45), 4), (W.nuclear(8_000, boost=50.0, n_genes=8,
                                                                             genes_on=4), 5)]
    extra = (W.mapk(6_000, drug_frac=0.0), 6)
    cap_a, cap_c = A.batch_capacity([m for m, _ in sims] + [extra[0]])
    bt = A.Batch(cap_a, cap_c, 4, births_per_step=4096)
    ids = [bt.add(m, s) for m, s in sims]
    bt.live_counts(True)

    def check(active):
        for slot, sid in enumerate(active):
            bt.counts_begin(sid, slot % A.READ_SLOTS)
            got = bt.counts_finish(slot % A.READ_SLOTS)
            assert np.array_equal(got, bt.counts(sid)), sid

    bt.step(5)
    check(ids)
    ids.append(bt.add(*extra))   # read right away: falls back to the counting pass
    check(ids)
    bt.step(3)
    check(ids)
    bt.remove(ids[1])
    active = [i for k, i in enumerate(ids) if k != 1]
    check(active)
    bt.step(4)
    check(active)
    bt.live_counts(False)
    bt.step(2)
    check(active)
    bt.close()


def test_live_counts_with_a_frozen_simulation(A):
    """A simulation frozen at its last step (as the server freezes finished
    jobs) keeps its agents in place: its live counts stay those of that step
    while the batch steps on, equal to the counting pass."""
    sims = [(W.mapk(9_000), 3), (W.nuclear(8_000, boost=50.0, n_genes=8, genes_on=4), 5)]
    cap_a, cap_c = A.batch_capacity([m for m, _ in sims])
    bt = A.Batch(cap_a, cap_c, 2, births_per_step=4096)
    ids = [bt.add(m, s) for m, s in sims]
    bt.live_counts(True)
    bt.set_max_step(ids[0], 6)
    frozen = None
    for k in range(12):
        bt.step(1)
        for slot, sid in enumerate(ids):
            bt.counts_begin(sid, slot)
            got = bt.counts_finish(slot)
            assert np.array_equal(got, bt.counts(sid)), (k, sid)
            if sid == ids[0] and k >= 5:
                frozen = got if frozen is None else frozen
                assert np.array_equal(got, frozen), k
    bt.close()


@pytest.mark.parametrize("n", [1_200_000, 2_600_000])
def test_live_counts_on_the_large_launch_shapes(A, n):
    """Capacities of 1M to 2M agents run the move pass in 128-thread blocks
    (its live-counting variant on a resident grid of its own), larger ones
    in its 48-register variant: with live counts on, the counts after every
    step equal the counting pass, and the trajectory equals the same
    simulation's without live counts."""
    m = W.mapk(n)
    g = A.Sim(m, 7)
    h = A.Sim(m, 7)
    try:
        g.live_counts(True)
        for t in range(1, 9):
            g.step(1)
            h.step(1)
            g.counts_begin(t % 2)
            live = g.counts_finish(t % 2)
            assert np.array_equal(live, g.counts()), (n, t)
        assert g.digest() == h.digest()
        assert np.array_equal(g.counts(), h.counts())
    finally:
        g.close()
        h.close()
