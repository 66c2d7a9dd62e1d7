"""Births at several hundred and at more than a thousand per step (GPU vs
oracle, bit-exact).

Sec. 2 and Sec. 3.4: expressors produce new molecules at a fixed rate
(transcription and translation births) and molecules degrade.  A child's id
is next_id + its rank among the step's births of its simulation, ordered by
parent id.  Here two birth-heavy simulations share one batch (so the births
of both land in one buffer and are ranked per simulation), about 360 and
1,200 births per step, with children that emit again (parents with large,
scattered ids) and bind, so some parents are immune while bound.  Digests
are compared after every step and the full id-sorted dumps at the end."""
import numpy as np
import pytest

import workloads as W
from gpu_common import assert_same_dump, engine, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    require_gpu()
    return engine()


def _births_per_step(counts_trace):
    return np.diff([int(c[-1]) for c in counts_trace])


def test_births_in_a_shared_batch_equal_the_oracle(A, oracle_mod):
    sims = [(W.births(300), 9), (W.births(1000), 10)]
    cap_a, cap_c = A.batch_capacity([m for m, _ in sims], headroom=8.0)
    bt = A.Batch(cap_a, cap_c, 2)
    ids = [bt.add(m, s) for m, s in sims]
    orcs = [oracle_mod.OracleSim(m, s) for m, s in sims]
    trace = [[o.counts()] for o in orcs]
    for t in range(1, 26):
        bt.step(1)
        for k, (sid, o) in enumerate(zip(ids, orcs)):
            o.step(1)
            assert bt.digest(sid) == o.digest(), f"sim {k} step {t}"
            c = o.counts()
            assert np.array_equal(bt.counts(sid), c), f"sim {k} step {t}"
            trace[k].append(c)
    per = [_births_per_step(tr) for tr in trace]
    assert per[0][5:].min() > 250 and per[1][5:].min() > 1024, per   # the loads this test is about
    for k, (sid, o) in enumerate(zip(ids, orcs)):
        assert_same_dump(bt.dump(sid), o.dump(), f"sim {k} after 25 steps")
        o.close()
    bt.close()


def test_births_alone_equal_the_oracle_for_60_steps(A, oracle_mod):
    m, seed = W.births(1500), 21
    sim = A.Sim(m, seed, capacity=40_000)
    o = oracle_mod.OracleSim(m, seed)
    for t in range(1, 61):
        sim.step(1)
        o.step(1)
        assert sim.digest() == o.digest(), f"step {t}"
    assert_same_dump(sim.dump(), o.dump(), "after 60 steps")
    o.close()
    sim.close()
