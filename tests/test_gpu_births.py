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


def test_fifty_thousand_births_per_step_equal_the_oracle(A, oracle_mod):
    """50,000 to 60,000 births per step in one simulation (its limit raised
    to 80,000): every child's id is next_id + its rank by parent id among
    that many parents, ranked on the GPU in parallel; digests every step and
    the dump at the end equal the oracle's."""
    m, seed = W.births(50_000), 31
    sim = A.Sim(m, seed, capacity=500_000, births_per_step=80_000)
    o = oracle_mod.OracleSim(m, seed)
    prev = o.counts()[-1]
    loads = []
    for t in range(1, 7):
        sim.step(1)
        o.step(1)
        c = o.counts()
        loads.append(int(c[-1] - prev))
        prev = c[-1]
        assert sim.digest() == o.digest(), f"step {t}"
    assert min(loads) >= 50_000, loads
    assert_same_dump(sim.dump(), o.dump(), "after 6 steps")
    o.close()
    sim.close()


def test_a_simulation_over_its_births_limit_stops_alone(A, oracle_mod):
    """Births of one step beyond a simulation's limit stop that simulation
    only (its own error; ECAPACITY from its status and reads): the other
    simulation of the batch goes on bit-exact, before and after the failed
    one is removed."""
    ok_m, bad_m = W.births(300), W.births(1000)          # ~360 and ~1,200 births per step
    cap_a, cap_c = A.batch_capacity([ok_m, bad_m], headroom=8.0)
    bt = A.Batch(cap_a, cap_c, 2, births_per_step=1024)
    good, bad = bt.add(ok_m, 9), bt.add(bad_m, 10)
    o = oracle_mod.OracleSim(ok_m, 9)
    for t in range(1, 16):
        bt.step(1)
        o.step(1)
        assert bt.digest(good) == o.digest(), f"step {t}"
    st, msg = bt.sim_status(bad)
    assert st == A.ECAPACITY and "births" in msg
    with pytest.raises(A.AbmError) as e:
        bt.counts(bad)
    assert e.value.status == A.ECAPACITY
    assert bt.sim_status(good) == (A.OK, "")
    bt.remove(bad)
    for t in range(16, 31):
        bt.step(1)
        o.step(1)
        assert bt.digest(good) == o.digest(), f"step {t}"
    assert_same_dump(bt.dump(good), o.dump(), "after 30 steps")
    o.close()
    bt.close()


def test_long_and_short_segments_in_one_batch_equal_the_oracle(A, oracle_mod):
    """A long births segment (more than 2,048 births a step: ranked through
    sorted tiles) between two short ones (ranked directly), so that blocks
    of the ranking hold births of two simulations: digests every step and
    the dumps at the end equal the oracle's."""
    sims = [(W.births(300), 41), (W.births(2000), 42), (W.births(250), 43)]
    cap_a, cap_c = A.batch_capacity([m for m, _ in sims], headroom=8.0)
    bt = A.Batch(cap_a, cap_c, 3)
    ids = [bt.add(m, s) for m, s in sims]
    orcs = [oracle_mod.OracleSim(m, s) for m, s in sims]
    prev = int(orcs[1].counts()[-1])
    loads = []
    for t in range(1, 13):
        bt.step(1)
        for k, (sid, o) in enumerate(zip(ids, orcs)):
            o.step(1)
            assert bt.digest(sid) == o.digest(), f"sim {k} step {t}"
        c = int(orcs[1].counts()[-1])
        loads.append(c - prev)
        prev = c
    assert min(loads[2:]) > 2048, loads                  # the middle segment takes the sorted path
    for k, (sid, o) in enumerate(zip(ids, orcs)):
        assert_same_dump(bt.dump(sid), o.dump(), f"sim {k} after 12 steps")
        o.close()
    bt.close()
