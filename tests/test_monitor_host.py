"""Threshold monitor on the CPU: the definition in oracle/monitor.py pinned
by hand-worked cases and by a conservation law of the toy model, and the
weight helper's layout (host logic, no device)."""
import numpy as np

import workloads as W
from oracle import monitor as M


def test_hand_worked_window_and_threshold():
    vals = {0: 5, 1: 7, 2: 12, 3: 3, 4: 15}
    r = M.evaluate(vals, begin=1, end=4, period=1, threshold=10, above=True)
    # evaluated at t = 1, 2, 3: 7 (no), 12 (yes), 3 (no); t = 4 lies outside [1, 4)
    assert r["trace"] == [7, 12, 3]
    assert (r["first_pass"], r["n_passed"], r["n_evaluated"]) == (2, 1, 3)
    assert r["state"] is False and r["value"] == 3 and r["last_step"] == 3


def test_below_threshold_period_and_late_install():
    vals = {t: 100 - 10 * t for t in range(10)}
    r = M.evaluate(vals, begin=2, end=None, period=3, threshold=45, above=False)
    # due steps 2, 5, 8: values 80, 50, 20; below 45 only at t = 8
    assert r["trace"] == [80, 50, 20] and r["first_pass"] == 8 and r["state"] is True
    r = M.evaluate(vals, begin=2, end=None, period=3, threshold=45, above=False, installed_at=3)
    assert r["trace"] == [50, 20] and r["n_evaluated"] == 2
    # strict comparison: equal to the threshold does not pass
    r = M.evaluate({0: 45}, begin=0, end=1, period=1, threshold=45, above=False)
    assert r["n_passed"] == 0 and r["state"] is False


def test_no_evaluation_and_ring():
    r = M.evaluate({0: 1, 1: 2}, begin=5, end=9, period=1, threshold=0, above=True)
    assert r["n_evaluated"] == 0 and r["state"] is None and r["first_pass"] is None
    vals = {t: t for t in range(1500)}
    r = M.evaluate(vals, begin=0, end=None, period=1, threshold=1200, above=True)
    assert r["n_evaluated"] == 1500 and len(r["trace"]) == 1024 and r["trace"][0] == 1500 - 1024
    assert r["first_pass"] == 1201


def test_value_weights_shorter_than_counts():
    assert M.value([3, 4, 5, 99], [1, -2]) == 3 - 8
    assert M.value([2 ** 40, 1], [2 ** 20, 0]) == 2 ** 60  # exact, no wraparound


def test_toy_conservation_through_the_monitor_value(oracle_mod):
    # A + B -> C converts A into C in place and removes B: n_A + n_C and
    # n_B + n_C stay at their initial 2500 at every step (counts: A, B, C, next id)
    model = W.toy()
    o = oracle_mod.OracleSim(model, 1)
    try:
        seen_c = []
        for _ in range(40):
            c = o.counts()
            assert M.value(c, [1, 0, 1]) == 2500
            assert M.value(c, [0, 1, 1]) == 2500
            seen_c.append(M.value(c, [0, 0, 1]))
            o.step(1)
        assert seen_c[-1] > seen_c[0]  # reactions happened
    finally:
        o.close()


def test_monitor_weights_layout():
    import paper_2606_14603_b300 as A
    toy = W.toy()
    # counts layout: A, B, C free, then one bound entry for the (CONVERT) reaction A + B
    assert A.monitor_weights(toy, ["C"]).tolist() == [0, 0, 1, 0]
    assert A.monitor_weights(toy, [0, 2]).tolist() == [1, 0, 1, 1]
    m = W.mapk(30_000, 0.05, 3.0, 1e-6)
    names = [s.name for s in m.species]
    w = A.monitor_weights(m, ["ppERK"])
    n_sp, n_comp = len(m.species), len(m.compartments)
    assert len(w) == n_sp * n_comp + len(m.reactions)
    pp = names.index("ppERK")
    expect = np.zeros_like(w)
    expect[pp * n_comp] = 1
    for r, rx in enumerate(m.reactions):
        expect[n_sp * n_comp + r] = (rx.a == pp) + (rx.b == pp)
    assert np.array_equal(w, expect) and expect[n_sp * n_comp:].sum() >= 1
    assert A.monitor_weights(m, ["ppERK"], include_bound=False).sum() == 1
