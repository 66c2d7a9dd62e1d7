"""Threshold monitor on the GPU against its definition applied to the
oracle's counts at every step (exact integers): windows, periods, lower and
upper thresholds, a monitor installed mid-run, a frozen simulation, reads
between steps (idempotent), the 1024-value trace ring, and errors.  The
monitor never changes the trajectory."""
import numpy as np
import pytest

import workloads as W
from gpu_common import engine, require_gpu
from oracle import monitor as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    require_gpu()
    return engine()


def _oracle_values(oracle_mod, model, seed, steps, weights, max_step=None):
    o = oracle_mod.OracleSim(model, seed)
    try:
        vals = {0: M.value(o.counts(), weights)}
        last = steps if max_step is None else min(steps, max_step)
        for t in range(1, last + 1):
            o.step(1)
            vals[t] = M.value(o.counts(), weights)
        return vals
    finally:
        o.close()


def _same(got, want, where):
    assert got.value == want["value"], where
    assert got.last_step == want["last_step"], where
    assert got.first_pass == want["first_pass"], where
    assert got.n_evaluated == want["n_evaluated"], where
    assert got.n_passed == want["n_passed"], where
    assert got.state == want["state"], where
    assert got.trace.tolist() == want["trace"], where


def test_toy_window_period_reads(A, oracle_mod):
    model = W.toy()
    w = A.monitor_weights(model, ["C"])
    vals = _oracle_values(oracle_mod, model, 1, 200, w)
    rule = dict(begin=10, end=170, period=3, threshold=100, above=True)
    with A.Sim(model, 1) as g:
        g.monitor(w, **rule)
        for upto in (7, 57, 57, 100, 200):
            g.step(upto - g.t)
            got = g.monitor_read()
            _same(got, M.evaluate({t: v for t, v in vals.items() if t <= upto}, **rule), f"t={upto}")
        assert got.first_pass is not None and got.n_evaluated == len(range(10, 170, 3))


def test_batch_monitors_mid_run_frozen_and_cleared(A, oracle_mod):
    models = [W.mapk(30_000, 0.0, 3.0, 1e-6), W.mapk(30_000, 0.05, 3.0, 1e-6), W.mapk(30_000, 0.1, 3.0, 1e-6)]
    seeds = [12, 42, 7]
    wpp = A.monitor_weights(models[0], ["ppERK"])
    werk = A.monitor_weights(models[1], ["pERK", "ppERK"])
    wneg = -A.monitor_weights(models[2], ["ERK"], include_bound=False)
    wneg[0] = 3  # mixed signs: 3 * free BRAF* in the cytosol - free ERK
    rules = [dict(begin=0, end=None, period=1, threshold=None, above=True),
             dict(begin=20, end=120, period=5, threshold=None, above=False),
             dict(begin=41, end=None, period=2, threshold=None, above=True)]
    vals = [_oracle_values(oracle_mod, m, s, 150, w, max_step=ms)
            for m, s, w, ms in zip(models, seeds, [wpp, werk, wneg], [None, 100, None])]
    # thresholds inside the range of the due values, so that some pass and some do not
    for rule, v, due in zip(rules, vals, [range(0, 151), range(20, 101, 5), range(41, 151, 2)]):
        lo, hi = min(v[t] for t in due), max(v[t] for t in due)
        assert hi > lo, "the followed quantity did not change"
        rule["threshold"] = (lo + hi) // 2 if rule["above"] else (lo + hi + 1) // 2
    cap_a, cap_c = A.batch_capacity(models)
    b = A.Batch(cap_a, cap_c, 4)
    try:
        sids = [b.add(m, s) for m, s in zip(models, seeds)]
        b.set_max_step(sids[1], 100)
        b.monitor(sids[0], wpp, **rules[0])
        b.monitor(sids[1], werk, **rules[1])
        t = 0
        for upto in (13, 40, 95, 150):
            b.step(upto - t)
            t = upto
            if t == 40:
                b.monitor(sids[2], wneg, **rules[2])   # installed mid-run, at step 40
            for k in (0, 1):
                want = M.evaluate({u: v for u, v in vals[k].items() if u <= min(t, 100 if k == 1 else t)},
                                  **rules[k])
                _same(b.monitor_read(sids[k]), want, f"sim {k} t={t}")
            if t >= 40:
                want = M.evaluate({u: v for u, v in vals[2].items() if u <= t}, installed_at=40, **rules[2])
                _same(b.monitor_read(sids[2]), want, f"sim 2 t={t}")
        assert b.monitor_read(sids[1]).last_step == 100  # frozen at 100, evaluated once
        for k in range(3):
            st = b.monitor_read(sids[k])
            assert 0 < st.n_passed < st.n_evaluated, (k, st)   # the thresholds were crossed
        b.monitor_clear(sids[0])
        with pytest.raises(A.AbmError) as e:
            b.monitor_read(sids[0])
        assert e.value.status == A.ESTATE
    finally:
        b.close()


def test_trace_ring_keeps_last_1024(A, oracle_mod):
    model = W.toy()
    w = A.monitor_weights(model, ["A"])
    vals = _oracle_values(oracle_mod, model, 3, 1100, w)
    rule = dict(begin=0, end=None, period=1, threshold=2400, above=False)
    with A.Sim(model, 3) as g:
        g.monitor(w, **rule)
        g.step(1100)
        got = g.monitor_read()
    want = M.evaluate(vals, **rule)
    assert want["n_evaluated"] == 1101 and len(want["trace"]) == 1024
    _same(got, want, "t=1100")


def test_monitor_does_not_change_the_trajectory(A):
    model = W.mapk(30_000, 0.05, 3.0, 1e-6)
    with A.Sim(model, 5) as g, A.Sim(model, 5) as h:
        g.monitor(A.monitor_weights(model, ["ppERK"]), threshold=0, period=1)
        g.step(60)
        h.step(60)
        assert g.digest() == h.digest()
        assert np.array_equal(g.counts(), h.counts())


def test_monitor_errors(A):
    model = W.toy()
    cap_a, cap_c = A.batch_capacity([model])
    b = A.Batch(cap_a * 2, cap_c * 2, 2)
    try:
        s = b.add(model, 1)
        with pytest.raises(A.AbmError) as e:
            b.monitor_read(s)
        assert e.value.status == A.ESTATE
        for kw in (dict(period=0), dict(begin=5, end=5)):
            with pytest.raises(A.AbmError) as e:
                b.monitor(s, [1], threshold=0, **kw)
            assert e.value.status == A.EINVAL
        with pytest.raises(A.AbmError) as e:
            b.monitor(s, [1, 1, 1, 1, 1], threshold=0)   # longer than the 4 countable entries
        assert e.value.status == A.EINVAL
        with pytest.raises(A.AbmError) as e:
            b.monitor(s, [2 ** 20 + 1], threshold=0)
        assert e.value.status == A.EINVAL
        with pytest.raises(A.AbmError) as e:
            b.monitor(3, [1], threshold=0)                # free slot
        assert e.value.status == A.ESTATE
        b.monitor(s, [1], threshold=0)
        b.step(3)
        assert b.monitor_read(s).n_evaluated == 4
        b.remove(s)                                       # removal clears the monitor
        s2 = b.add(model, 2)
        with pytest.raises(A.AbmError) as e:
            b.monitor_read(s2)
        assert e.value.status == A.ESTATE
        b.step(2)
        assert b.counts(s2)[-1] == 5000   # the new simulation steps normally (no births in the toy)
    finally:
        b.close()
