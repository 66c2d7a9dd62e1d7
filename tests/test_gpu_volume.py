"""Volume invariance of the dose readout (Sec. 3.2, simulation performance
factors: the final relative change of pERK + ppERK agrees within about one
percentage point between a volume and ten times that volume, at every dose).

Two tests: at 200k vs 2M agents per dose the property itself; at 20k vs
200k agents per dose, a size the oracle runs, the engine's readout (taken
by the threshold monitor inside the batched step) against the oracle's
counts: every sampled value and every change in percent, exactly."""
import multiprocessing as mp

import pytest

import workloads as W
from gpu_common import engine, require_gpu

pytestmark = pytest.mark.gpu


def test_readout_volume_invariant():
    require_gpu()
    A = engine()
    from paper_2606_14603_b300.experiments import volume_invariance
    r = volume_invariance(lambda n, d: W.mapk(n, d), [0.0, 0.05, 0.10], 200_000, factor=10,
                          steps=2000, period=100)
    assert r["agents"][1] == pytest.approx(10 * r["agents"][0], rel=1e-6)
    for small, large in zip(*r["change_pct"]):
        assert small < 0 and large < 0          # the readout falls over the run at every dose
    assert r["max_diff_pp"] <= 1.0, r


def test_readout_equals_the_oracle():
    require_gpu()
    A = engine()
    from paper_2606_14603_b300.experiments import volume_invariance
    import oracle_jobs
    doses, n, factor, steps, period, seed = [0.0, 0.05, 0.10], 20_000, 10, 300, 50, 12
    readout = ("pERK", "ppERK")
    r = volume_invariance(lambda nn, d: W.mapk(nn, d), doses, n, factor=factor, steps=steps, period=period,
                          seed=seed, readout=readout)
    jobs = [((n * vol, d), seed + k, steps, period, readout) for vol in (1, factor) for k, d in enumerate(doses)]
    with mp.get_context("spawn").Pool(min(len(jobs), mp.cpu_count())) as pool:
        want = pool.map(oracle_jobs.readout_trace, jobs, chunksize=1)
    for v in range(2):
        for k in range(len(doses)):
            tr = want[v * len(doses) + k]
            assert r["trace"][v][k] == tr, (v, k)
            assert r["change_pct"][v][k] == 100.0 * (tr[-1] - tr[0]) / tr[0], (v, k)
    assert all(c < 0 for row in r["change_pct"] for c in row)
