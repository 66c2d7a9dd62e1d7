"""Serving: continuous batching of jobs that arrive over time (GPU).

Jobs arrive while others are resident; they are admitted as memory and slots
free up and are stepped together.  Every job's result (counts and digest at
its last step) must equal the same job run alone, bit for bit, and the
oracle's (the jobs are at most 30k agents x 200 steps)."""
import numpy as np
import pytest

import workloads as W
from gpu_common import engine, require_gpu

pytestmark = pytest.mark.gpu


def _jobs():
    specs = [
        (0.000, W.mapk(20_000), 5, 120),
        (0.001, W.nuclear(15_000, boost=100.0, n_genes=16, genes_on=8), 6, 200),
        (0.002, W.mapk(12_000, drug_frac=0.0), 7, 60),
        (0.050, W.toy(800, 700, edge_um=0.5), 8, 150),
        (0.060, W.mapk(30_000, drug_frac=0.05), 9, 90),
        (0.200, W.nuclear(9_000, boost=50.0, n_genes=8, genes_on=4), 10, 70),
        (0.210, W.mapk(8_000), 11, 40),
    ]
    return [W.Job(k, t, m, s, n) for k, (t, m, s, n) in enumerate(specs)]


@pytest.fixture(scope="module")
def oracle_results(oracle_mod):
    out = {}
    for j in _jobs():
        o = oracle_mod.OracleSim(j.model, j.seed)
        o.step(j.steps)
        out[j.job_id] = (o.digest(), o.counts())
        o.close()
    return out


@pytest.mark.parametrize("groups", [1, 2])
def test_served_jobs_equal_alone_runs(groups, oracle_results):
    require_gpu()
    A = engine()
    from paper_2606_14603_b300 import serve
    jobs = _jobs()
    # small capacities: not all jobs fit at once, so admission has to wait
    caps = [A.model_grid(j.model)[1] for j in jobs]
    # one batch: 45k agent slots and 3 jobs; two batches: one job slot each
    srv = serve.Server(capacity_agents=45_000 * groups, capacity_cells=2 * max(caps) * groups,
                       max_sims=3 if groups == 1 else groups, epoch=25, groups=groups)
    out = serve.run(jobs, srv, real_time=False)
    srv.close()
    assert out["jobs_completed"] == len(jobs) and out["jobs_rejected"] == 0
    assert out["max_resident"] >= 2                       # work overlapped on the device
    assert out["admissions_waited"] >= 1                  # admission by the budget
    by_id = {r.job_id: r for r in out["results"]}
    for j in jobs:
        alone = A.Sim(j.model, j.seed)
        alone.step(j.steps)
        r = by_id[j.job_id]
        assert r.digest == alone.digest(), f"job {j.job_id}"
        assert np.array_equal(r.counts, alone.counts()), f"job {j.job_id}"
        alone.close()
        od, oc = oracle_results[j.job_id]
        assert r.digest == od and np.array_equal(r.counts, oc), f"job {j.job_id} vs the oracle"
    lat = [r.latency_s for r in out["results"]]
    assert out["latency_p50_s"] <= out["latency_p99_s"] and min(lat) >= 0


def test_server_rejects_jobs_that_can_never_fit():
    require_gpu()
    engine()
    from paper_2606_14603_b300 import serve
    jobs = [W.Job(0, 0.0, W.mapk(200_000), 1, 10), W.Job(1, 0.0, W.mapk(5_000), 2, 10)]
    srv = serve.Server(capacity_agents=20_000, capacity_cells=10_000_000, max_sims=2)
    out = serve.run(jobs, srv, real_time=False)
    srv.close()
    assert out["jobs_rejected"] == 1 and out["jobs_completed"] == 1


def test_a_failing_job_fails_alone_in_a_shared_batch():
    """A job whose births in one step exceed its limit stops with its own
    error (its simulation is frozen, reported failed and removed); the
    healthy job resident in the same batch, and a later job admitted into
    it, complete equal to their alone runs and to the oracle."""
    require_gpu()
    A = engine()
    from paper_2606_14603_b300 import serve
    import oracle
    flood = W.Model("flood", [W.Species("G", 20_000, 0.0, p_emit=1.0, emit=1), W.Species("P", 0, 0.0)], [],
                    [W.Compartment(W.CUBE, 2.0)])
    jobs = [W.Job(0, 0.000, W.mapk(12_000), 3, 80),
            W.Job(1, 0.001, flood, 4, 30),
            W.Job(2, 0.050, W.mapk(9_000, drug_frac=0.0), 5, 60)]
    caps = [A.model_grid(j.model)[1] for j in jobs]
    srv = serve.Server(capacity_agents=80_000, capacity_cells=4 * max(caps), max_sims=3, epoch=20, groups=1)
    out = serve.run(jobs, srv, real_time=False)
    srv.close()
    assert out["jobs_failed"] == 1 and out["batch_failures"] == 0 and out["sim_failures"] == 1
    assert [r.job_id for r in out["failed"]] == [1] and "births" in out["failed"][0].error
    assert sorted(r.job_id for r in out["results"]) == [0, 2]
    assert out["max_resident"] >= 2                       # the failing job shared the batch
    for r in out["results"]:
        j = jobs[r.job_id]
        alone = A.Sim(j.model, j.seed)
        alone.step(j.steps)
        assert r.digest == alone.digest(), f"job {j.job_id}"
        assert np.array_equal(r.counts, alone.counts()), f"job {j.job_id}"
        alone.close()
        o = oracle.OracleSim(j.model, j.seed)
        o.step(j.steps)
        assert r.digest == o.digest(), f"job {j.job_id} vs the oracle"
        o.close()


def test_a_failing_batch_fails_only_its_jobs():
    """A job that overflows its batch's agent capacity (births within its
    own limit, but more agents than the batch holds) makes that batch report
    ECAPACITY: the jobs resident in that batch are reported failed, the batch
    is replaced, and the other batch's jobs (and later jobs) complete, equal
    to their alone runs."""
    require_gpu()
    A = engine()
    from paper_2606_14603_b300 import serve
    grow = W.Model("grow", [W.Species("G", 8_000, 0.0, p_emit=1.0, emit=1), W.Species("P", 0, 0.0)], [],
                   [W.Compartment(W.CUBE, 2.0)])                 # 8,000 births a step: within its limit
    jobs = [W.Job(0, 0.000, W.mapk(12_000), 3, 80),
            W.Job(1, 0.001, grow, 4, 30),
            W.Job(2, 0.050, W.mapk(9_000, drug_frac=0.0), 5, 60)]
    caps = [A.model_grid(j.model)[1] for j in jobs]
    srv = serve.Server(capacity_agents=2 * 40_000, capacity_cells=4 * max(caps), max_sims=2, epoch=20, groups=2)
    out = serve.run(jobs, srv, real_time=False)
    srv.close()
    assert out["jobs_failed"] == 1 and out["batch_failures"] == 1
    assert [r.job_id for r in out["failed"]] == [1] and "agent capacity" in out["failed"][0].error
    assert sorted(r.job_id for r in out["results"]) == [0, 2]
    for r in out["results"]:
        j = jobs[r.job_id]
        alone = A.Sim(j.model, j.seed)
        alone.step(j.steps)
        assert r.digest == alone.digest(), f"job {j.job_id}"
        alone.close()


def test_backfill_lets_small_jobs_pass_a_large_one_and_stays_exact():
    """Backfill admission: a large job that does not fit yet is passed by
    small ones that do (overtakes counted); every result still equals its
    alone run, and FIFO on the same jobs admits in arrival order."""
    require_gpu()
    A = engine()
    from paper_2606_14603_b300 import serve
    jobs = [W.Job(0, 0.0, W.mapk(30_000), 3, 60),
            W.Job(1, 0.0, W.mapk(30_000, drug_frac=0.0), 4, 40),     # does not fit next to job 0
            W.Job(2, 0.0, W.toy(600, 500, edge_um=0.4), 5, 50),     # fits next to job 0
            W.Job(3, 0.0, W.toy(700, 400, edge_um=0.4), 6, 30)]
    caps = [A.model_grid(j.model)[1] for j in jobs]
    res = {}
    for policy in ("fifo", "backfill"):
        srv = serve.Server(capacity_agents=50_000, capacity_cells=3 * max(caps), max_sims=4, epoch=10, groups=1)
        res[policy] = serve.run(jobs, srv, real_time=False, admission=policy, backfill_limit_s=1e9)
        srv.close()
        assert res[policy]["jobs_completed"] == 4 and res[policy]["jobs_censored"] == 0
    assert res["fifo"]["overtakes"] == 0 and res["backfill"]["overtakes"] >= 1
    done_fifo = {r.job_id: r.finished_s for r in res["fifo"]["results"]}
    done_bf = {r.job_id: r.finished_s for r in res["backfill"]["results"]}
    assert done_bf[2] < done_fifo[2]                       # the small job no longer waits for job 1
    by_id = {r.job_id: r for r in res["backfill"]["results"]}
    for j in jobs:
        alone = A.Sim(j.model, j.seed)
        alone.step(j.steps)
        assert by_id[j.job_id].digest == alone.digest(), f"job {j.job_id}"
        alone.close()


def test_censored_jobs_count_in_the_latency():
    """Stopping at the horizon without draining: jobs still queued or running
    are counted at their age (lower bounds) and reported as censored."""
    require_gpu()
    engine()
    from paper_2606_14603_b300 import serve
    jobs = [W.Job(k, 0.001 * k, W.mapk(20_000), k + 1, 4000) for k in range(4)]
    srv = serve.Server(capacity_agents=30_000, capacity_cells=4 * 30_000, max_sims=2, epoch=50, groups=1)
    out = serve.run(jobs, srv, duration_s=0.05, real_time=False, drain=False)
    srv.close()
    assert out["jobs_offered"] == 4
    assert out["jobs_completed"] + out["jobs_censored"] + out["jobs_failed"] == 4
    assert out["jobs_censored"] >= 1 and out["latency_is_lower_bound"]
    assert out["latency_max_s"] >= max(0.0, out["wall_s"] - 0.003)
