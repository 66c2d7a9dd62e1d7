"""Longer parity runs, engine vs oracle, bit-exact (digest at checkpoints):
the 1M-agent cascade for its first 200 steps, a 50k-agent cascade for the
cascade's full 10,000 steps, a boosted 40k-agent two-compartment model for
2,000 steps, every simulation of
the 64-simulation sweep for its first 100 steps in the batch (the 8 smallest
to 1,000), and all 64 in the batch against the same simulations run alone
for 5,000 steps.  (The 4M-agent two-compartment model is checked for 3 steps
in test_gpu_parity: the oracle needs about 25 s per step of it.)

The oracle runs execute in worker processes (spawned, one per host core)
while the GPU side runs."""
import multiprocessing as mp
import os

import pytest

import workloads as W
from gpu_common import engine, require_gpu
from oracle_jobs import build_model, digest_trace

pytestmark = pytest.mark.gpu

SWEEP = W.sweep()
SMALLEST = sorted(range(len(SWEEP)), key=lambda k: SWEEP[k][0].n_agents)[:8]
JOBS = {
    "mapk_1M": ("mapk", {"n_total": 1_000_000}, W.MAPK_SEED, list(range(25, 201, 25))),
    "mapk_50k": ("mapk", {"n_total": 50_000}, W.MAPK_SEED, list(range(1000, 10_001, 1000))),
    "nuclear_40k": ("nuclear", {"n_total": 40_000, "boost": 100.0, "n_genes": 32, "genes_on": 16},
                    W.NUCLEAR_SEED, list(range(250, 2001, 250))),
}
for k, (m, seed) in enumerate(SWEEP):
    JOBS[f"sweep_{k}"] = ("sweep", {"k": k}, seed, [100, 500, 1000] if k in SMALLEST else [100])


@pytest.fixture(scope="module")
def oracle_runs():
    require_gpu()
    order = sorted(JOBS, key=lambda name: -build_model(*JOBS[name][:2]).n_agents * JOBS[name][3][-1])
    pool = mp.get_context("spawn").Pool(os.cpu_count() or 1)
    results = {name: pool.apply_async(digest_trace, (JOBS[name],)) for name in order}
    yield lambda name: results[name].get(timeout=1800)
    pool.terminate()
    pool.join()


@pytest.fixture(scope="module")
def A():
    require_gpu()
    return engine()


@pytest.mark.parametrize("name", ["mapk_1M", "mapk_50k", "nuclear_40k"])
def test_long_single(A, oracle_runs, name):
    kind, params, seed, checkpoints = JOBS[name]
    g = A.Sim(build_model(kind, params), seed)
    got = {}
    t = 0
    for c in checkpoints:
        g.step(c - t)
        t = c
        got[c] = g.digest()
    g.close()
    want = oracle_runs(name)
    for c in checkpoints:
        assert got[c] == want[c], f"{name}: digest differs at step {c}"


def test_sweep_batch_against_oracle_and_alone(A, oracle_runs):
    models = [m for m, _ in SWEEP]
    cap_a, cap_c = A.batch_capacity(models)
    b = A.Batch(cap_a, cap_c, len(SWEEP))
    ids = [b.add(m, s) for m, s in SWEEP]
    got = {c: {} for c in (100, 500, 1000, 5000)}
    t = 0
    for c in (100, 500, 1000, 5000):
        b.step(c - t)
        t = c
        for k, sid in enumerate(ids):
            if c == 100 or c == 5000 or k in SMALLEST:
                got[c][k] = b.digest(sid)
    b.close()
    for k in range(len(SWEEP)):
        want = oracle_runs(f"sweep_{k}")
        for c, d in want.items():
            assert got[c][k] == d, f"sweep sim {k} ({models[k].n_agents} agents): step {c}"
    for k, (m, s) in enumerate(SWEEP):  # the full length, alone on the GPU
        g = A.Sim(m, s)
        g.step(5000)
        assert g.digest() == got[5000][k], f"sweep sim {k}: batch and alone differ at step 5000"
        g.close()
