"""Engine vs oracle on seeded random models, bit-exact.

Each model draws its own shape from a seeded generator: 2-7 species (some
with no initial agents, some immobile), first-order conversions and deaths,
expressors, 0-6 CONVERT or BIND reactions between distinct species pairs
with radii of 3-25 nm, and either a cube or a spherical cell with an
off-centre nucleus whose membrane some species may cross.  The same rules
the library enforces (Sec. 2 inputs: species, reactions with radii and
probabilities, compartments) bound every choice, so every model is valid.
Each runs alone on the engine and on the oracle in lock step (digest every
step, dump and counts at the end); then all of them share one batch, in
three launch shapes and grids, and each member must equal its oracle run
again."""
import random

import numpy as np
import pytest

import workloads as W
from gpu_common import assert_same_dump, engine, require_gpu

pytestmark = pytest.mark.gpu

N_MODELS = 32
STEPS = 60


@pytest.fixture(scope="module")
def A():
    require_gpu()
    return engine()


def random_model(r: random.Random, k: int) -> W.Model:
    n_sp = r.randint(2, 7)
    two = r.random() < 0.5
    if two:
        comps = [W.Compartment(W.SPHERE, r.choice([0.5, 0.6, 0.8])),
                 W.Compartment(W.SPHERE, r.choice([0.2, 0.25]), parent=0,
                               center_um=(r.uniform(-0.05, 0.05), r.uniform(-0.05, 0.05), 0.0))]
    else:
        comps = [W.Compartment(W.CUBE, r.choice([0.3, 0.5, 0.7]))]
    species = []
    for i in range(n_sp):
        count = r.choice([0, 1, 7, 200, 800, 1500, 3000])
        D = r.choice([0.0, 0.3, 1.0, 3.0, 8.0])
        s = W.Species(f"S{i}", count, D, comp=r.randrange(len(comps)),
                      p_cross=r.choice([0.0, 0.3, 1.0]) if two else 0.0)
        if r.random() < 0.3:
            s.p_uni = r.choice([0.005, 0.02, 0.1])
            s.uni_to = r.choice([-1] + list(range(n_sp)))
        if r.random() < 0.2:
            s.p_emit = r.choice([0.005, 0.02])
            s.emit = r.randrange(n_sp)
        species.append(s)
    pairs = [(a, b) for a in range(n_sp) for b in range(n_sp) if a < b]
    r.shuffle(pairs)
    reactions = []
    for a, b in pairs[: r.randint(0, min(6, len(pairs)))]:
        if r.random() < 0.5:
            a, b = b, a
        kind = r.choice([W.CONVERT, W.BIND])
        reactions.append(W.Reaction(a, b, kind, r.choice([-1] + list(range(n_sp))),
                                    r.choice([-1] + list(range(n_sp))), r.uniform(3.0, 25.0),
                                    r.choice([0.1, 0.5, 1.0]),
                                    r.choice([0.0, 0.05, 0.3]) if kind == W.BIND else 0.0))
    return W.Model(f"random_{k}", species, reactions, comps)


def models():
    r = random.Random(20261204)
    return [(random_model(r, k), 1000 + k) for k in range(N_MODELS)]


def test_random_models_alone_equal_the_oracle(A, oracle_mod):
    for m, seed in models():
        g = A.Sim(m, seed)
        o = oracle_mod.OracleSim(m, seed)
        try:
            assert_same_dump(g.dump(), o.dump(), f"{m.name} step 0")
            for t in range(1, STEPS + 1):
                g.step(1)
                o.step(1)
                if g.digest() != o.digest():
                    assert_same_dump(g.dump(), o.dump(), f"{m.name} step {t}")
                    raise AssertionError(f"{m.name}: digest differs at step {t} although dumps agree")
            assert_same_dump(g.dump(), o.dump(), f"{m.name} step {STEPS}")
            assert np.array_equal(g.counts(), o.counts()), m.name
        finally:
            g.close()
            o.close()


# launch shapes and grids of the batch: (threads per block, CTAs per SM,
# proposal chunk, cell edge one step above the automatic one); none may
# change a result
SHAPES = [(0, 0, 0, False), (128, 2, 1024, False), (512, 0, 4096, True)]


@pytest.mark.parametrize("threads,blocks,chunk,coarse", SHAPES)
def test_random_models_in_one_batch_equal_the_oracle(A, oracle_mod, threads, blocks, chunk, coarse):
    ms = models()
    cap = sum(int(m.n_agents * 1.5) + 4096 for m, _ in ms)
    b = A.Batch(cap, 64 << 20, len(ms), blocks_per_sm=blocks, threads_per_block=threads, propose_chunk=chunk)
    try:
        sids = [b.add(m, seed, cell_log2=A.model_grid(m)[0] + 1 if coarse else 0) for m, seed in ms]
        b.step(STEPS)
        for (m, seed), sid in zip(ms, sids):
            o = oracle_mod.OracleSim(m, seed)
            o.step(STEPS)
            assert b.digest(sid) == o.digest(), m.name
            assert_same_dump(b.dump(sid), o.dump(), f"{m.name} in the batch")
            assert np.array_equal(b.counts(sid), o.counts()), m.name
            o.close()
    finally:
        b.close()


def test_random_models_checkpoint_and_restore(A, oracle_mod):
    """Half-way checkpoints of the random models restore into fresh
    simulations that finish equal to the oracle's uninterrupted runs."""
    for m, seed in models()[:12]:
        g = A.Sim(m, seed)
        g.step(STEPS // 2)
        ck = g.checkpoint()
        g.close()
        rng = np.random.default_rng(seed)
        rec = ck[0][rng.permutation(len(ck[0]))]          # records in any order
        h = A.Sim(m, seed, restore=(rec, ck[1], ck[2]))
        h.step(STEPS - STEPS // 2)
        o = oracle_mod.OracleSim(m, seed)
        o.step(STEPS)
        try:
            assert h.digest() == o.digest(), m.name
            assert_same_dump(h.dump(), o.dump(), f"{m.name} restored")
        finally:
            h.close()
            o.close()


def test_random_models_admitted_and_removed_mid_run(A, oracle_mod):
    """Members join a running batch at different steps and others leave it;
    each member still equals the oracle run for its own number of steps."""
    ms = models()
    cap = sum(int(m.n_agents * 1.5) + 4096 for m, _ in ms)
    b = A.Batch(cap, 64 << 20, len(ms))
    steps = {}
    sids = {}
    try:
        for k, (m, seed) in enumerate(ms):
            if k % 4 == 0 and k:
                b.step(7)                                  # members so far advance
                for j in sids:
                    steps[j] += 7
            sids[k] = b.add(m, seed)
            steps[k] = 0
            if k % 5 == 4:                                 # an earlier member leaves
                gone = k - 3
                b.remove(sids.pop(gone))
                steps.pop(gone)
        b.step(11)
        for j in sids:
            steps[j] += 11
        for k, sid in sids.items():
            m, seed = ms[k]
            o = oracle_mod.OracleSim(m, seed)
            o.step(steps[k])
            assert b.digest(sid) == o.digest(), (m.name, steps[k])
            assert_same_dump(b.dump(sid), o.dump(), f"{m.name} after {steps[k]} steps")
            o.close()
    finally:
        b.close()


def test_random_models_live_counts(A, oracle_mod):
    """With live counts on, the pipelined read after every step equals the
    oracle's counts of that step."""
    for m, seed in models()[:12]:
        g = A.Sim(m, seed)
        o = oracle_mod.OracleSim(m, seed)
        try:
            g.live_counts(True)
            for t in range(1, 31):
                g.step(1)
                g.counts_begin(t % 2)
                o.step(1)
                assert np.array_equal(g.counts_finish(t % 2), o.counts()), (m.name, t)
        finally:
            g.close()
            o.close()
