"""Engine vs oracle, bit-exact: every config's small case for its full length
(digest every step, dumps and counts at intervals), full-size prefixes in the
launch configuration the bench times, and the RNG against cuRAND's device
Philox.  Tolerance is zero: the state is integer."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import workloads as W
from gpu_common import assert_same_dump, engine, require_gpu

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def A():
    require_gpu()
    return engine()


def _curand_lib():
    d = tempfile.mkdtemp()
    so = os.path.join(d, "libcurand_philox.so")
    subprocess.check_call(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a",
                           "-shared", "-Xcompiler", "-fPIC", "-o", so,
                           os.path.join(HERE, "helpers", "curand_philox.cu")])
    return ctypes.CDLL(so)


def test_philox_engine_oracle_curand_device(A, oracle_mod):
    rng = np.random.default_rng(1234)
    n = 1 << 20
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:16] = [[i, 0, 0, 0] for i in range(16)]           # small counters too
    ctr[16:32, 1:] = 0
    got = A.device_philox(ctr, key)
    ref = np.zeros_like(ctr)
    lib = _curand_lib()
    assert lib.curand_philox_batch(ctr.ctypes.data_as(ctypes.c_void_p), key.ctypes.data_as(ctypes.c_void_p),
                                   ref.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    assert np.array_equal(got, ref)
    for i in list(range(40)) + list(rng.integers(0, n, 200)):
        assert oracle_mod.philox4x32_10(ctr[i].tolist(), key[i].tolist()) == ref[i].tolist()


def _lockstep(A, oracle_mod, model, seed, steps, dump_every, digest_every=1, cell_log2=0):
    g = A.Sim(model, seed, cell_log2=cell_log2)
    o = oracle_mod.OracleSim(model, seed)
    try:
        assert_same_dump(g.dump(), o.dump(), "step 0")
        assert g.digest() == o.digest()
        t = 0
        while t < steps:
            k = min(digest_every, steps - t)
            g.step(k)
            o.step(k)
            t += k
            if g.digest() != o.digest():
                assert_same_dump(g.dump(), o.dump(), f"step {t}")
                raise AssertionError(f"digest differs at step {t} although dumps agree")
            if t % dump_every == 0 or t == steps:
                assert_same_dump(g.dump(), o.dump(), f"step {t}")
                assert np.array_equal(g.counts(), o.counts()), f"counts at step {t}"
        assert g.t == o.t == steps
        return g.counts()
    finally:
        g.close()
        o.close()


def test_toy_full_length(A, oracle_mod):
    c = _lockstep(A, oracle_mod, W.toy(), W.TOY_SEED, W.TOY_STEPS, dump_every=25)
    assert c[2] > 100                                          # C formed


def test_toy_one_launch_of_all_steps(A, oracle_mod):
    """All 200 steps in one abm_step call (25 replays of the 8-step graph)."""
    g = A.Sim(W.toy(), W.TOY_SEED)
    o = oracle_mod.OracleSim(W.toy(), W.TOY_SEED)
    g.step(W.TOY_STEPS)
    o.step(W.TOY_STEPS)
    assert g.t == W.TOY_STEPS and g.digest() == o.digest()
    assert_same_dump(g.dump(), o.dump(), "step 200")
    g.close()
    o.close()


@pytest.mark.parametrize("kind", ["antisymmetric", "skewed"])
def test_caller_gaussian_table(A, oracle_mod, kind):
    """A caller's Gaussian table (abm_options.ncdf_table), antisymmetric like
    the default one or not, gives the oracle's results with that table."""
    base = oracle_mod.ncdf_table()
    if kind == "antisymmetric":
        tab = np.trunc(base.astype(np.float64) * 1.5).astype(np.int16)
        assert np.array_equal(tab[::-1], -tab)
    else:
        tab = base.copy()
        tab[::97] += 1
        assert not np.array_equal(tab[::-1], -tab)
    for m, seed, steps in [(W.toy(700, 600, edge_um=0.45), 31, 60), (W.mapk(20_000), 32, 40)]:
        g = A.Sim(m, seed, ncdf_table=tab)
        o = oracle_mod.OracleSim(m, seed, table=tab)
        ref = oracle_mod.OracleSim(m, seed)
        for _ in range(4):
            g.step(steps // 4)
            o.step(steps // 4)
            ref.step(steps // 4)
            assert g.digest() == o.digest(), (kind, m.name, g.t)
        assert o.digest() != ref.digest()  # the table was used
        assert_same_dump(g.dump(), o.dump(), f"{kind} {m.name}")
        for x in (g, o, ref):
            x.close()


@pytest.mark.parametrize("mobile", [False, True])
def test_dense_conflicts(A, oracle_mod, mobile):
    """About four agents within a contact radius of each: most acceptors are
    contested and many proposers are proposed to, so the final-edge rule
    decides most outcomes (the static case is the one the oracle is pinned
    on by brute force); the mobile case adds moves and releases."""
    import dataclasses
    from test_oracle_p5 import _model
    m = _model()
    if mobile:
        m = dataclasses.replace(m, species=[dataclasses.replace(sp, D=d) for sp, d in zip(m.species, [2.0, 1.0, 1.5, 0.5])],
                                reactions=[dataclasses.replace(r, p_release=0.2) if r.kind == W.BIND else r
                                           for r in m.reactions])
    for seed in (5, 6):
        g = A.Sim(m, seed)
        o = oracle_mod.OracleSim(m, seed)
        for t in range(30):
            g.step(1)
            o.step(1)
            assert g.digest() == o.digest(), (mobile, seed, t + 1)
        assert_same_dump(g.dump(), o.dump(), f"dense mobile={mobile} seed {seed}")
        g.close()
        o.close()


def test_brute_force_models(A, oracle_mod):
    """The small models the oracle is pinned on draw by draw: moves in a cube
    and in a cell with an off-centre nucleus (rejections, crossings), and
    first-order events with births; 30 steps, digest every step."""
    cell = W.Compartment(W.SPHERE, 0.3)
    nucleus = W.Compartment(W.SPHERE, 0.15, parent=0, center_um=(0.02, -0.01, 0.0))
    models = [
        W.Model("cube_moves", [W.Species("X", 300, 3.0), W.Species("Y", 200, 0.6)], [], [W.Compartment(W.CUBE, 0.2)]),
        W.Model("cell_moves", [W.Species("P", 400, 5.0, comp=0, p_cross=0.5),
                               W.Species("R", 300, 5.0, comp=1, p_cross=0.0),
                               W.Species("S", 200, 5.0, comp=1, p_cross=0.5)], [], [cell, nucleus]),
        W.Model("events", [W.Species("U", 200, 0.0, p_uni=0.3, uni_to=1), W.Species("V", 0, 0.0),
                           W.Species("Dd", 200, 0.0, p_uni=0.2, uni_to=-1),
                           W.Species("E", 200, 0.0, p_emit=0.4, emit=4), W.Species("K", 0, 0.0),
                           W.Species("F", 200, 0.0, p_uni=0.25, uni_to=1, p_emit=0.5, emit=4)], [],
                [W.Compartment(W.CUBE, 0.3)]),
    ]
    for m in models:
        g = A.Sim(m, 9, births_per_step=1024)
        o = oracle_mod.OracleSim(m, 9)
        for t in range(30):
            g.step(1)
            o.step(1)
            assert g.digest() == o.digest(), (m.name, t + 1)
        assert_same_dump(g.dump(), o.dump(), m.name)
        g.close()
        o.close()


def test_mapk_scaled_parity(A, oracle_mod):
    c = _lockstep(A, oracle_mod, W.mapk(30_000), W.MAPK_SEED, 400, dump_every=100, digest_every=4)
    assert c[9:-1].sum() > 0                                  # complexes present


def test_nuclear_boosted_parity(A, oracle_mod):
    m = W.nuclear(30_000, boost=100.0, n_genes=32, genes_on=16)
    c = _lockstep(A, oracle_mod, m, W.NUCLEAR_SEED, 400, dump_every=100, digest_every=4)
    n_sp, n_c = len(m.species), len(m.compartments)
    free = c[: n_sp * n_c].reshape(n_sp, n_c)
    assert c[-1] > m.n_agents + 1000                           # many births
    assert free[8].sum() + free[9].sum() > 0                   # mRNA / cFos present


def test_grid_size_does_not_change_results(A, oracle_mod):
    m = W.mapk(20_000)
    digests = []
    for cl in (0, 8, 9, 11):
        g = A.Sim(m, 5, cell_log2=cl)
        g.step(50)
        digests.append(g.digest())
        g.close()
    o = oracle_mod.OracleSim(m, 5)
    o.step(50)
    assert digests == [o.digest()] * 4


def test_mapk_full_size_prefix(A, oracle_mod):
    """The 1,000,000-agent cascade in the bench's launch configuration."""
    m = W.mapk(1_000_000)
    g = A.Sim(m, W.MAPK_SEED)
    o = oracle_mod.OracleSim(m, W.MAPK_SEED)
    for t in range(1, 9):
        g.step(1)
        o.step(1)
        assert g.digest() == o.digest(), f"step {t}"
    assert_same_dump(g.dump(), o.dump(), "step 8")
    assert np.array_equal(g.counts(), o.counts())


def test_nuclear_full_size_prefix(A, oracle_mod):
    m = W.nuclear(4_000_000)
    g = A.Sim(m, W.NUCLEAR_SEED)
    o = oracle_mod.OracleSim(m, W.NUCLEAR_SEED)
    assert g.digest() == o.digest()
    for t in range(1, 4):
        g.step(1)
        o.step(1)
        assert g.digest() == o.digest(), f"step {t}"
    assert np.array_equal(g.counts(), o.counts())


def test_nuclear_full_size_50_steps_against_the_oracle_record(A):
    """The two-compartment workload at 4M agents for 50 steps, digest after
    every step and counts every 10, against tests/golden/nuclear_4M_trace.txt,
    which tests/golden/make_nuclear_4M.py writes from the oracle alone (about
    20 s of oracle time per step)."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "nuclear_4M_trace.txt")) if not l.startswith("#")]
    want = {int(r[0]): (int(r[1], 16), [int(v) for v in r[2:]]) for r in rows}
    assert sorted(want) == list(range(51))
    g = A.Sim(W.nuclear(4_000_000), W.NUCLEAR_SEED)
    for t in range(51):
        if t:
            g.step(1)
        d, counts = want[t]
        assert g.digest() == d, f"step {t}"
        if counts:
            assert g.counts().tolist() == counts, f"step {t}"
    g.close()


def test_batch_members_equal_alone_and_oracle(A, oracle_mod):
    sims = [(W.mapk(8000 + 3000 * k, drug_frac=0.02 * k), 100 + k) for k in range(4)]
    sims.append((W.nuclear(12_000, boost=50.0, n_genes=16), 7))
    sims.append((W.toy(600, 500, edge_um=0.4), 3))
    cap = sum(m.n_agents for m, _ in sims) * 2 + 100_000
    b = A.Batch(cap, 4_000_000, 16)
    ids = [b.add(m, s) for m, s in sims]
    orcs = [oracle_mod.OracleSim(m, s) for m, s in sims]
    for t in range(6):
        b.step(20)
        for o in orcs:
            o.step(20)
        for sid, o in zip(ids, orcs):
            assert b.digest(sid) == o.digest(), f"sim {sid} step {20 * (t + 1)}"
    for sid, o in zip(ids, orcs):
        assert_same_dump(b.dump(sid), o.dump(), f"sim {sid}")
        assert np.array_equal(b.counts(sid), o.counts())
    b.close()


def test_batch_admission_and_removal_mid_run(A, oracle_mod):
    m1, m2, m3 = W.mapk(10_000), W.nuclear(9_000, boost=50.0, n_genes=8), W.mapk(7_000, drug_frac=0.0)
    b = A.Batch(200_000, 2_000_000, 4)
    s1 = b.add(m1, 11)
    b.step(30)
    s2 = b.add(m2, 22)
    b.step(30)
    b.remove(s1)
    b.step(1)
    s3 = b.add(m3, 33)                                        # may reuse s1's slot
    b.step(40)
    o2 = oracle_mod.OracleSim(m2, 22)
    o2.step(71)
    o3 = oracle_mod.OracleSim(m3, 33)
    o3.step(40)
    assert b.digest(s2) == o2.digest()
    assert b.digest(s3) == o3.digest()
    assert_same_dump(b.dump(s3), o3.dump(), "s3")
    b.close()


def test_torch_arena_and_stream(A, oracle_mod):
    import torch
    m = W.toy()
    nbytes = A.arena_bytes(m)
    arena = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    g = A.Sim(m, 1, arena=arena, stream=stream)
    g.step(30)
    o = oracle_mod.OracleSim(m, 1)
    o.step(30)
    assert g.digest() == o.digest()
    g.close()


def test_arena_too_small_or_misaligned_is_refused(A):
    import torch
    m = W.toy()
    nbytes = A.arena_bytes(m)
    small = torch.empty(nbytes - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(A.AbmError) as e:
        A.Sim(m, 1, arena=small)
    assert e.value.status == A.ENOMEM
    big = torch.empty(nbytes + 512, dtype=torch.uint8, device="cuda")
    with pytest.raises(A.AbmError) as e:
        A.Sim(m, 1, arena=big[16:])                         # not 256-byte aligned
    assert e.value.status == A.ENOMEM


def test_injected_launch_failure_leaves_a_destroyable_handle(A, oracle_mod):
    """Host-side failure injection: a step whose launch 'fails' returns ECUDA,
    the handle refuses further work (ESTATE) but is destroyed cleanly, and the
    device keeps working for other handles."""
    m = W.toy()
    g = A.Sim(m, 1)
    g.step(3)
    A.inject_launch_error(701)          # cudaErrorLaunchOutOfResources, reported, not raised on the device
    with pytest.raises(A.AbmError) as e:
        g.step(1)
    assert e.value.status == A.ECUDA and "injected" in str(e.value)
    with pytest.raises(A.AbmError) as e:
        g.counts()
    assert e.value.status == A.ESTATE
    g.close()
    h = A.Sim(m, 1)
    h.step(10)
    o = oracle_mod.OracleSim(m, 1)
    o.step(10)
    assert h.digest() == o.digest()
    h.close()


def test_edge_cases(A, oracle_mod):
    # no agents at all
    m = W.Model("empty", [W.Species("X", 0, 1.0)], [], [W.Compartment(W.CUBE, 1.0)])
    g = A.Sim(m, 1)
    g.step(5)
    o = oracle_mod.OracleSim(m, 1)
    o.step(5)
    assert g.digest() == o.digest() and list(g.counts()) == [0, 0]
    g.close()
    # one agent, immobile expressor creating a lineage of mobile dying children
    m = W.Model("one", [W.Species("G", 1, 0.0, p_emit=0.5, emit=1), W.Species("P", 0, 5.0, p_uni=0.05)], [],
                [W.Compartment(W.CUBE, 0.2)])
    _lockstep(A, oracle_mod, m, 9, 300, dump_every=50)
    # everything dies
    m = W.Model("die", [W.Species("X", 5000, 1.0, p_uni=0.3)], [], [W.Compartment(W.CUBE, 1.0)])
    c = _lockstep(A, oracle_mod, m, 2, 60, dump_every=20)
    assert c[0] == 0
    # p = 1 everywhere, CONVERT into death of both
    m = W.Model("burn", [W.Species("A", 3000, 1.0), W.Species("B", 3000, 1.0)],
                [W.Reaction(0, 1, W.CONVERT, -1, -1, 20.0, 1.0)], [W.Compartment(W.CUBE, 0.5)])
    _lockstep(A, oracle_mod, m, 4, 80, dump_every=20)
    # carrier is the acceptor b (smaller D), release kills the proposer
    m = W.Model("bcar", [W.Species("A", 3000, 5.0), W.Species("B", 3000, 1.0), W.Species("P", 0, 2.0)],
                [W.Reaction(0, 1, W.BIND, -1, 2, 15.0, 0.7, 0.2)], [W.Compartment(W.CUBE, 0.5)])
    _lockstep(A, oracle_mod, m, 6, 120, dump_every=30)
    # ragged: counts not a multiple of any tile, cells not a multiple of 4096
    m = W.Model("rag", [W.Species("A", 4097, 2.0), W.Species("B", 1, 2.0)],
                [W.Reaction(0, 1, W.BIND, 0, 1, 30.0, 1.0, 0.5)], [W.Compartment(W.CUBE, 0.77)])
    _lockstep(A, oracle_mod, m, 8, 100, dump_every=25)


def test_positions_near_the_extent_limit(A, oracle_mod):
    """A cube of 2,097,000 position units (209.7 um at 0.1 nm), just below the
    2^21 that the packed record holds per axis: positions use every bit of
    x, y and z, including those split across the record's first two words.
    A 2.5 um contact radius makes pairs react and bind across that domain."""
    m = W.Model("wide", [W.Species("A", 2500, 10.0), W.Species("B", 2500, 2.0), W.Species("C", 0, 1.0)],
                [W.Reaction(0, 1, W.BIND, 2, 1, 2500.0, 1.0, 0.1)], [W.Compartment(W.CUBE, 209.7)])
    c = _lockstep(A, oracle_mod, m, 11, 40, dump_every=10)
    n_sp = 3
    assert c[n_sp] > 0 or c[2] > 0                              # complexes formed or released
    g = A.Sim(m, 11)
    d = g.dump()
    g.close()
    assert d["x"].max() >= 1 << 20 and d["y"].max() >= 1 << 20 and d["z"].max() >= 1 << 20


def test_births_overflow_is_reported_not_written(A):
    m = W.Model("flood", [W.Species("G", 20_000, 0.0, p_emit=1.0, emit=1), W.Species("P", 0, 0.0)], [],
                [W.Compartment(W.CUBE, 2.0)])
    g = A.Sim(m, 1, births_per_step=1024)
    g.step(1)
    with pytest.raises(A.AbmError) as e:
        g.sync()
    assert e.value.status == A.ECAPACITY
    with pytest.raises(A.AbmError) as e:
        g.step(1)
    assert e.value.status == A.ESTATE
    g.close()


def test_capacity_overflow_is_reported(A):
    m = W.Model("grow", [W.Species("G", 1000, 0.0, p_emit=1.0, emit=1), W.Species("P", 0, 0.0)], [],
                [W.Compartment(W.CUBE, 2.0)])
    g = A.Sim(m, 1, capacity=4000)
    g.step(5)
    with pytest.raises(A.AbmError) as e:
        g.counts()
    assert e.value.status == A.ECAPACITY
    g.close()


def test_admission_right_after_removal_compacts(A, oracle_mod):
    """Capacity is only enough once the retired sim's agents are dropped:
    the admission compacts the arrays without stepping anything."""
    m1, m2, m3 = W.mapk(9_000), W.mapk(6_000, drug_frac=0.0), W.toy(900, 800, edge_um=0.5)
    cells = sum(A.model_grid(m)[1] for m in (m1, m2, m3))
    b = A.Batch(16_000, cells, 3)
    s1 = b.add(m1, 1)
    s2 = b.add(m2, 2)
    b.step(17)
    b.remove(s1)
    s3 = b.add(m3, 3)                      # 6k + 1.7k live, 9k retired: needs compaction
    b.step(23)
    o2 = oracle_mod.OracleSim(m2, 2)
    o2.step(40)
    o3 = oracle_mod.OracleSim(m3, 3)
    o3.step(23)
    assert b.digest(s2) == o2.digest()
    assert b.digest(s3) == o3.digest()
    b.close()


def test_admission_reuses_a_retired_slot_before_any_step(A, oracle_mod):
    """Every slot taken; retiring one frees it for an admission right away
    (the admission drops the retired agents itself), several times between
    two steps, as a server retiring and admitting jobs does."""
    toys = [W.toy(300 + 10 * k, 300, edge_um=0.4) for k in range(5)]
    cells = 2 * max(A.model_grid(m)[1] for m in toys)
    b = A.Batch(4_000, cells, 2)
    s0 = b.add(toys[0], 10)
    s1 = b.add(toys[1], 11)
    b.step(5)
    b.remove(s0)
    s2 = b.add(toys[2], 12)                # no step since the removal
    b.remove(s2)
    s3 = b.add(toys[3], 13)
    b.step(7)
    o1 = oracle_mod.OracleSim(toys[1], 11)
    o1.step(12)
    o3 = oracle_mod.OracleSim(toys[3], 13)
    o3.step(7)
    assert b.digest(s1) == o1.digest()
    assert b.digest(s3) == o3.digest()
    with pytest.raises(A.AbmError) as e:
        b.add(toys[4], 14)                 # both slots live: no slot
    assert e.value.status == A.ECAPACITY
    b.close()


@pytest.mark.parametrize("which", ["mapk", "nuclear"])
def test_checkpoint_restore_continues_bit_exact(A, oracle_mod, which):
    if which == "mapk":
        m, seed = W.mapk(25_000), 12
    else:
        m, seed = W.nuclear(20_000, boost=100.0, n_genes=16, genes_on=8), 42
    g = A.Sim(m, seed)
    g.step(60)
    rec, t, next_id = g.checkpoint()
    assert t == 60 and np.count_nonzero(rec["flags"] & 2) > 0
    r = A.Sim(m, seed, restore=(rec[::-1].copy(), t, next_id))   # any record order
    assert r.digest() == g.digest()
    g.step(70)
    r.step(70)
    assert r.digest() == g.digest()
    o = oracle_mod.OracleSim(m, seed)
    o.step(130)
    assert r.digest() == o.digest()
    assert_same_dump(r.dump(), o.dump(), "restored at 130")
    g.close()
    r.close()


def test_restore_rejects_inconsistent_records(A):
    m = W.mapk(10_000)
    g = A.Sim(m, 3)
    g.step(40)
    rec, t, next_id = g.checkpoint()
    g.close()
    bad = rec.copy()
    bad["id"][1] = bad["id"][0]                           # duplicate id
    with pytest.raises(A.AbmError):
        A.Sim(m, 3, restore=(bad, t, next_id))
    bad = rec.copy()
    bad["x"][0] = -5                                      # outside the domain
    with pytest.raises(A.AbmError):
        A.Sim(m, 3, restore=(bad, t, next_id))
    hid = np.nonzero(rec["flags"] & 2)[0]
    if len(hid):
        bad = np.delete(rec, hid[0])                      # a complex without its hidden partner
        with pytest.raises(A.AbmError):
            A.Sim(m, 3, restore=(bad, t, next_id))



def test_large_grid_takes_the_tile_prefix_kernel(A, oracle_mod):
    """A batch whose grid exceeds 8192 scan tiles (67M cells) computes the tile
    prefixes in k_tile_prefix instead of inside the scan: same results."""
    m = W.toy(700, 600, edge_um=0.5)
    b = A.Batch(200_000, 8193 * 8192, 2)
    s = b.add(m, 9)
    o = oracle_mod.OracleSim(m, 9)
    for t in range(4):
        b.step(10)
        o.step(10)
        assert b.digest(s) == o.digest(), f"step {10 * (t + 1)}"
    assert_same_dump(b.dump(s), o.dump(), "step 40")
    assert b.profile_step(1)["k_tile_prefix"] > 0
    b.close()
