"""Pins of the serial oracle against things other than itself.

Each test ties one part of the oracle to a library routine, a closed form, an
invariant or a brute-force computation, chosen so that a plausible slip (a
dropped term, a wrong sign or index, a swapped operand) fails at least one:

  Philox            cuRAND's host Philox4x32-10 generator (run, not read)
  Gaussian table    Python's statistics.NormalDist.inv_cdf (FP64, AS241)
  thresholds        exact rational arithmetic (fractions.Fraction)
  move              mean squared displacement = 3 n E[d^2] and E[d^2] = 2 D dt
  axes / streams    zero correlation between axes and with the event block
  mirror / sphere   uniform measure stays uniform (exact stationarity)
  membrane          crossing equilibrium = lattice-volume ratio
  neighbour search  brute-force O(N^2) proposals give identical trajectories
  bookkeeping       stoichiometric conservation and per-id species families
  first order       binomial counts of conversions, deaths and births
  births            ids ranked by parent id; child at the parent's position
  bimolecular rate  Smoluchowski / Spitzer mean-sausage closed form
"""
import ctypes
import math
import os
from fractions import Fraction
from statistics import NormalDist

import numpy as np
import pytest

import workloads as W


# --------------------------------------------------------------------------
def _curand():
    names = ["libcurand.so", "libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so"]
    for n in names:
        try:
            return ctypes.CDLL(n)
        except OSError:
            continue
    pytest.skip("libcurand not found")


def _curand_host_blocks(seed, n_blocks):
    """cuRAND's host Philox4x32-10 generator: output block j is
    Philox(counter=(0, 0, j, 0), key=(seed lo, seed hi))."""
    cr = _curand()
    gen = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = (ctypes.c_uint32 * (4 * n_blocks))()
        assert cr.curandGenerate(gen, out, ctypes.c_size_t(4 * n_blocks)) == 0
        return np.frombuffer(out, dtype=np.uint32).reshape(n_blocks, 4)
    finally:
        cr.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 1, 12, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 2**32 + 7])
def test_philox_matches_curand_host(oracle_mod, seed):
    ref = _curand_host_blocks(seed, 300)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in list(range(40)) + [123, 299]:
        assert oracle_mod.philox4x32_10([0, 0, j, 0], key) == ref[j].tolist()


def test_philox_counter_words_all_matter(oracle_mod):
    base = oracle_mod.philox4x32_10([5, 6, 7, 8], [9, 10])
    for w in range(4):
        c = [5, 6, 7, 8]
        c[w] ^= 1
        assert oracle_mod.philox4x32_10(c, [9, 10]) != base
    assert oracle_mod.philox4x32_10([5, 6, 7, 8], [9, 11]) != base


# --------------------------------------------------------------------------
def test_ncdf_table_matches_normaldist(oracle_mod):
    tab = oracle_mod.ncdf_table()
    nd = NormalDist()
    ref = np.array([math.floor(abs(4096 * nd.inv_cdf((i + 0.5) / 65536)) + 0.5) *
                    (1 if i >= 32768 else -1) for i in range(65536)])
    assert np.array_equal(tab.astype(np.int64), ref)
    assert np.all(np.diff(tab.astype(np.int64)) >= 0)
    assert np.array_equal(tab[::-1].astype(np.int64), -tab.astype(np.int64))
    # the table is a discretised standard normal: variance ~ 4096^2
    var = np.mean((tab.astype(np.float64) / 4096.0) ** 2)
    assert abs(var - 1.0) < 2e-3


def test_threshold_exact(oracle_mod):
    assert oracle_mod.threshold(0.0) == 0
    assert oracle_mod.threshold(1.0) == 2 ** 32
    assert oracle_mod.threshold(0.5) == 2 ** 31
    rng = np.random.default_rng(5)
    for p in list(rng.random(200)) + [1e-3, 1e-9, 0.999999999, 2 ** -32, 2 ** -33]:
        exact = math.floor(Fraction(float(p)) * 2 ** 32)
        assert oracle_mod.threshold(float(p)) == exact


def test_gauss_step_second_moment_is_2Ddt(oracle_mod):
    tab = oracle_mod.ncdf_table().astype(np.int64)
    for D, dt in [(1.0, 1e-6), (10.0, 1e-6), (3.0, 3.125e-6), (0.1, 1e-5)]:
        m = oracle_mod.mult(D, dt, 0.1)
        d = np.array([oracle_mod.gauss_step(int(z), m) for z in tab[::7]])
        assert np.array_equal(d, -np.array([oracle_mod.gauss_step(int(-z), m) for z in tab[::7]]))
        e2 = np.mean(d.astype(np.float64) ** 2) * (0.1e-3) ** 2        # um^2 per axis
        assert abs(e2 - 2 * D * dt) / (2 * D * dt) < 2e-3


def _exact_mult(D, dt, unit):
    """2^20 * sqrt(2 D dt) * 1000 / unit as an exact value of the binary
    inputs (rational arithmetic, the square root to 60 digits), returned with
    its distance to the nearest rounding boundary (a half integer)."""
    import decimal
    from fractions import Fraction
    decimal.getcontext().prec = 60
    var = Fraction(D) * Fraction(dt) * 2                     # um^2, exact
    root = decimal.Decimal(var.numerator).sqrt() / decimal.Decimal(var.denominator).sqrt()
    scale = Fraction(1000) * Fraction(2 ** 20) / Fraction(unit)
    v = root * decimal.Decimal(scale.numerator) / decimal.Decimal(scale.denominator)
    frac = v - int(v)
    return v, abs(frac - decimal.Decimal("0.5"))


def test_mult_is_the_nearest_integer_of_its_definition(oracle_mod):
    """M = round(2^20 * sigma / unit) with sigma = sqrt(2 D dt) (Sec. 2:
    Brownian displacement from the diffusion coefficient; the fixed-point
    reading of the step size).  Checked against exact arithmetic, not the
    oracle's own floating-point order: over the workloads' coefficients and
    2,000 random (D, dt, unit), M is the nearest integer of the exact value
    (ties are not met: every case lies more than 1e-6 from a half integer),
    halves are rounded away from zero, and a mistake such as a missing
    factor 2, sigma^2 instead of sigma, or truncation instead of rounding
    fails here."""
    import decimal
    rng = np.random.default_rng(20261204)
    cases = [(D, 1e-6, 0.1) for D in (0.1, 1.0, 2.0, 3.0, 4.0, 10.0)]
    cases += [(float(10 ** rng.uniform(-3, 2)), float(10 ** rng.uniform(-7, -4)),
               float(rng.choice([0.05, 0.1, 0.25, 1.0]))) for _ in range(2000)]
    truncations_differ = 0
    for D, dt, unit in cases:
        v, gap = _exact_mult(D, dt, unit)
        assert gap > decimal.Decimal("1e-6"), (D, dt, unit)
        want = int(v.to_integral_value(rounding=decimal.ROUND_HALF_UP))
        got = oracle_mod.mult(D, dt, unit)
        assert got == want, (D, dt, unit, got, str(v))
        truncations_differ += int(v) != want
    assert truncations_differ > 500          # the cases do tell rounding from truncation
    # a worked value: D = 1 um^2/s, dt = 1 us, 0.1 nm units: sigma = 1.41421356 nm
    # = 14.1421356 units; 2^20 * 14.1421356237... = 14,829,104.004 -> 14,829,104
    assert oracle_mod.mult(1.0, 1e-6, 0.1) == 14_829_104


# --------------------------------------------------------------------------
def _exact_e2(oracle_mod, m):
    tab = oracle_mod.ncdf_table().astype(np.int64)
    mags = np.unique(np.abs(tab), return_counts=True)
    tot = 0.0
    for z, c in zip(*mags):
        tot += c * float(oracle_mod.gauss_step(int(z), m)) ** 2
    return tot / 65536.0


def test_msd_free_diffusion(oracle_mod):
    n, steps, D, dt = 100_000, 20, 1.0, 1e-6
    m = W.Model("free", [W.Species("X", n, D)], [], [W.Compartment(W.CUBE, 100.0)], dt_s=dt)
    sim = oracle_mod.OracleSim(m, 77)
    d0 = sim.dump()
    sim.step(steps)
    d1 = sim.dump()
    assert np.array_equal(d0["id"], d1["id"])
    dx = np.stack([(d1[k].astype(np.int64) - d0[k]) for k in "xyz"], 1).astype(np.float64)
    e2 = _exact_e2(oracle_mod, oracle_mod.mult(D, dt, 0.1))
    msd = np.mean(np.sum(dx ** 2, 1))
    expect = 3 * steps * e2
    assert abs(msd / expect - 1) < 4 * math.sqrt(2.0 / (3 * n))
    # mean zero per axis, uncorrelated axes
    for k in range(3):
        assert abs(dx[:, k].mean()) < 4 * math.sqrt(steps * e2 / n)
    c = np.corrcoef(dx.T)
    assert np.max(np.abs(c - np.eye(3))) < 4 / math.sqrt(n)
    # 6 D t in um^2
    assert abs(expect * 1e-8 - 6 * D * dt * steps) / (6 * D * dt * steps) < 2e-3


def test_move_independent_of_event_draw(oracle_mod):
    # species X converts to Y with p = 1/2; the displacement of the step must
    # not depend on whether the conversion fired (separate Philox blocks)
    n = 100_000
    m = W.Model("ev", [W.Species("X", n, 1.0, p_uni=0.5, uni_to=1), W.Species("Y", 0, 1.0)], [],
                [W.Compartment(W.CUBE, 100.0)])
    sim = oracle_mod.OracleSim(m, 5)
    d0 = sim.dump()
    sim.step(1)
    d1 = sim.dump()
    conv = d1["sp"] == 1
    assert abs(conv.mean() - 0.5) < 4 * math.sqrt(0.25 / n)
    dx = (d1["x"].astype(np.int64) - d0["x"]).astype(np.float64)
    for sel in (conv, ~conv):
        assert abs(np.mean(dx[sel] ** 2) / np.mean(dx ** 2) - 1) < 4 * math.sqrt(2.0 / sel.sum()) + 1e-3


# --------------------------------------------------------------------------
def test_mirror_keeps_uniform(oracle_mod):
    n, L = 200_000, 10_000
    m = W.Model("box", [W.Species("X", n, 10.0)], [], [W.Compartment(W.CUBE, 1.0)])
    sim = oracle_mod.OracleSim(m, 9)
    sim.step(200)
    d = sim.dump()
    for k in "xyz":
        v = d[k].astype(np.int64)
        assert v.min() >= 0 and v.max() <= L
        # every lattice value has probability 1/(L+1): no pile-up at the walls
        p = 1.0 / (L + 1)
        for wall in (0, L):
            cnt = np.sum(v == wall)
            assert cnt < n * p + 6 * math.sqrt(n * p) + 3
        # a band of 2 sigma at each wall holds its uniform share
        band = 90
        cnt = np.sum(v < band) + np.sum(v > L - band)
        ex = n * 2 * band / (L + 1)
        assert abs(cnt - ex) < 4.5 * math.sqrt(ex)
        hist, _ = np.histogram(v, bins=20, range=(0, L + 1))
        ex = n / 20
        chi2 = np.sum((hist - ex) ** 2 / ex)
        assert chi2 < 50                                      # 19 dof


def test_sphere_rejection_keeps_uniform(oracle_mod):
    n = 100_000
    m = W.Model("sph", [W.Species("X", n, 10.0)], [], [W.Compartment(W.SPHERE, 1.0)])
    sim = oracle_mod.OracleSim(m, 10)
    sim.step(100)
    d = sim.dump()
    r = 5000
    r2 = sum((d[k].astype(np.int64) - r) ** 2 for k in "xyz")
    assert r2.max() <= r * r
    inner = np.mean(r2 <= (r // 2) ** 2)                     # volume fraction 1/8
    assert abs(inner - 0.125) < 4 * math.sqrt(0.125 * 0.875 / n)
    shell = np.mean(r2 > (0.95 * r) ** 2)                     # 1 - 0.95^3
    ex = 1 - 0.95 ** 3
    assert abs(shell - ex) < 4 * math.sqrt(ex * (1 - ex) / n)


def test_membrane_crossing_equilibrium(oracle_mod):
    # all start in the cytoplasm; with rejection and a symmetric crossing
    # probability the lattice-uniform measure is stationary, so the nuclear
    # share relaxes to (lattice points in nucleus) / (lattice points in cell)
    n = 5000
    m = W.Model("cross", [W.Species("X", n, 10.0, comp=0, p_cross=0.5)], [],
                [W.Compartment(W.SPHERE, 0.4), W.Compartment(W.SPHERE, 0.2, parent=0)], dt_s=1e-5)
    sim = oracle_mod.OracleSim(m, 11)
    assert sim.counts()[1] == 0
    fr = []
    for _ in range(6):
        sim.step(300)
        c = sim.counts()
        fr.append(c[1] / n)
    d = sim.dump()
    r2c = sum((d[k].astype(np.int64) - 2000) ** 2 for k in "xyz")
    assert np.all((r2c <= 1000 ** 2) == (d["comp"] == 1))       # compartment = geometry
    ratio = 1000 ** 3 / 2000 ** 3
    late = np.mean(fr[3:])
    assert abs(late - ratio) < 4 * math.sqrt(ratio * (1 - ratio) / n)
    assert fr[0] > 0.02                                          # crossings happen early


def test_no_crossing_without_probability(oracle_mod):
    n = 3000
    m = W.Model("nocross", [W.Species("X", n, 10.0, comp=0), W.Species("Y", n, 10.0, comp=1)], [],
                [W.Compartment(W.SPHERE, 0.4), W.Compartment(W.SPHERE, 0.2, parent=0)], dt_s=1e-5)
    sim = oracle_mod.OracleSim(m, 12)
    sim.step(300)
    c = sim.counts()
    assert c[0] == n and c[1] == 0 and c[2] == 0 and c[3] == n


# --------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["toy", "mapk", "nuclear"])
def test_cell_list_matches_brute_force(oracle_mod, which):
    if which == "toy":
        m, seed, steps = W.toy(400, 400, edge_um=0.3), 1, 60
    elif which == "mapk":
        m, seed, steps = W.mapk(1500, edge_um=0.25), 12, 60
    else:
        m, seed, steps = W.nuclear(1500, boost=200.0, n_genes=8), 42, 60
    a = oracle_mod.OracleSim(m, seed)
    b = oracle_mod.OracleSim(m, seed, brute_force=True)
    for _ in range(steps // 10):
        a.step(10)
        b.step(10)
        assert a.digest() == b.digest()
        assert np.array_equal(a.counts(), b.counts())
    bound = a.counts()[len(m.species) * len(m.compartments):-1]
    assert bound.sum() + a.counts()[2] > 0 or which == "toy"


# --------------------------------------------------------------------------
def test_toy_conservation(oracle_mod):
    sim = oracle_mod.OracleSim(W.toy(), W.TOY_SEED)
    for _ in range(20):
        sim.step(10)
        c = sim.counts()
        assert c[0] + c[2] == 2500 and c[1] + c[2] == 2500
    assert c[2] > 50


def _families_conserved(model, counts):
    """Left-null-space invariants of the cascade: BRAF*, drug, phosphatase,
    MEK family and ERK family totals, counting the members held in complexes."""
    n_sp, n_c = len(model.species), len(model.compartments)
    free = counts[: n_sp * n_c].reshape(n_sp, n_c).sum(1)
    bound = counts[n_sp * n_c: -1]
    fams = {"BRAF": [0], "D": [1], "MEK": [2, 3, 4], "ERK": [5, 6, 7], "PP": [8]}
    tot = {}
    for f, mem in fams.items():
        v = int(sum(free[s] for s in mem))
        for r, rx in enumerate(model.reactions):
            v += int(bound[r]) * ((rx.a in mem) + (rx.b in mem))
        tot[f] = v
    return tot


def test_mapk_conservation_and_families(oracle_mod):
    m = W.mapk(30_000)
    sim = oracle_mod.OracleSim(m, 12)
    fam0 = _families_conserved(m, sim.counts())
    d0 = sim.dump()
    fam_of = {0: 0, 1: 1, 2: 2, 3: 2, 4: 2, 5: 3, 6: 3, 7: 3, 8: 4}
    start = {int(i): fam_of[int(s)] for i, s in zip(d0["id"], d0["sp"])}
    binds = 0
    for _ in range(8):
        sim.step(25)
        c = sim.counts()
        assert _families_conserved(m, c) == fam0
        binds += int(c[9:-1].sum())
        d = sim.dump()
        assert len(d) == m.n_agents
        for i, s in zip(d["id"].tolist(), d["sp"].tolist()):
            assert start[i] == fam_of[s]
        # a complex is one carrier and one hidden partner at the same place
        car = d[(d["flags"] & 1) == 1]
        hid = d[(d["flags"] & 2) == 2]
        assert len(car) == len(hid)
        hid_by_id = {int(h["id"]): h for h in hid}
        for cr in car:
            h = hid_by_id[int(cr["partner"])]
            assert int(h["partner"]) == int(cr["id"]) and h["rxn"] == cr["rxn"]
            assert (h["x"], h["y"], h["z"], h["comp"]) == (cr["x"], cr["y"], cr["z"], cr["comp"])
            rx = m.reactions[int(cr["rxn"])]
            ca, ha = bool(cr["flags"] & 4), bool(h["flags"] & 4)
            assert ca != ha
            assert int(cr["sp"]) == (rx.a if ca else rx.b) and int(h["sp"]) == (rx.a if ha else rx.b)
            # carrier: the smaller diffusion coefficient, ties to the proposer
            Da, Db = m.species[rx.a].D, m.species[rx.b].D
            assert ca == (not (Db < Da))
    assert binds > 0
    # products were released: pMEK / pERK appear
    assert c[3] + c[6] > 0


# --------------------------------------------------------------------------
def test_first_order_binomial(oracle_mod):
    n, p, steps = 100_000, 0.01, 10
    m = W.Model("uni", [W.Species("X", n, 1.0, p_uni=p, uni_to=1), W.Species("Y", 0, 1.0, p_uni=p, uni_to=-1)],
                [], [W.Compartment(W.CUBE, 20.0)])
    sim = oracle_mod.OracleSim(m, 3)
    sim.step(steps)
    c = sim.counts()
    q = (1 - p) ** steps
    assert abs(c[0] - n * q) < 4.5 * math.sqrt(n * q * (1 - q))
    # X -> Y -> death chain: P(Y alive at t) = t p (1-p)^(t-1)
    py = steps * p * (1 - p) ** (steps - 1)
    assert abs(c[1] - n * py) < 4.5 * math.sqrt(n * py * (1 - py))
    assert sim.n_agents == c[0] + c[1]
    assert c[-1] == n                                       # no births: next_id fixed


def test_emission_binomial_ids_and_places(oracle_mod):
    n, p = 20_000, 0.02
    m = W.Model("emit", [W.Species("G", n, 0.0, p_emit=p, emit=1), W.Species("P", 0, 0.0)], [],
                [W.Compartment(W.CUBE, 20.0)])
    sim = oracle_mod.OracleSim(m, 4)
    d0 = sim.dump()
    pos = {(int(r["x"]), int(r["y"]), int(r["z"])): int(r["id"]) for r in d0}
    assert len(pos) == n
    total = 0
    for _ in range(5):
        before = sim.counts()[-1]
        sim.step(1)
        d = sim.dump()
        new = d[d["id"] >= before]
        total += len(new)
        assert sim.counts()[-1] == before + len(new)
        parents = [pos[(int(r["x"]), int(r["y"]), int(r["z"]))] for r in new]
        assert parents == sorted(parents) and len(set(parents)) == len(parents)
        assert np.all(new["sp"] == 1)
    ex = n * 5 * p
    assert abs(total - ex) < 4.5 * math.sqrt(ex * (1 - p))


def test_bound_hold_is_geometric_and_immune(oracle_mod):
    """Immobile E + S bind (E carries: equal D, tie to the proposer) and release
    E + P with probability q per step: complex lifetimes are geometric with
    parameter q, and a bound E never dies although free E dies at rate 0.2."""
    n, q = 20_000, 0.05
    m = W.Model("hold", [W.Species("E", n, 0.0, p_uni=0.2, uni_to=-1), W.Species("S", n, 0.0),
                         W.Species("P", 0, 0.0)],
                [W.Reaction(0, 1, W.BIND, 0, 2, 30.0, 1.0, q)], [W.Compartment(W.CUBE, 1.2)])
    sim = oracle_mod.OracleSim(m, 8)
    sim.step(1)
    prev = {}
    at_risk = releases = 0
    for it in range(40):
        d = sim.dump()
        alive = set(d["id"].tolist())
        cur = {(int(r["id"]), int(r["partner"])) for r in d[(d["flags"] & 1) == 1]}
        for (c, h) in prev:
            assert c in alive and h in alive           # nobody in a complex dies
            at_risk += 1
            if (c, h) not in cur:
                releases += 1
        for r in d[(d["flags"] & 1) == 1]:
            assert r["sp"] == 0
        prev = cur
        if it < 39:
            sim.step(1)
    qhat = releases / at_risk
    assert at_risk > 50_000
    assert abs(qhat - q) < 4 * math.sqrt(q * (1 - q) / at_risk)
    assert sim.counts()[2] == releases                # every release makes one P


def test_smoluchowski_rate(oracle_mod):
    """Sparse mobile A among immobile, Poisson-placed traps B of density c:
    the fraction of A that has hit a trap by time t tends, as dt -> 0, to
    1 - exp(-c E|W_R(t)|) with Spitzer's mean Wiener-sausage volume
    E|W_R(t)| = 4/3 pi R^3 + 4 pi D R t + 8 R^2 sqrt(pi D t); its time
    derivative is the Smoluchowski rate 4 pi D R (1 + R / sqrt(pi D t)).
    Discrete-time contact checks miss excursions between steps, so the count
    approaches the closed form from below with a bias of order
    rho = sqrt(2 D dt) / R."""
    nA, cB, edge, R_nm, D, T = 20_000, 100.0, 5.0, 50.0, 1.0, 1e-3
    R = R_nm * 1e-3
    L = int(round(edge * 1e4))
    margin = 3000                               # > 6 sigma of travel in T
    out = {}
    for rho in (0.2, 0.1, 0.05):
        dt = (rho * R) ** 2 / (2 * D)
        steps = int(round(T / dt))
        nB = int(round(cB * edge ** 3))
        m = W.Model("smol", [W.Species("A", nA, D), W.Species("B", nB, 0.0), W.Species("C", 0, D)],
                    [W.Reaction(0, 1, W.CONVERT, 2, 1, R_nm, 1.0)], [W.Compartment(W.CUBE, edge)], dt_s=dt)
        sim = oracle_mod.OracleSim(m, 3)
        d0 = sim.dump()
        a0 = d0[d0["sp"] == 0]
        inner = a0["id"][np.all([(a0[k] > margin) & (a0[k] < L - margin) for k in "xyz"], axis=0)]
        sim.step(steps)
        d = sim.dump()
        F = np.isin(inner, d["id"][d["sp"] == 2]).mean()
        t = steps * dt
        EW = 4 / 3 * math.pi * R ** 3 + 4 * math.pi * D * R * t + 8 * R * R * math.sqrt(math.pi * D * t)
        Fc = 1 - math.exp(-cB * EW)
        out[rho] = (F, Fc, len(inner))
    F2, F1, F05 = out[0.2][0], out[0.1][0], out[0.05][0]
    Fc, n = out[0.05][1], out[0.05][2]
    sig = math.sqrt(Fc * (1 - Fc) / n)
    assert F2 < F1 < F05 < Fc + 3 * sig                      # approaches from below
    assert Fc * (1 - 1.5 * 0.05) - 3 * sig < F05            # bias allowance 1.5 rho
    extrap = 2 * F05 - F1                                    # first-order Richardson
    assert abs(extrap - Fc) < 3 * math.sqrt(5) * sig


# --------------------------------------------------------------------------
def test_initial_placement(oracle_mod):
    m = W.nuclear(20_000, n_genes=16)
    sim = oracle_mod.OracleSim(m, 42)
    d = sim.dump()
    assert np.array_equal(d["id"], np.arange(m.n_agents))
    starts = np.cumsum([0] + [s.count for s in m.species])
    for i, s in enumerate(m.species):
        seg = d[starts[i]:starts[i + 1]]
        assert np.all(seg["sp"] == i) and np.all(seg["comp"] == s.comp)
    r = int(round(m.compartments[0].size_um * 1e4 / 2))
    rn = int(round(m.compartments[1].size_um * 1e4 / 2))
    r2 = sum((d[k].astype(np.int64) - r) ** 2 for k in "xyz")
    assert np.all(r2 <= r * r)
    assert np.all((r2 <= rn * rn) == (d["comp"] == 1))
    # cytoplasm agents uniform in the shell: share beyond the mid radius
    cy = d["comp"] == 0
    rm = (r ** 3 + rn ** 3) / 2
    frac = np.mean(r2[cy] ** 1.5 > rm)
    ncy = cy.sum()
    assert abs(frac - 0.5) < 4 * math.sqrt(0.25 / ncy)


@pytest.mark.parametrize("bad", ["aa", "dup", "rev", "prob", "radius", "species", "child"])
def test_invalid_models_rejected(oracle_mod, bad):
    m = W.toy()
    if bad == "aa":
        m.reactions = [W.Reaction(0, 0, W.CONVERT, 2, 2, 5.0, 1.0)]
    elif bad == "dup":
        m.reactions = m.reactions * 2
    elif bad == "rev":
        m.reactions = m.reactions + [W.Reaction(1, 0, W.CONVERT, 2, 2, 5.0, 1.0)]
    elif bad == "prob":
        m.reactions[0].p_bind = 1.5
    elif bad == "radius":
        m.reactions[0].radius_nm = 0.0
    elif bad == "species":
        m.reactions[0].prod_a = 7
    else:
        m.compartments = [W.Compartment(W.CUBE, 1.0), W.Compartment(W.SPHERE, 2.0, parent=0)]
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.OracleSim(m, 1)


def test_golden_toy_trace(oracle_mod):
    """Regression fixture written by tests/golden/make_golden.py (oracle only)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "toy_trace.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    sim = oracle_mod.OracleSim(W.toy(), W.TOY_SEED)
    t = 0
    for row in rows:
        step = int(row[0])
        sim.step(step - t)
        t = step
        assert format(sim.digest(), "016x") == row[1]
        assert [int(v) for v in row[2:]] == sim.counts().tolist()
