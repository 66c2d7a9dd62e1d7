"""The oracle's initial placement, first-order events (P1), moves (P2) and
births (P6) against a per-agent brute force (CPU), a few steps from the
initial dump.

The statistical pins (binomial counts, mean squared displacement, wall and
membrane equilibria) fix rates and laws; these fix every draw.  Each test
predicts each agent's exact state from the readings that define the step:

  P1  a free agent draws e = Philox(key = seed, ctr = (id, t, 1, 0)); it
      converts (or dies) iff e[1] < floor(p_uni * 2^32), else emits one
      child iff e[2] < floor(p_emit * 2^32);
  P2  an agent of a species with M > 0 draws m = Philox(ctr = (id, t, 0, 0))
      and steps by d = sgn(Z) * ((|Z| * M + 2^31) >> 32) per axis, with
      Z = table[m[axis] >> 16] (x, y, z from words 0, 1, 2).  A cube folds
      about the half-integer walls (x < 0 -> -1 - x, x > L -> 2L + 1 - x).  A
      spherical cell rejects a move that ends outside it; a move that ends
      in another compartment (child spheres, boundary inclusive) is a
      crossing, kept iff m[3] < floor(p_cross * 2^32);
  P6  the step's children get ids next_id + k, k ranking their parents by
      id, at the parent's place and compartment.

Geometry: a cube root spans [0, L] with L = llround(edge * 1000 / unit); a
spherical root of diameter d has radius r = llround(d * 1000 / unit / 2),
spans [0, 2r] and is centred at (r, r, r); a child sphere is centred at that
centre plus llround(offset * 1000 / unit) per axis.  Shared with the oracle:
only the Philox primitive (pinned against cuRAND), the threshold and
multiplier helpers (pinned against exact arithmetic) and the Gaussian table
(pinned against NormalDist)."""
import math

import numpy as np
import pytest

import workloads as W


def _llround(x):
    return int(math.floor(x + 0.5)) if x >= 0 else -int(math.floor(-x + 0.5))


def _step(z, M):
    mag = (abs(int(z)) * M + (1 << 31)) >> 32
    return mag if z >= 0 else -mag


class _Geo:
    def __init__(self, model):
        root = model.compartments[0]
        u = model.unit_nm
        if root.shape == W.CUBE:
            self.sphere = False
            self.L = _llround(root.size_um * 1000.0 / u)
            self.c0 = (self.L // 2,) * 3
        else:
            self.sphere = True
            self.r = _llround(root.size_um * 1000.0 / u / 2.0)
            self.L = 2 * self.r
            self.c0 = (self.r,) * 3
        self.kids = [(tuple(self.c0[d] + _llround(c.center_um[d] * 1000.0 / u) for d in range(3)),
                      _llround(c.size_um * 1000.0 / u / 2.0)) for c in model.compartments[1:]]

    def locate(self, p):
        d2 = lambda c: sum((p[d] - c[d]) ** 2 for d in range(3))
        if self.sphere and d2(self.c0) > self.r * self.r:
            return -1
        for k, (c, r) in enumerate(self.kids, start=1):
            if d2(c) <= r * r:
                return k
        return 0

    def fold(self, v):
        if v < 0:
            return -1 - v
        if v > self.L:
            return 2 * self.L + 1 - v
        return v


def _predict(oracle_mod, model, seed, rec, steps):
    """Every agent's (species, compartment, x, y, z) after `steps` steps."""
    key = (seed & 0xFFFFFFFF, seed >> 32)
    thr = oracle_mod.threshold
    geo = _Geo(model)
    Z = oracle_mod.ncdf_table()
    M = [oracle_mod.mult(s.D, model.dt_s, model.unit_nm) for s in model.species]
    agents = {int(r["id"]): [int(r["sp"]), int(r["comp"]), int(r["x"]), int(r["y"]), int(r["z"])] for r in rec}
    next_id = max(agents) + 1
    for t in range(steps):
        # P1, in id order: conversions, deaths, emissions
        parents = []
        for i in sorted(agents):
            a = agents[i]
            sp = model.species[a[0]]
            e = oracle_mod.philox4x32_10((i, t, 1, 0), key)
            if e[1] < thr(sp.p_uni):
                if sp.uni_to >= 0:
                    a[0] = sp.uni_to
                else:
                    del agents[i]
            elif e[2] < thr(sp.p_emit):
                parents.append(i)
        # P2
        for i, a in agents.items():
            if M[a[0]] == 0:
                continue
            m = oracle_mod.philox4x32_10((i, t, 0, 0), key)
            q = [a[2 + d] + _step(Z[m[d] >> 16], M[a[0]]) for d in range(3)]
            if not geo.sphere:
                q = [geo.fold(v) for v in q]
            c = geo.locate(q)
            if c < 0:
                continue  # outside the spherical cell: rejected
            if c != a[1]:
                if m[3] >= thr(model.species[a[0]].p_cross):
                    continue  # membrane: rejected
                a[1] = c
            a[2:] = q
        # P6: children ranked by parent id, at the parent's place
        for k, pid in enumerate(sorted(parents)):
            p = agents.get(pid)
            assert p is not None  # a parent that emits did not die this step
            agents[next_id + k] = [model.species[p[0]].emit, p[1], p[2], p[3], p[4]]
        next_id += len(parents)
    return agents


def _oracle_run(oracle_mod, model, seed, steps):
    o = oracle_mod.OracleSim(model, seed)
    before = o.dump()
    o.step(steps)
    after = o.dump()
    o.close()
    got = {int(r["id"]): [int(r["sp"]), int(r["comp"]), int(r["x"]), int(r["y"]), int(r["z"])] for r in after}
    return before, got


def _moved_and_folded(before, got):
    b = {int(r["id"]): (int(r["x"]), int(r["y"]), int(r["z"])) for r in before}
    moved = sum(1 for i, a in got.items() if i in b and tuple(a[2:]) != b[i])
    return moved


@pytest.mark.parametrize("seed", [3, 77, 2 ** 33 + 5])
def test_moves_in_a_cube(oracle_mod, seed):
    # 0.2 um cube; sigma 2.4 nm and 1.1 nm per axis: a few dozen agents fold at a wall
    model = W.Model("cube_moves", [W.Species("X", 300, 3.0), W.Species("Y", 200, 0.6)], [],
                    [W.Compartment(W.CUBE, 0.2)])
    before, got = _oracle_run(oracle_mod, model, seed, 3)
    want = _predict(oracle_mod, model, seed, before, 3)
    assert got == want
    assert _moved_and_folded(before, got) >= 450
    L = _Geo(model).L
    near = sum(1 for r in before if min(r["x"], r["y"], r["z"], L - r["x"], L - r["y"], L - r["z"]) < 60)
    assert near >= 20  # the fold is exercised


@pytest.mark.parametrize("seed", [4, 91])
def test_moves_in_a_cell_with_a_nucleus(oracle_mod, seed):
    # 0.3 um spherical cell with an off-centre 0.15 um nucleus; sigma 3.2 nm
    # per axis: many moves leave the cell (rejected) or cross the membrane
    # (kept with probability 1/2 for P, never for R)
    cell = W.Compartment(W.SPHERE, 0.3)
    nucleus = W.Compartment(W.SPHERE, 0.15, parent=0, center_um=(0.02, -0.01, 0.0))
    species = [W.Species("P", 400, 5.0, comp=0, p_cross=0.5), W.Species("R", 300, 5.0, comp=1, p_cross=0.0),
               W.Species("S", 200, 5.0, comp=1, p_cross=0.5)]
    model = W.Model("cell_moves", species, [], [cell, nucleus])
    before, got = _oracle_run(oracle_mod, model, seed, 3)
    want = _predict(oracle_mod, model, seed, before, 3)
    assert got == want
    crossed = sum(1 for r in before if got[int(r["id"])][1] != int(r["comp"]))
    assert crossed >= 5  # membrane crossings happened (P and S), none for R
    assert all(got[int(r["id"])][1] == 1 for r in before if int(r["sp"]) == 1)


@pytest.mark.parametrize("seed", [5, 123])
def test_first_order_events_and_births(oracle_mod, seed):
    # immobile: U converts to V, Dd dies, E emits K, F converts (to V) or
    # else emits K (conversion wins in the same step), over three steps
    species = [W.Species("U", 200, 0.0, p_uni=0.3, uni_to=1), W.Species("V", 0, 0.0),
               W.Species("Dd", 200, 0.0, p_uni=0.2, uni_to=-1), W.Species("E", 200, 0.0, p_emit=0.4, emit=4),
               W.Species("K", 0, 0.0), W.Species("F", 200, 0.0, p_uni=0.25, uni_to=1, p_emit=0.5, emit=4)]
    model = W.Model("events", species, [], [W.Compartment(W.CUBE, 0.3)])
    before, got = _oracle_run(oracle_mod, model, seed, 3)
    want = _predict(oracle_mod, model, seed, before, 3)
    assert got == want
    sp = [a[0] for a in got.values()]
    assert sp.count(4) >= 100 and sp.count(1) >= 100 and sp.count(2) < 150  # births, conversions, deaths


def _placement(oracle_mod, model, seed):
    """Initial places: ids species-major; agent id draws
    w = Philox(ctr = (id, attempt, 0, 2)) for attempt = 0, 1, ... and takes
    ((w[0] * (L + 1)) >> 32, (w[1] * (L + 1)) >> 32, (w[2] * (L + 1)) >> 32)
    at the first attempt that lies in its species' compartment."""
    key = (seed & 0xFFFFFFFF, seed >> 32)
    geo = _Geo(model)
    out, i = {}, 0
    for s, sp in enumerate(model.species):
        for _ in range(sp.count):
            for attempt in range(1 << 16):
                w = oracle_mod.philox4x32_10((i, attempt, 0, 2), key)
                p = [(w[d] * (geo.L + 1)) >> 32 for d in range(3)]
                if geo.locate(p) == sp.comp:
                    out[i] = [s, sp.comp] + p
                    break
            i += 1
    return out


@pytest.mark.parametrize("seed", [1, 2 ** 36 + 3])
def test_initial_placement(oracle_mod, seed):
    cell = W.Compartment(W.SPHERE, 0.3)
    nucleus = W.Compartment(W.SPHERE, 0.15, parent=0, center_um=(0.02, -0.01, 0.0))
    for model in (W.Model("cube", [W.Species("X", 300, 1.0), W.Species("Y", 200, 1.0)], [],
                          [W.Compartment(W.CUBE, 0.2)]),
                  W.Model("cell", [W.Species("P", 400, 1.0, comp=0), W.Species("R", 300, 1.0, comp=1)], [],
                          [cell, nucleus])):
        o = oracle_mod.OracleSim(model, seed)
        got = {int(r["id"]): [int(r["sp"]), int(r["comp"]), int(r["x"]), int(r["y"]), int(r["z"])]
               for r in o.dump()}
        o.close()
        assert got == _placement(oracle_mod, model, seed), model.name
