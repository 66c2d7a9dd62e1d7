"""The oracle's proposal and acceptance phases against a brute force (CPU).

With every species immobile (D = 0) and no first-order events, one step is
exactly P4 (proposals) followed by P5 (acceptance and application), on the
positions of the initial dump.  This file derives that step independently,
by brute force over all pairs, from the readings that define it:

  P4  a free agent of a reaction's species a proposes to the free agent b
      that minimises (dist^2, id_b) among those in the same compartment,
      with a reaction (a, b), dist^2 <= R^2 (R = llround(radius_nm / unit))
      and the pair draw Philox(key = seed, ctr = (min id, max id, t, 1)).x
      below floor(p_bind * 2^32);
  P5  acc[b] = min over b's proposers of (dist^2, id_a); the edge a -> b is
      final iff acc[b] names a and nobody proposed to a.  CONVERT turns a
      and b into their products (-1: gone).  BIND forms a complex whose
      carrier is the reactant with the smaller D, ties to the proposer: the
      carrier is flagged bound (1), plus role a (4) if it is the proposer;
      the other is hidden (2), plus 4 if it is the proposer; each names the
      other as partner and the hidden one sits at the carrier's place.

The brute force shares only the Philox primitive (pinned separately against
cuRAND) and the threshold helper (pinned against exact rationals) with the
oracle.  At this density most acceptors receive several proposals and many
proposers are proposed to, so the final-edge rule decides most outcomes.
This pins the oracle's implementation of the conflict rule; the rule itself
is a reading of the paper, which says only that molecules bind by
proximity."""
import math

import numpy as np
import pytest

import workloads as W

A, B, C, Q = 0, 1, 2, 3


def _model():
    species = [W.Species("A", 150, 0.0), W.Species("B", 150, 0.0), W.Species("C", 0, 0.0),
               W.Species("Q", 150, 0.0)]
    reactions = [W.Reaction(A, B, W.CONVERT, C, -1, 5.0, 0.7),
                 W.Reaction(Q, B, W.BIND, Q, B, 4.0, 0.8, 0.0),
                 W.Reaction(A, Q, W.CONVERT, C, C, 5.0, 0.6)]
    return W.Model(name="dense_static", species=species, reactions=reactions,
                   compartments=[W.Compartment(W.CUBE, 0.04)])


def _llround(x):
    return int(math.floor(x + 0.5)) if x >= 0 else -int(math.floor(-x + 0.5))


def _brute_force_step(oracle_mod, model, seed, rec, t=0):
    """Expected {id: (species or None if gone, flags, partner, reaction)}
    after P4 + P5 of step t among the free agents in rec."""
    key = (seed & 0xFFFFFFFF, seed >> 32)
    ids = rec["id"].astype(np.int64)
    sp = rec["sp"].astype(np.int64)
    comp = rec["comp"].astype(np.int64)
    pos = np.stack([rec["x"], rec["y"], rec["z"]], axis=1).astype(np.int64)
    assert (rec["flags"] == 0).all()  # everyone free at t = 0
    rx = {(r.a, r.b): (k, r) for k, r in enumerate(model.reactions)}
    n = len(ids)
    d2 = ((pos[:, None, :] - pos[None, :, :]) ** 2).sum(axis=2)
    best = {}  # proposer index -> (d2, id_b, b index, reaction index)
    for i in range(n):
        for j in range(n):
            if i == j or comp[i] != comp[j] or (sp[i], sp[j]) not in rx:
                continue
            k, r = rx[(sp[i], sp[j])]
            R = _llround(r.radius_nm / model.unit_nm)
            if d2[i, j] > R * R:
                continue
            lo, hi = min(ids[i], ids[j]), max(ids[i], ids[j])
            u = oracle_mod.philox4x32_10((lo, hi, t, 1), key)[0]
            if u >= oracle_mod.threshold(r.p_bind):
                continue
            cand = (int(d2[i, j]), int(ids[j]), j, k)
            if i not in best or cand[:2] < best[i][:2]:
                best[i] = cand
    acc = {}  # acceptor index -> (d2, id_a, proposer index)
    for i, (dd, _, j, _) in best.items():
        if j not in acc or (dd, int(ids[i])) < acc[j][:2]:
            acc[j] = (dd, int(ids[i]), i)
    out = {int(ids[i]): (int(sp[i]), 0, None, None) for i in range(n)}
    n_final = 0
    for i, (dd, _, j, k) in best.items():
        if acc[j][2] != i or i in acc:  # not the acceptor's choice, or proposed to itself
            continue
        n_final += 1
        r = model.reactions[k]
        ia, ib = int(ids[i]), int(ids[j])
        if r.kind == W.CONVERT:
            out[ia] = (r.prod_a if r.prod_a >= 0 else None, 0, None, None)
            out[ib] = (r.prod_b if r.prod_b >= 0 else None, 0, None, None)
        else:
            Da, Db = model.species[sp[i]].D, model.species[sp[j]].D
            if Da <= Db:  # the proposer carries (ties included)
                out[ia] = (int(sp[i]), 1 | 4, ib, k)
                out[ib] = (int(sp[j]), 2, ia, k)
            else:
                out[ib] = (int(sp[j]), 1, ia, k)
                out[ia] = (int(sp[i]), 2 | 4, ib, k)
    stats = {"proposals": len(best), "final": n_final,
             "contested": sum(1 for j in acc if sum(1 for v in best.values() if v[2] == j) > 1),
             "blocked": sum(1 for i in best if i in acc)}
    return out, stats


def _state(rec):
    return {int(r["id"]): {"sp": int(r["sp"]), "comp": int(r["comp"]), "flags": int(r["flags"]),
                           "partner": int(r["partner"]), "rxn": int(r["rxn"]),
                           "pos": (int(r["x"]), int(r["y"]), int(r["z"]))} for r in rec}


def _release_then_pair(oracle_mod, model, seed, state, t):
    """One step of immobile agents from `state` (possibly with complexes):
    P1 releases (a carrier draws e = Philox(ctr = (id, t, 1, 0)) and lets go
    iff e[0] < floor(p_release * 2^32); the carrier takes its reaction's
    product for its role and the hidden partner the other, at the carrier's
    place, both free), then P4 + P5 among the free agents."""
    key = (seed & 0xFFFFFFFF, seed >> 32)
    st = {i: dict(a) for i, a in state.items()}
    n_released = 0
    for i in sorted(st):
        a = st[i]
        if not a["flags"] & 1:
            continue  # only carriers draw (hidden partners have no events)
        r = model.reactions[a["rxn"]]
        if oracle_mod.philox4x32_10((i, t, 1, 0), key)[0] >= oracle_mod.threshold(r.p_release):
            continue
        h = st[a["partner"]]
        carrier_is_a = bool(a["flags"] & 4)
        a_prod, h_prod = (r.prod_a, r.prod_b) if carrier_is_a else (r.prod_b, r.prod_a)
        for x, sp in ((a, a_prod), (h, h_prod)):
            x.update(sp=sp, flags=0, partner=0xFFFFFFFF, rxn=0xFF)
        h["pos"], h["comp"] = a["pos"], a["comp"]
        n_released += 1
    free = [i for i in sorted(st) if st[i]["flags"] == 0]
    rec = np.zeros(len(free), dtype=oracle_mod.RECORD_DTYPE)
    for k, i in enumerate(free):
        a = st[i]
        rec[k]["id"], rec[k]["sp"], rec[k]["comp"] = i, a["sp"], a["comp"]
        rec[k]["x"], rec[k]["y"], rec[k]["z"] = a["pos"]
    out, stats = _brute_force_step(oracle_mod, model, seed, rec, t)
    for i, (spc, flags, partner, rxn) in out.items():
        if spc is None:
            del st[i]
            continue
        st[i]["sp"], st[i]["flags"] = spc, flags
        if partner is not None:
            st[i]["partner"], st[i]["rxn"] = partner, rxn
            carrier = i if flags & 1 else partner
            st[i]["pos"] = st[carrier]["pos"]
    stats["released"] = n_released
    return st, stats


def test_two_steps_with_releases(oracle_mod):
    """Complexes formed in step 1 (the BIND's acceptor becomes C when
    released) release with probability 1/2 in step 2, and the freed agents
    take part in that step's proposals."""
    import dataclasses
    base = _model()
    model = dataclasses.replace(base, reactions=[base.reactions[0],
                                                 W.Reaction(Q, B, W.BIND, Q, C, 4.0, 0.8, 0.5),
                                                 base.reactions[2]])
    for seed in (7, 8):
        o = oracle_mod.OracleSim(model, seed)
        st = _state(o.dump())
        released = 0
        for t in range(3):
            st, stats = _release_then_pair(oracle_mod, model, seed, st, t)
            released += stats["released"]
            o.step(1)
            got = _state(o.dump())
            want = {i: {k: v for k, v in a.items() if k != "rxn" and (k != "partner" or a["flags"])}
                    for i, a in st.items()}
            got = {i: {k: v for k, v in a.items() if k != "rxn" and (k != "partner" or a["flags"])}
                   for i, a in got.items()}
            assert got == want, (seed, t + 1)
        o.close()
        assert released >= 10, released


@pytest.mark.parametrize("seed", [1, 2, 3, 11, 12345, 2 ** 40 + 7])
def test_one_static_step_equals_the_brute_force(oracle_mod, seed):
    model = _model()
    o = oracle_mod.OracleSim(model, seed)
    before = o.dump()
    o.step(1)
    after = o.dump()
    o.close()
    want, stats = _brute_force_step(oracle_mod, model, seed, before)
    # the case is dense: conflicts decide many outcomes
    assert stats["final"] >= 10 and stats["contested"] >= 5 and stats["blocked"] >= 5, stats
    got = {int(r["id"]): r for r in after}
    assert set(got) == {i for i, v in want.items() if v[0] is not None}
    pos_of = {int(r["id"]): (int(r["x"]), int(r["y"]), int(r["z"])) for r in before}
    for i, (spc, flags, partner, _) in want.items():
        if spc is None:
            continue
        r = got[i]
        assert (int(r["sp"]), int(r["flags"])) == (spc, flags), i
        if partner is not None:
            assert int(r["partner"]) == partner, i
            carrier = i if flags & 1 else partner
            assert (int(r["x"]), int(r["y"]), int(r["z"])) == pos_of[carrier], i
        else:
            assert (int(r["x"]), int(r["y"]), int(r["z"])) == pos_of[i], i
