"""The oracle with a caller's Gaussian table (CPU).  The table is data (the
step draws Z[i] for the top 16 bits of a Philox word, Sec. 2 of the method
as read here), so both implementations accept one; these pins fix what a
table does to the move independently of its values:

- an all-zero table moves nobody;
- a constant table +k (or -k) moves every agent by exactly
  d = (k * M + 2^31) >> 32 per axis, folded at the half-integer walls
  (x' < 0 -> -1 - x', x' > L -> 2L + 1 - x'), for every agent, whatever the
  draw;
- a table whose largest step leaves the domain is refused."""
import dataclasses

import numpy as np
import pytest

import workloads as W


def _inert(n=400, D=4.0, edge_um=0.3):
    # one species, no reactions, no events: the move is all that happens
    return W.Model(name="inert", species=[W.Species("X", n, D)], reactions=[],
                   compartments=[W.Compartment(W.CUBE, edge_um)])


def _pos(d):
    o = np.argsort(d["id"])
    return np.stack([d["x"][o], d["y"][o], d["z"][o]], axis=1).astype(np.int64), d["id"][o]


def test_zero_table_moves_nobody(oracle_mod):
    m = _inert()
    o = oracle_mod.OracleSim(m, 3, table=np.zeros(65536, np.int16))
    p0, i0 = _pos(o.dump())
    o.step(5)
    p1, i1 = _pos(o.dump())
    assert np.array_equal(i0, i1) and np.array_equal(p0, p1)


@pytest.mark.parametrize("k", [1000, -1000, 150, -32768])
def test_constant_table_moves_every_axis_by_d(oracle_mod, k):
    m = _inert()
    o = oracle_mod.OracleSim(m, 4, table=np.full(65536, k, np.int16))
    ext = int(round(m.compartments[0].size_um * 1000 / m.unit_nm))
    M = oracle_mod.mult(m.species[0].D, m.dt_s, m.unit_nm)
    d = (abs(k) * M + (1 << 31)) >> 32
    d = d if k > 0 else -d
    p0, i0 = _pos(o.dump())
    o.step(1)
    p1, i1 = _pos(o.dump())
    assert np.array_equal(i0, i1)
    want = p0 + d
    want = np.where(want > ext, 2 * ext + 1 - want, want)
    want = np.where(want < 0, -1 - want, want)
    assert d != 0 and np.array_equal(p1, want)


def test_default_table_passed_explicitly_changes_nothing(oracle_mod):
    m = W.toy(300, 300, edge_um=0.3)
    a = oracle_mod.OracleSim(m, 9)
    b = oracle_mod.OracleSim(m, 9, table=oracle_mod.ncdf_table())
    a.step(20)
    b.step(20)
    assert a.digest() == b.digest()


def test_table_stepping_past_the_domain_is_refused(oracle_mod):
    m = dataclasses.replace(_inert(edge_um=0.002), species=[W.Species("X", 4, 100.0)])
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.OracleSim(m, 1, table=np.full(65536, 32767, np.int16))
