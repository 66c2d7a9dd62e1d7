"""Oracle runs for the long GPU parity tests, executed in worker processes
(test infrastructure: only tests use this module).

A job is (kind, params, seed, checkpoints); it returns {step: digest} of the
oracle simulation at every checkpoint step."""
from __future__ import annotations


def build_model(kind, params):
    import workloads as W
    if kind == "mapk":
        return W.mapk(**params)
    if kind == "nuclear":
        return W.nuclear(**params)
    if kind == "sweep":
        return W.sweep()[params["k"]][0]
    raise ValueError(kind)


def digest_trace(job):
    kind, params, seed, checkpoints = job
    import oracle
    sim = oracle.OracleSim(build_model(kind, params), seed)
    out = {}
    t = 0
    try:
        for c in checkpoints:
            sim.step(c - t)
            t = c
            out[c] = sim.digest()
    finally:
        sim.close()
    return out
