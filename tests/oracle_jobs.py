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


def readout_trace(job):
    """(model_args, seed, steps, period, names): the oracle's count of the
    named species, free anywhere or inside complexes (each complex adds the
    number of its two reactants that are named), at t = 0, period, ...,
    steps.  The readout of the volume-invariance experiment (Sec. 3.2),
    written from the counts layout: free agents by species and compartment,
    then bound complexes by reaction."""
    (n, dose), seed, steps, period, names = job
    import oracle
    import workloads as W
    model = W.mapk(n, dose)
    sp_names = [s.name for s in model.species]
    want = {sp_names.index(x) for x in names}
    n_c = len(model.compartments)
    n_free = len(model.species) * n_c
    weight = [1 if k // n_c in want else 0 for k in range(n_free)]
    weight += [int(r.a in want) + int(r.b in want) for r in model.reactions]

    def value(counts):
        return sum(w * int(c) for w, c in zip(weight, counts[:-1]))

    sim = oracle.OracleSim(model, seed)
    try:
        out = [value(sim.counts())]
        for _ in range(steps // period):
            sim.step(period)
            out.append(value(sim.counts()))
        return out
    finally:
        sim.close()
