"""Volume invariance of the dose readout, and runtime against volume.

Sec. 3.2 (simulation performance factors): at fixed concentrations the number of
molecule-agents grows in proportion to the simulated volume, the work per
agent stays about the same, so the cost of a step grows about linearly with
volume; and the biological readout, the final relative change of pERK + ppERK
in percent, agrees between a volume and ten times that volume to within about
one percentage point at every dose.

This driver runs one batch per volume, each holding one simulation per dose
at the same concentrations, and follows pERK + ppERK (free agents and the
complexes that contain them) with each simulation's threshold monitor, whose
trace records the value every `period` steps.  Host-side orchestration over
the C ABI: every step runs in the engine's kernels.
"""
from __future__ import annotations

import time
from typing import Callable, Sequence

from . import Batch, batch_capacity, monitor_weights


def volume_invariance(make_model: Callable[[int, float], object], doses: Sequence[float], n_agents: int,
                      factor: int = 10, steps: int = 4000, period: int = 0, seed: int = 12,
                      readout: Sequence[str] = ("pERK", "ppERK"), stream=None) -> dict:
    """make_model(n_total, dose) builds the model at n_total agents (its
    volume in proportion); doses run at n_agents and at factor * n_agents.
    Returns the readout change (percent of the initial value) per dose and
    volume, the readout itself every `period` steps (trace[volume][dose]),
    the largest difference between the volumes in percentage points, and the
    wall time per step of each batch."""
    period = period or max(1, steps // 20)
    out = {"doses": list(doses), "volumes": [1, factor], "steps": steps, "readout": list(readout),
           "agents": [], "change_pct": [], "ms_per_step": [], "trace_period": period, "trace": []}
    for vol in (1, factor):
        models = [make_model(n_agents * vol, d) for d in doses]
        cap_a, cap_c = batch_capacity(models)
        b = Batch(cap_a, cap_c, len(models), stream=stream)
        try:
            sids = [b.add(m, seed + k) for k, m in enumerate(models)]
            for s, m in zip(sids, models):
                b.monitor(s, monitor_weights(m, list(readout)), threshold=0, period=period)
            b.sync()
            t0 = time.perf_counter()
            b.step(steps)
            b.sync()
            wall = time.perf_counter() - t0
            change, traces = [], []
            for s in sids:
                st = b.monitor_read(s)
                first, last = int(st.trace[0]), int(st.trace[-1])
                assert st.last_step == steps and len(st.trace) == steps // period + 1
                change.append(100.0 * (last - first) / first)
                traces.append([int(v) for v in st.trace])
            out["agents"].append(sum(m.n_agents for m in models))
            out["change_pct"].append(change)
            out["trace"].append(traces)
            out["ms_per_step"].append(wall / steps * 1e3)
        finally:
            b.close()
    small, large = out["change_pct"]
    out["diff_pp"] = [abs(a - c) for a, c in zip(small, large)]
    out["max_diff_pp"] = max(out["diff_pp"])
    out["time_ratio"] = out["ms_per_step"][1] / out["ms_per_step"][0]
    return out
