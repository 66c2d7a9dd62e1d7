"""Threshold monitor written out from its definition.

TEST INFRASTRUCTURE ONLY (imported by tests/): the product package never
imports it, and it never imports the product package.

Sec. 2 (simulator description): the user designates molecular species to
follow continuously and sets a concentration threshold for a time window;
the cell is classified by whether the level passes the threshold (the
paper's example follows ppERK: above the healthy level too early means
aberrant signalling; a drug that brings it back below means normal).

Reading used here and by the engine: the followed quantity is a weighted sum
of the counts vector (free agents by species and compartment, bound
complexes by reaction), taken at the state after t completed steps, for
every t in [begin, end) with (t - begin) % period == 0 that the run passes
through after the monitor is installed; a state passes when the value is
above the threshold (or below, for a lower bound).
"""
from __future__ import annotations

from typing import Dict, List, Optional

TRACE_KEEP = 1024


def value(counts, weights) -> int:
    """sum_k weights[k] * counts[k], exact (Python integers); weights may be
    shorter than counts (missing entries are 0)."""
    return sum(int(w) * int(c) for w, c in zip(weights, counts))


def evaluate(values: Dict[int, int], begin: int, end: Optional[int], period: int, threshold: int,
             above: bool, installed_at: int = 0) -> dict:
    """Monitor state after a run that visited the states `values` (step ->
    value, every step from installed_at to the last one).  Returns the last
    value and step, first passing step, counts, last outcome and the last
    TRACE_KEEP evaluated values, oldest first."""
    end = 0xFFFFFFFF if end is None else end
    evaluated: List[int] = []
    steps: List[int] = []
    passed: List[bool] = []
    for t in sorted(values):
        if t < installed_at or t < begin or t >= end or (t - begin) % period:
            continue
        v = values[t]
        evaluated.append(v)
        steps.append(t)
        passed.append(v > threshold if above else v < threshold)
    first = next((s for s, p in zip(steps, passed) if p), None)
    return {
        "value": evaluated[-1] if evaluated else 0,
        "last_step": steps[-1] if steps else 0,
        "first_pass": first,
        "n_evaluated": len(evaluated),
        "n_passed": sum(passed),
        "state": passed[-1] if passed else None,
        "trace": evaluated[-TRACE_KEEP:],
    }
