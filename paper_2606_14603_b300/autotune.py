"""Autotuner for a batch of simulations: grid cell size and launch shape.

Neither knob changes a result (the proposal search covers every partner
within reach for any cell edge not below the largest contact radius, and the
kernels are grid-stride loops), so the tuner is free to pick whatever is
fastest.  It builds trial batches of the given simulations, times a few
steps of each candidate with CUDA events on the batch's stream, and returns
the fastest configuration together with all timings.
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import List, Sequence, Tuple

from . import Batch, model_grid


@dataclasses.dataclass
class Choice:
    cell_delta: int          # added to each model's automatic cell_log2
    blocks_per_sm: int       # 0 = the CTAs of the move pass that fit on an SM at once
    ms_per_step: float


def batch_for(sims: Sequence[Tuple[object, int]], cell_delta: int = 0, blocks_per_sm: int = 0,
              headroom: float = 1.25, stream=None):
    """(batch, ids) with every sim added at its automatic cell size + delta.
    Deltas that would make a cell smaller than a contact radius fall back to
    the automatic size."""
    shifts = []
    for m, _ in sims:
        base, _ = model_grid(m)
        sh = base + cell_delta
        try:
            model_grid(m, sh)
        except Exception:
            sh = base
        shifts.append(sh)
    cells = sum(model_grid(m, sh)[1] for (m, _), sh in zip(sims, shifts))
    cap = int(sum(m.n_agents for m, _ in sims) * headroom) + 65536
    b = Batch(cap, cells, len(sims), stream=stream, blocks_per_sm=blocks_per_sm)
    ids = [b.add(m, s, sh) for (m, s), sh in zip(sims, shifts)]
    return b, ids


def tune(sims: Sequence[Tuple[object, int]], cell_deltas=(-1, 0, 1), blocks=(0, 8, 16),
         steps: int = 20, warmup: int = 3) -> Tuple[Choice, List[Choice]]:
    import torch
    stream = torch.cuda.Stream()
    results = []
    for d, bps in itertools.product(cell_deltas, blocks):
        b, _ = batch_for(sims, d, bps, stream=stream)
        b.step(warmup)
        b.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        b.sync()
        results.append(Choice(d, bps, e0.elapsed_time(e1) / steps))
        b.close()
    best = min(results, key=lambda c: c.ms_per_step)
    return best, results
