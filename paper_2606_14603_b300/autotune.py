"""Autotuner for a batch of simulations: grid cell size, launch shape and
the number of concurrent batches.

The knobs: the cell edge (offset from each model's automatic size); the
block size (128, 256 or 512 threads) and CTAs per SM of the move and
scatter passes; the proximity search's chunk of sorted agents per block
(1024, 2048 or 4096: since simulations are contiguous ranges of the sorted
array, this is also how many small simulations -- or how much of a large
one -- a block covers); and the number of batches the simulations are dealt
over, each stepped on its own CUDA stream.  No knob changes a result (the
proposal search covers every partner within reach for any cell edge not
below the largest contact radius, the kernels are grid-stride loops, and a
simulation's arithmetic does not depend on what else shares its batch), so
the tuner is free to pick whatever is fastest.  Splitting the simulations
over several batches on separate CUDA streams lets the latency-bound kernels
of one batch overlap the memory-bound kernels of another.  The tuner builds
trial groups of the given simulations, times a few steps of each candidate
with CUDA events, and returns the fastest configuration together with all
timings: over the full product of the axes, or axis by axis (coordinate
descent from the first value of each axis) when the product is large.
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
    groups: int = 1          # batches stepped concurrently, one CUDA stream each
    threads_per_block: int = 0   # move / scatter block size, 0 = the library default (128 from 1M to 2M agents of capacity, else 256)
    propose_chunk: int = 0       # sorted agents per proximity-search block, 0 = by capacity

    def key(self):
        return (self.cell_delta, self.blocks_per_sm, self.groups, self.threads_per_block, self.propose_chunk)


def batch_for(sims: Sequence[Tuple[object, int]], cell_delta: int = 0, blocks_per_sm: int = 0,
              headroom: float = 1.25, stream=None, threads_per_block: int = 0, propose_chunk: int = 0):
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
    b = Batch(cap, cells, len(sims), stream=stream, blocks_per_sm=blocks_per_sm,
              threads_per_block=threads_per_block, propose_chunk=propose_chunk)
    ids = [b.add(m, s, sh) for (m, s), sh in zip(sims, shifts)]
    return b, ids


class BatchGroup:
    """The simulations split over `groups` batches (dealt by size in snake
    order, 0 1 .. G-1 G-1 .. 1 0 ..., so that the groups hold nearly equal
    agent counts), each on its own CUDA stream and stepped together.
    Simulation k of the input keeps index k here."""

    def __init__(self, sims: Sequence[Tuple[object, int]], cell_delta: int = 0, blocks_per_sm: int = 0,
                 groups: int = 1, headroom: float = 1.25, streams=None, threads_per_block: int = 0,
                 propose_chunk: int = 0):
        import torch
        groups = max(1, min(groups, len(sims)))
        order = sorted(range(len(sims)), key=lambda k: sims[k][0].n_agents)
        members = [[] for _ in range(groups)]
        for r, k in enumerate(order):
            pos = r % groups
            members[pos if (r // groups) % 2 == 0 else groups - 1 - pos].append(k)
        self.streams = streams or [torch.cuda.Stream() for _ in range(groups)]
        self.batches, self.where = [], {}
        for g, ks in enumerate(members):
            b, ids = batch_for([sims[k] for k in ks], cell_delta, blocks_per_sm, headroom, self.streams[g],
                               threads_per_block, propose_chunk)
            self.batches.append(b)
            for k, sid in zip(ks, ids):
                self.where[k] = (g, sid)

    def step(self, n: int, chunk: int = 8) -> None:
        """n steps of every batch; launches interleave in chunks so that every
        stream has work queued."""
        while n > 0:
            k = min(n, chunk)
            for b in self.batches:
                b.step(k)
            n -= k

    def sync(self) -> None:
        for b in self.batches:
            b.sync()

    def counts(self, k: int):
        g, sid = self.where[k]
        return self.batches[g].counts(sid)

    def digest(self, k: int) -> int:
        g, sid = self.where[k]
        return self.batches[g].digest(sid)

    def timed_step(self, n: int) -> float:
        """Milliseconds of n steps of the whole group, from CUDA events joined
        across the streams (the first stream starts and ends the interval)."""
        import torch
        s0 = self.streams[0]
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(s0)
        for st in self.streams[1:]:
            st.wait_event(start)
        self.step(n)
        for st in self.streams[1:]:
            e = torch.cuda.Event()
            e.record(st)
            s0.wait_event(e)
        end.record(s0)
        end.synchronize()
        return start.elapsed_time(end)

    def close(self) -> None:
        for b in self.batches:
            b.close()
        self.batches = []


def _time(sims, c: Choice, steps: int, warmup: int) -> float:
    grp = BatchGroup(sims, c.cell_delta, c.blocks_per_sm, c.groups, threads_per_block=c.threads_per_block,
                     propose_chunk=c.propose_chunk)
    try:
        grp.step(warmup)
        grp.sync()
        return grp.timed_step(steps) / steps
    finally:
        grp.sync()
        grp.close()


def tune(sims: Sequence[Tuple[object, int]], cell_deltas=(-1, 0, 1), blocks=(0, 8, 16), groups=(1, 2, 4),
         steps: int = 20, warmup: int = 3, threads=(0,), chunks=(0,),
         search: str = "grid") -> Tuple[Choice, List[Choice]]:
    """Fastest configuration and every timed candidate.  search="grid" times
    the product of the axes; "axes" starts from the first value of each axis
    and, axis by axis (groups, cell size, block size, chunk, CTAs per SM),
    keeps the fastest value with the others fixed."""
    results = {}

    def run(c: Choice) -> Choice:
        if c.key() not in results:
            c.ms_per_step = _time(sims, c, steps, warmup)
            results[c.key()] = c
        return results[c.key()]

    if search == "grid":
        for d, bps, ng, tb, ch in itertools.product(cell_deltas, blocks, groups, threads, chunks):
            run(Choice(d, bps, 0.0, ng, tb, ch))
    elif search == "axes":
        cur = {"cell_delta": cell_deltas[0], "blocks_per_sm": blocks[0], "groups": groups[0],
               "threads_per_block": threads[0], "propose_chunk": chunks[0]}
        for name, values in (("groups", groups), ("cell_delta", cell_deltas), ("threads_per_block", threads),
                             ("propose_chunk", chunks), ("blocks_per_sm", blocks)):
            tried = [run(Choice(ms_per_step=0.0, **dict(cur, **{name: v}))) for v in values]
            cur[name] = getattr(min(tried, key=lambda c: c.ms_per_step), name)
    else:
        raise ValueError(f"unknown search {search!r}")
    allc = list(results.values())
    best = min(allc, key=lambda c: c.ms_per_step)
    return best, allc
