"""Continuous-batching server for simulation jobs on one GPU.

Jobs (a model, a seed, a step count) arrive over time.  The server keeps one
batch whose arena is sized from an HBM budget; between epochs it admits every
arrived job that fits (agent slots, grid cells, simulation slots), steps all
resident jobs together for an epoch, and retires the jobs that reached their
step count, reading their counts and digest first.  A job's latency runs from
its arrival to the moment its result is back on the host.

The engine's arithmetic does not depend on what else is in the batch, so every
job's result is bit-identical to the same job run alone (tests check this).
A job whose own simulation stops with an error (births of one step beyond its
limit) fails alone: it is reported with the error and removed, and the jobs
sharing its batch go on.  A device error of a whole batch (e.g. its agent
capacity exceeded) fails the jobs resident in that batch, which are reported
with the error; the batch is replaced and serving goes on.

Admission is FIFO by default (no overtaking).  With admission="backfill" a
job that fits may be admitted ahead of an earlier one that does not, as long
as the earliest waiting job has waited less than `backfill_limit_s`; after
that nothing overtakes it until it is admitted (no starvation).

Latency statistics cover every offered job: a job still queued or running
when the run stops is counted at its age then (a lower bound of its
latency), and the number of such censored jobs is reported.

This is host-side orchestration over the C ABI: admission, retirement and
epoch sizing happen here, every step runs in the engine's kernels.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

from . import AbmError, Batch, model_grid

# bytes of one agent slot and one grid cell in the batch arena (see the
# layout in csrc/api.cu); used only to turn an HBM budget into capacities
BYTES_PER_AGENT_SLOT = 100
BYTES_PER_CELL = 12


@dataclasses.dataclass
class JobResult:
    job_id: int
    arrival_s: float
    admitted_s: float
    finished_s: float
    steps: int
    agents: int
    counts: Optional[np.ndarray]
    digest: Optional[int]
    error: Optional[str] = None

    @property
    def latency_s(self) -> float:
        return self.finished_s - self.arrival_s


@dataclasses.dataclass
class _Resident:
    job: object
    sid: int
    remaining: int
    admitted_s: float
    agents: int
    cells: int


class Server:
    """Continuous batching of simulation jobs under an HBM budget.

    budget_bytes: device memory for the arenas (agents and cells split by
    `cells_per_agent`, unless capacities are given); max_sims: concurrent
    jobs; epoch: steps between admission points; groups: batches stepped
    concurrently, each on its own CUDA stream with an equal share of the
    budget and the job slots (the latency-bound kernels of one overlap the
    memory-bound kernels of another).  A job is frozen on the device at its
    own last step, so epochs need not stop at job boundaries."""

    def __init__(self, budget_bytes: float = 150e9, max_sims: int = 256, epoch: int = 50,
                 cells_per_agent: float = 1.3, headroom: float = 1.25, stream=None,
                 capacity_agents: Optional[int] = None, capacity_cells: Optional[int] = None,
                 groups: int = 1):
        per_agent = BYTES_PER_AGENT_SLOT + cells_per_agent * BYTES_PER_CELL
        cap_agents = capacity_agents or min(int(budget_bytes / per_agent), 2_000_000_000)
        cap_cells = capacity_cells or min(int(cap_agents * cells_per_agent), 4_000_000_000)
        self.groups = max(1, groups)
        # per group
        self.cap_agents, self.cap_cells = cap_agents // self.groups, cap_cells // self.groups
        self.max_sims = max(1, max_sims // self.groups)
        self.epoch = epoch
        self.headroom = headroom
        # one library-owned stream per batch unless a single batch gets the caller's
        self.batches = [Batch(self.cap_agents, self.cap_cells, self.max_sims,
                              stream=stream if self.groups == 1 else None) for _ in range(self.groups)]
        self.resident: Dict[Tuple[int, int], _Resident] = {}
        self.used_agents = [0] * self.groups
        self.used_cells = [0] * self.groups
        self.stream = stream
        self.steps_run = 0
        self.molecule_steps = 0
        self.max_resident = 0
        self.waited = 0          # admissions that had to wait for capacity
        self.failed: List[JobResult] = []   # failed jobs not yet reported
        self.batch_failures = 0
        self.sim_failures = 0    # jobs stopped by their own simulation's error

    @property
    def batch(self):
        return self.batches[0]

    # -- capacity accounting (reserved per job: initial agents x headroom) --
    def need(self, job):
        return int(job.model.n_agents * self.headroom) + 1, model_grid(job.model)[1]

    def can_ever_fit(self, job) -> bool:
        a, c = self.need(job)
        return a <= self.cap_agents and c <= self.cap_cells

    def _group_for(self, job) -> Optional[int]:
        need_a, need_c = self.need(job)
        best = None
        for g in range(self.groups):
            n_res = sum(1 for (gg, _) in self.resident if gg == g)
            if (n_res < self.max_sims and self.used_agents[g] + need_a <= self.cap_agents
                    and self.used_cells[g] + need_c <= self.cap_cells):
                if best is None or self.used_agents[g] < self.used_agents[best]:
                    best = g
        return best

    def fits(self, job) -> bool:
        return self._group_for(job) is not None

    def _fail_group(self, g: int, err: str, now: float) -> None:
        """Batch g reported a device error: its resident jobs fail; a fresh
        batch takes its place."""
        for key in [k for k in self.resident if k[0] == g]:
            r = self.resident.pop(key)
            self.failed.append(JobResult(r.job.job_id, r.job.arrival_s, r.admitted_s, now, r.job.steps,
                                         r.job.model.n_agents, None, None, err))
        self.used_agents[g] = 0
        self.used_cells[g] = 0
        self.batches[g].close()
        self.batches[g] = Batch(self.cap_agents, self.cap_cells, self.max_sims,
                                stream=self.stream if self.groups == 1 else None)
        self.batch_failures += 1

    def admit(self, job, now: float) -> None:
        g = self._group_for(job)
        need_a, need_c = self.need(job)
        try:
            sid = self.batches[g].add(job.model, job.seed)
        except AbmError as e:
            if e.status in (-1, -5):   # EINVAL / ECAPACITY of this job: the batch is intact
                raise
            self._fail_group(g, str(e), now)   # an earlier device error surfaced here
            g = self._group_for(job)
            sid = self.batches[g].add(job.model, job.seed)
        self.batches[g].set_max_step(sid, job.steps)
        self.resident[(g, sid)] = _Resident(job, sid, job.steps, now, need_a, need_c)
        self.used_agents[g] += need_a
        self.used_cells[g] += need_c
        self.max_resident = max(self.max_resident, len(self.resident))

    def step_epoch(self) -> int:
        """Step every batch with resident jobs for one epoch (at most the
        largest remaining count); jobs that reach their own last step inside
        it are frozen there.  Launches interleave across the batches."""
        if not self.resident:
            return 0
        k = min(max(r.remaining for r in self.resident.values()), self.epoch)
        active = sorted({g for (g, _) in self.resident})
        left = k
        while left > 0:
            c = min(left, 8)
            for g in active:
                try:
                    self.batches[g].step(c)
                except AbmError:
                    pass        # reported by the next synchronising call of this batch
            left -= c
        for r in self.resident.values():
            done = min(k, r.remaining)
            r.remaining -= done
            self.molecule_steps += r.job.model.n_agents * done
        self.steps_run += k
        return k

    def _retire_failed_sims(self, g: int, now: float) -> None:
        """Jobs of batch g whose own simulation stopped with an error: report
        them failed and remove them; the batch and its other jobs go on."""
        for key in [k for k in self.resident if k[0] == g]:
            st, msg = self.batches[g].sim_status(key[1])
            if st == 0:
                continue
            r = self.resident.pop(key)
            self.failed.append(JobResult(r.job.job_id, r.job.arrival_s, r.admitted_s, now, r.job.steps,
                                         r.job.model.n_agents, None, None, msg))
            self.batches[g].remove(key[1])
            self.used_agents[g] -= r.agents
            self.used_cells[g] -= r.cells
            self.sim_failures += 1

    def retire_finished(self, clock: Callable[[], float]) -> List[JobResult]:
        for g in sorted({g for (g, _) in self.resident}):
            try:
                self.batches[g].sync()
            except AbmError as e:
                self._fail_group(g, str(e), clock())
                continue
            self._retire_failed_sims(g, clock())
        done, self.failed = self.failed, []
        for key in [key for key, r in self.resident.items() if r.remaining == 0]:
            g, sid = key
            r = self.resident.pop(key)
            counts = self.batches[g].counts(sid)
            digest = self.batches[g].digest(sid)
            now = clock()
            self.batches[g].remove(sid)
            self.used_agents[g] -= r.agents
            self.used_cells[g] -= r.cells
            done.append(JobResult(r.job.job_id, r.job.arrival_s, r.admitted_s, now, r.job.steps,
                                  r.job.model.n_agents, counts, digest))
        return done

    def sync(self) -> None:
        for b in self.batches:
            try:
                b.sync()
            except AbmError:
                pass            # handled by retire_finished

    def close(self) -> None:
        for b in self.batches:
            b.close()


def _percentile(values, q):
    return float(np.percentile(values, q)) if len(values) else None


def run(jobs, server: Server, duration_s: Optional[float] = None, real_time: bool = True,
        drain: bool = True, admission: str = "fifo", backfill_limit_s: float = 10.0) -> dict:
    """Serve `jobs` (sorted by arrival_s) and return throughput and latency
    statistics.  With real_time the arrivals follow the wall clock; otherwise
    a job arrives as soon as the server looks for new work after its arrival
    time on a virtual clock that only advances with the GPU work done.
    Arrivals stop at duration_s; with drain the run goes on until every
    arrived job is done, otherwise it stops at duration_s and the jobs still
    queued or running are censored (counted at their age then)."""
    if admission not in ("fifo", "backfill"):
        raise ValueError(f"unknown admission policy {admission!r}")
    pending = list(jobs)
    pending.sort(key=lambda j: j.arrival_s)
    queue: List = []                    # arrived, not admitted (FIFO by arrival)
    results: List[JobResult] = []
    rejected: List[int] = []
    waited = set()
    overtakes = 0
    t0 = time.perf_counter()
    virtual = [0.0]

    def clock() -> float:
        if real_time:
            return time.perf_counter() - t0
        return virtual[0]

    i = 0
    horizon = duration_s if duration_s is not None else math.inf
    while True:
        now = clock()
        while i < len(pending) and pending[i].arrival_s <= now and pending[i].arrival_s < horizon:
            if server.can_ever_fit(pending[i]):
                queue.append(pending[i])
            else:
                rejected.append(pending[i].job_id)
            i += 1
        if queue and not server.fits(queue[0]) and queue[0].job_id not in waited:
            waited.add(queue[0].job_id)
            server.waited += 1
        # admit in arrival order while they fit; with backfill, later jobs that
        # fit may pass a head that does not, until the head has waited too long
        while queue and server.fits(queue[0]):
            server.admit(queue.pop(0), clock())
        if admission == "backfill" and queue and clock() - queue[0].arrival_s < backfill_limit_s:
            k = 1
            while k < len(queue):
                if server.fits(queue[k]):
                    server.admit(queue.pop(k), clock())
                    overtakes += 1
                else:
                    k += 1
        if server.resident:
            w0 = time.perf_counter()
            server.step_epoch()
            if not real_time:
                server.sync()           # the virtual clock advances by GPU time
            results += server.retire_finished(clock)
            if not real_time:
                virtual[0] += time.perf_counter() - w0
        else:
            if i >= len(pending) or pending[i].arrival_s >= horizon:
                if not queue:
                    break
            elif real_time:
                time.sleep(max(0.0, min(pending[i].arrival_s - clock(), 0.01)))
            else:
                virtual[0] = max(virtual[0], pending[i].arrival_s)
        if not drain and clock() >= horizon:
            break
    wall = clock()
    failed = [r for r in results if r.error is not None]
    results = [r for r in results if r.error is None]
    offered_jobs = [j for j in pending if j.arrival_s < horizon]
    done_ids = {r.job_id for r in results} | {r.job_id for r in failed} | set(rejected)
    # censored: arrived (within the window) but neither completed, failed nor rejected
    censored = [j for j in offered_jobs if j.job_id not in done_ids and j.arrival_s <= wall]
    lat_done = np.array([r.latency_s for r in results]) if results else np.zeros(0)
    lat_all = np.concatenate([lat_done, np.array([wall - j.arrival_s for j in censored])]) if censored \
        else lat_done
    offered = sum(j.model.n_agents * j.steps for j in offered_jobs)
    return {
        "jobs_offered": len(offered_jobs),
        "jobs_completed": len(results),
        "jobs_censored": len(censored),
        "wall_s": wall,
        "throughput_molecule_steps_per_s": server.molecule_steps / wall if wall > 0 else 0.0,
        "completed_molecule_steps_per_s": sum(r.agents * r.steps for r in results) / wall if wall > 0 else 0.0,
        "jobs_per_s": len(results) / wall if wall > 0 else 0.0,
        "offered_molecule_steps_per_s": offered / horizon if math.isfinite(horizon) and horizon > 0 else None,
        # over every offered job, censored ones at their age when the run stopped (lower bounds)
        "latency_p50_s": _percentile(lat_all, 50),
        "latency_p99_s": _percentile(lat_all, 99),
        "latency_max_s": float(lat_all.max()) if len(lat_all) else None,
        "latency_is_lower_bound": len(censored) > 0,
        # over the completed jobs only
        "completed_latency_p50_s": _percentile(lat_done, 50),
        "completed_latency_p99_s": _percentile(lat_done, 99),
        "jobs_rejected": len(rejected),
        "jobs_failed": len(failed),
        "batch_failures": server.batch_failures,
        "sim_failures": server.sim_failures,
        "admission": admission,
        "overtakes": overtakes,
        "steps_run": server.steps_run,
        "max_resident": server.max_resident,
        "admissions_waited": server.waited,
        "results": results,
        "failed": failed,
    }
