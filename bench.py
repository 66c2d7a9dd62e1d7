#!/usr/bin/env python3
"""Benchmark of the molecule-agent step engine on B300.

Default workload: the MAPK-like cascade with 1,000,000 agents in a 10 um cube
(9 species, 12 bind/release reactions, dt = 1 us), seed 12.  One "step" is
one full pass of the hot path over every agent: first-order events, Brownian
move, grid build (histogram, scan, scatter), 27-cell proposals, acceptance
and births.  The state (about 86 MB) fits in the 126 MB L2, so L2 is flushed
(a 256 MB write) between timed steps and each step is timed on its own with
CUDA events on the engine's stream.

Prints one JSON line.  `value` = molecule-steps/s summed over ranks (each rank
runs an independent replica: weak scaling).  `--impl reference` times the CPU
oracle (the serial simulator under oracle/) on a bounded sample instead.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "molecule-steps/s @1M agents (%HBM roofline); batched vs serial sweep; p50/p99"
UNIT = "molecule-steps/s"
# per-kernel bytes each launch must move per unit (agent or cell) in this
# design; the step as a whole must read and rewrite the 20-byte agent record
STEP_BYTES_PER_AGENT = 40
E2E_STEPS = 500          # steps of the end-to-end loop (creation amortised over them)
KERNEL_BYTES = {"k_move": (36, "agent"), "k_tile_prefix": (8 / 8192, "cell"), "k_scan": (12, "cell"),
                "k_scatter": (45, "agent"), "k_propose": (20, "agent"), "k_accept": (4, "agent")}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["cascade", "nuclear", "toy", "sweep", "serve"], default="cascade")
    p.add_argument("--serve-seconds", type=float, default=20.0,
                   help="seconds of job arrivals in the serving measurement (the served config runs 600)")
    p.add_argument("--sweep-steps", type=int, default=50, help="steps per sim in the sweep summary")
    p.add_argument("--serve-groups", type=int, default=4,
                   help="batches the server steps concurrently (one CUDA stream each)")
    p.add_argument("--serve-rate", type=float, default=20.0, help="job arrivals per second (the served config: 20)")
    p.add_argument("--serve-sub-rate", type=float, default=10.0,
                   help="a rate below the GPU's capacity, served to completion (0 = skip)")
    p.add_argument("--serve-admission", choices=["fifo", "backfill"], default="backfill")
    p.add_argument("--size-steps", type=int, default=100,
                   help="steps of the 4M/16M-agent cascade summary (0 = skip)")
    p.add_argument("--volume-steps", type=int, default=4000,
                   help="steps of the volume-invariance summary (1M vs 10M agents per dose; 0 = skip)")
    p.add_argument("--births-steps", type=int, default=20,
                   help="steps of the birth-heavy summary (about 50k-60k births per step; 0 = skip)")
    p.add_argument("--agents", type=int, default=0, help="override the agent count")
    p.add_argument("--profile-steps", type=int, default=50)
    p.add_argument("--no-flush", action="store_true", help="do not flush L2 between steps")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--ref-seconds", type=float, default=90.0, help="oracle time budget of --impl reference")
    return p.parse_args()


def workload(args):
    import workloads as W
    if args.workload == "cascade":
        n = args.agents or 1_000_000
        return W.mapk(n), W.MAPK_SEED, f"cascade_{n}"
    if args.workload == "nuclear":
        n = args.agents or 4_000_000
        return W.nuclear(n), W.NUCLEAR_SEED, f"two_compartment_{n}"
    return W.toy(), W.TOY_SEED, "toy_5000"


def config_of(args, model, name, extra=None):
    c = {"workload": name, "agents": model.n_agents, "species": len(model.species),
         "reactions": len(model.reactions), "compartments": len(model.compartments),
         "dt_s": model.dt_s, "position_unit_nm": model.unit_nm,
         "l2": "no flush" if args.no_flush else
               "flushed between timed steps: 256 MB write, then a 256 MB read (cold, clean L2)"}
    if extra:
        c.update(extra)
    return c


def molecules(counts, model):
    n_sp, n_c = len(model.species), len(model.compartments)
    free = int(counts[: n_sp * n_c].sum())
    bound = int(counts[n_sp * n_c: -1].sum())
    return free + 2 * bound


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons in the background.

    Every sample carries nvidia-smi's own timestamp, so the summary does not
    depend on how the pipe is buffered.  ``__enter__`` waits (up to a second)
    for the first sample so that the sampler is running when the caller's
    timed region starts, and ``mark(t0, t1)`` (``time.perf_counter`` values)
    names that region.  The summary is taken over the samples inside it; a
    region shorter than the sampling interval falls back to the two samples
    that bracket it, and ``window`` says which."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 20

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.region = None

    def _read(self):
        for line in self.proc.stdout:
            if line.strip():
                self.lines.append(line)

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", str(self.INTERVAL_MS), "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()
        t_end = time.perf_counter() + 1.0
        while not self.lines and self.proc.poll() is None and time.perf_counter() < t_end:
            time.sleep(0.005)
        return self

    def mark(self, t0, t1):
        # perf_counter -> wall-clock seconds, the clock nvidia-smi stamps with
        off = time.time() - time.perf_counter()
        self.region = (t0 + off, t1 + off)

    def __exit__(self, *a):
        if self.proc:
            time.sleep(3 * self.INTERVAL_MS / 1000.0)     # let one sample land after the region
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
            self.reader.join(timeout=5)

    @staticmethod
    def parse(line):
        """One CSV sample -> (epoch seconds, sm MHz, max MHz, watts, [active reasons]) or None."""
        import datetime
        f = [x.strip() for x in line.split(",")]
        if len(f) < 10:
            return None
        try:
            sm, mx, pw = float(f[2]), float(f[3]), float(f[4])
        except ValueError:
            return None
        try:
            t = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            t = None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        return t, sm, mx, pw, [nm for nm, v in zip(names, f[6:10]) if v.lower() == "active"]

    def summary(self):
        rows = [r for r in map(self.parse, self.lines) if r]
        window = "whole sampler run"
        if rows and any(r[0] is None for r in rows):
            window = "whole sampler run (timestamps unreadable)"
        elif self.region and rows:
            t0, t1 = self.region
            slack = self.INTERVAL_MS / 1000.0
            inside = [r for r in rows if t0 <= r[0] <= t1 + slack]
            if inside:
                rows, window = inside, "timed region"
            else:
                rows = [r for r in rows if r[0] < t0][-1:] + [r for r in rows if r[0] > t1][:1]
                window = "the two samples bracketing the timed region (shorter than the interval)"
        if not rows:
            return None
        sm = sorted(r[1] for r in rows)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[2] for r in rows), "samples": len(rows),
                "interval_ms": self.INTERVAL_MS, "window": window,
                "power_w_max": max(r[3] for r in rows),
                "reasons": sorted({nm for r in rows for nm in r[4]})}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6400.0}, "fallback"


def kernel_source_sha():
    import hashlib
    h = hashlib.sha256()
    for f in ("kernels.cu", "engine.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2606_14603_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def launches_per_step(cells):
    """Engine kernels one step launches: five, plus k_tile_prefix on grids of
    more than 8192 scan tiles of 8192 cells."""
    return 5 + (1 if (cells + 8191) // 8192 > 8192 else 0)


def ncu_traffic(kernel):
    """DRAM bytes (read + write) per 1M-agent launch of a kernel from the
    committed ncu summary, if the kernel sources (kernels.cu + engine.cuh) are
    unchanged since the capture (else None): (bytes, units, unit, note)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    try:
        sha = kernel_source_sha()
        for line in open(path):
            f = line.split(None, 5)
            if len(f) >= 5 and not line.startswith("#") and f[0] == kernel and f[1] == sha:
                return float(f[2]), float(f[3]), f[4], (f[5].strip() if len(f) > 5 else "")
    except OSError:
        pass
    return None


# ---------------------------------------------------------------------------
def reduce_over_ranks(total_ms, molecule_steps, device="cuda"):
    """Whole-job numbers over all ranks: the slowest rank's timed total and
    the sum of the molecule-steps every rank processed."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms, molecule_steps], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def cpu_model():
    """The host CPU's model name (from /proc/cpuinfo) and its core count."""
    name = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return name, os.cpu_count() or 1


def run_reference(args, rank):
    """The oracle on the host cores, on a bounded sample of the same workload:
    exactly `warmup` untimed steps, then `steps` timed steps (fewer only if
    they would exceed the time budget, which the line then says)."""
    import oracle
    model, seed, name = workload(args)
    sim = oracle.OracleSim(model, seed)
    t0 = time.perf_counter()
    sim.step(1)
    est = time.perf_counter() - t0
    if args.warmup > 1:
        sim.step(args.warmup - 1)
    budget = args.ref_seconds
    steps = max(1, min(args.steps, int(budget / max(est, 1e-6))))
    n0 = molecules(sim.counts(), model)
    t0 = time.perf_counter()
    sim.step(steps)
    el = time.perf_counter() - t0
    n1 = molecules(sim.counts(), model)
    value = 0.5 * (n0 + n1) * steps / el
    cpu, cores = cpu_model()
    sample = (f"{name}: {steps} oracle steps after {max(1, args.warmup)} untimed, single thread"
              + ("" if steps == args.steps else f" (capped from {args.steps} by the {budget:.0f} s budget)"))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": max(1, args.warmup), "ms_per_step": 1e3 * el / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": config_of(args, model, name, {"parallelism": f"replicas x{args.gpus}", "seed": seed}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu, "host_cores": cores},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(model, seed, name, seconds=12.0):
    import oracle
    sim = oracle.OracleSim(model, seed)
    t0 = time.perf_counter()
    steps = 0
    n = 0
    while time.perf_counter() - t0 < seconds:
        n += molecules(sim.counts(), model) if steps == 0 else 0
        sim.step(1)
        steps += 1
    el = time.perf_counter() - t0
    n = molecules(sim.counts(), model)
    cpu, cores = cpu_model()
    return {"value": n * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{name}: the first {steps} steps from t = 0, serial oracle, one thread",
            "cpu_model": cpu, "host_cores": cores}


def _sweep_oracle_task(args):
    """One sweep simulation on the oracle (a worker process): molecule-steps
    and seconds of `steps` steps from t = 0 (creation not timed)."""
    k, steps, scale = args
    import oracle
    import workloads as W
    model, seed = W.sweep(scale)[k]
    sim = oracle.OracleSim(model, seed)
    t0 = time.perf_counter()
    sim.step(steps)
    el = time.perf_counter() - t0
    sim.close()
    return model.n_agents * steps, el


def sweep_cpu_baseline(steps=2, scale=1.0):
    """The 64 sweep simulations on the oracle, one process per host core
    (spawned: CUDA is already initialised in this process)."""
    import multiprocessing as mp
    import workloads as W
    cores = os.cpu_count() or 1
    n = len(W.sweep(scale))
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_sweep_oracle_task, [(k, steps, scale) for k in range(n)], chunksize=1)
    ms = sum(r[0] for r in res)
    busy = sum(r[1] for r in res)
    cpu, _ = cpu_model()
    return {"value": ms / (busy / cores), "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu,
            "sample": f"all {n} sweep simulations, the first {steps} steps of each from t = 0, serial "
                      f"oracle in {cores} worker processes; value = molecule-steps / (summed step "
                      f"seconds / {cores}), creation not timed"}


def run_sweep(A, torch, stream, steps, warmup=5, scale=1.0, cpu=True):
    """The 64-sim dose x seed sweep: all sims stepped together (one batch, or
    the autotuner's number of batches on concurrent streams) versus each sim
    alone, one after the other (same library, same step count, CUDA-graph
    replay in both, no L2 flush: the batch's 12.6M-agent state exceeds L2
    while the small sims alone fit in it)."""
    import workloads as W
    from paper_2606_14603_b300 import autotune
    sims = W.sweep(scale)
    models = [m for m, _ in sims]
    n_total = sum(m.n_agents for m in models)
    best, tried = autotune.tune(sims, cell_deltas=(0, 1), blocks=(0, 3, 2), groups=(2, 1, 4, 8),
                                threads=(256, 128, 512), chunks=(0, 1024, 2048, 4096), steps=10, warmup=2,
                                search="axes")
    grp = autotune.BatchGroup(sims, best.cell_delta, best.blocks_per_sm, best.groups,
                              threads_per_block=best.threads_per_block, propose_chunk=best.propose_chunk)
    grp.step(warmup)
    grp.sync()
    torch.cuda.synchronize()
    batched_ms = grp.timed_step(steps)
    grp.sync()
    live = sum(molecules(grp.counts(k), m) for k, m in enumerate(models))
    grp.close()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    serial_ms = 0.0
    for m, s in sims:
        sim = A.Sim(m, s, stream=stream)
        sim.step(warmup)
        sim.sync()
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        serial_ms += e0.elapsed_time(e1)
        sim.close()
    batched = n_total * steps / (batched_ms / 1e3)
    serial = n_total * steps / (serial_ms / 1e3)
    cpu_line = sweep_cpu_baseline(scale=scale) if cpu else None
    return {"cpu_baseline": cpu_line, "sims": len(sims), "agents": n_total, "live_after": live, "steps": steps,
            "autotune": {"cell_delta": best.cell_delta, "blocks_per_sm": best.blocks_per_sm,
                         "groups": best.groups, "threads_per_block": best.threads_per_block,
                         "propose_chunk": best.propose_chunk, "search": "axis by axis",
                         "candidates": [[c.cell_delta, c.blocks_per_sm, c.groups, c.threads_per_block,
                                         c.propose_chunk, round(c.ms_per_step, 4)] for c in tried],
                         "candidate_fields": ["cell_delta", "blocks_per_sm", "groups", "threads_per_block",
                                              "propose_chunk", "ms_per_step"]},
            "batched_value": batched, "serial_value": serial, "unit": UNIT,
            "batched_over_serial": batched / serial, "batched_ms_per_step": batched_ms / steps,
            "serial_ms_per_round": serial_ms / steps}


def run_serve(A, seconds, budget=150e9, groups=1, rate=20.0, drain=False, admission="backfill"):
    """Served workload: Poisson arrivals (rate per s, seed 7) of cascade or
    two-compartment jobs, 10k-2M agents, 1k-20k steps, admitted under an HBM
    budget, continuous batching; `seconds` of arrivals in real time.  Without
    drain the run stops at the end of the window and the jobs still queued or
    running count in the latency at their age then (censored, lower bounds);
    with drain every arrived job is served to completion."""
    import workloads as W
    from paper_2606_14603_b300 import serve
    jobs = W.served_jobs(duration_s=seconds, rate_per_s=rate)
    srv = serve.Server(budget_bytes=budget, groups=groups)
    out = serve.run(jobs, srv, duration_s=seconds, real_time=True, drain=drain, admission=admission)
    srv.close()
    out.pop("results")
    out.pop("failed")
    out["arrival_rate_per_s"] = rate
    out["budget_bytes"] = budget
    out["window_s"] = seconds
    out["drained"] = drain
    out["groups"] = groups
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, rank)
        return

    import numpy as np
    import torch
    from paper_2606_14603_b300 import build as engine_build
    engine_build.build()
    import paper_2606_14603_b300 as A

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    if args.workload == "serve":
        with Clocks(local) as clk:
            sv = run_serve(A, args.serve_seconds, groups=args.serve_groups, rate=args.serve_rate,
                           admission=args.serve_admission)
        line = {"metric": METRIC, "value": sv["throughput_molecule_steps_per_s"], "unit": UNIT, "n_gpus": world,
                "steps": sv["steps_run"], "warmup": 0, "ms_per_step": None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": f"served_poisson_{args.serve_rate:g}_per_s", "window_s": args.serve_seconds,
                           "budget_gb": 150, "admission": args.serve_admission},
                "serve": sv, "clocks": clk.summary()}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return

    if args.workload == "sweep":
        stream = torch.cuda.Stream()
        with Clocks(local) as clk:
            sw = run_sweep(A, torch, stream, args.steps, args.warmup, cpu=not args.no_cpu_baseline and world == 1)
        line = {"metric": METRIC, "value": sw["batched_value"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": sw["batched_ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
                "data": "synthetic",
                "config": {"workload": "sweep_64_sims_50k_500k", "agents": sw["agents"],
                           "l2": "no flush (batched state 12.6M agents exceeds L2)"},
                "sweep": sw, "gpu_launches": launches_per_step(sw["agents"]) * args.steps, "clocks": clk.summary()}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return

    model, seed, name = workload(args)
    seed = seed + rank                      # independent replicas
    stream = torch.cuda.Stream()
    sim = A.Sim(model, seed, stream=stream)
    sim_cells = sim.grid_cells()
    flush = None if args.no_flush else torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flush_src = None if args.no_flush else torch.ones(64 << 20, dtype=torch.float32, device="cuda")

    def flush_l2():
        # write 256 MB (evicts the simulation state from the 126 MB L2), then
        # read 256 MB so that the flush's own dirty lines are written back here
        # and not inside the next timed step
        with torch.cuda.stream(stream):
            flush.zero_()
            flush_src.sum()

    # warm-up (untimed); one flush too, so that loading the flush's kernels
    # falls outside the timed region
    sim.step(args.warmup)
    if flush is not None:
        flush_l2()
    sim.sync()
    n_before = molecules(sim.counts(), model)

    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        wall0 = time.perf_counter()
        for k in range(K):
            if flush is not None:
                flush_l2()
            starts[k].record(stream)
            sim.step(1)
            ends[k].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        clk.mark(wall0, wall0 + wall)
    sim.sync()
    if dist:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = float(sum(step_ms))
    n_after = molecules(sim.counts(), model)
    mol_steps = 0.5 * (n_before + n_after) * K
    if dist:
        total_ms_max, mol_steps_all = reduce_over_ranks(total_ms, mol_steps)
    else:
        total_ms_max, mol_steps_all = total_ms, mol_steps
    value = mol_steps_all / (total_ms_max / 1e3)
    per_step = sorted(step_ms)

    # per-kernel breakdown with the same L2 state (flushed before each step)
    prof = {k: 0.0 for k in KERNEL_BYTES}
    P = max(1, args.profile_steps)
    for _ in range(P):
        if flush is not None:
            flush_l2()
        for k, v in sim.profile_step(1).items():
            prof[k] += v
    tot = sum(prof.values())
    share = {k: v / tot for k, v in prof.items()}
    dom = max(prof, key=prof.get)
    peaks, peak_src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    n_agents = 0.5 * (n_before + n_after)
    bpu, unit_name = KERNEL_BYTES[dom]
    units = n_agents
    if unit_name == "cell":
        units = sim.grid_cells()
    dom_ms = prof[dom] / P
    achieved = bpu * units / (dom_ms / 1e3) / 1e9
    traffic = ncu_traffic(dom)
    # the dominant kernel's time inside the graphed step (launches overlap through
    # programmatic dependent launch there): its share of the event-timed kernels
    # times the graphed step time
    step_ms_avg = total_ms / K
    dom_ms_graph = share[dom] * step_ms_avg
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic[0] if traffic else None,
            "bytes_per_unit": bpu, "units_per_launch": units, "unit_of_work": unit_name,
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback 6.4 TB/s",
            "kernel_ms": dom_ms,
            "kernel_ms_is": ("CUDA events around the kernel, the step's kernels serialised (no overlap between "
                             "kernels), events and launches replayed as one graph (frac uses this)"),
            "kernel_ms_graph_est": dom_ms_graph,
            "frac_graph_est": bpu * units / (dom_ms_graph / 1e3) / 1e9 / hbm,
            "traffic_source": (f"ncu {traffic[3]}" if traffic and len(traffic) > 3 else None)}
    step_roof = {"bytes_per_molecule_step": STEP_BYTES_PER_AGENT,
                 "achieved_gbs": STEP_BYTES_PER_AGENT * n_agents / (step_ms_avg / 1e3) / 1e9,
                 "frac": STEP_BYTES_PER_AGENT * n_agents / (step_ms_avg / 1e3) / 1e9 / hbm}

    # end to end, through the C ABI with host-side inputs and outputs: the
    # model structs go in by abm_create (upload and device-side placement,
    # timed and reported on its own), then E2E_STEPS times (abm_step + that
    # step's counts vector back to the host): pipelined (the step keeps its
    # result's counts; each step's copy is queued into a pinned slot and
    # collected while the next step runs) and, for comparison, synchronous
    # (abm_counts, a counting pass and a wait, after every step).  `value`
    # charges the creation to the loop (creation + steps); `steady_value`
    # is the loop alone.  Fixed step count, independent of --steps.
    e2e = None
    if not args.no_e2e:
        Ke = E2E_STEPS

        def e2e_run(pipelined):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s2 = A.Sim(model, seed, stream=stream)
            if pipelined:
                s2.live_counts(True)  # each step keeps its result's counts: a read is a copy
            s2.sync()
            t1 = time.perf_counter()
            cvec = None
            for k in range(Ke):
                s2.step(1)
                if pipelined:
                    s2.counts_begin(k % 2)
                    if k:
                        cvec = s2.counts_finish((k - 1) % 2)
                else:
                    cvec = s2.counts()
            if pipelined:
                cvec = s2.counts_finish((Ke - 1) % 2)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            s2.close()
            return cvec, t1 - t0, t2 - t1

        cvec, cr, loop = e2e_run(True)
        cvec_s, cr_s, loop_s = e2e_run(False)
        assert np.array_equal(cvec, cvec_s)
        n_counts = len(cvec)
        # host-to-device at creation: Gaussian table, integer model tables, sim entry, control words
        model_bytes = 2 * 65536 + 15376 + 512
        ms_e2e = molecules(cvec, model) * Ke
        e2e = {"value": ms_e2e / (cr + loop), "unit": UNIT,
               "h2d_bytes_per_step": model_bytes / Ke, "d2h_bytes_per_step": 8 * n_counts,
               "steps": Ke, "create_s": cr, "loop_s": loop, "steady_value": ms_e2e / loop,
               "includes": f"abm_create (model upload, device-side placement; create_s) + {Ke} x "
                           "(abm_step + that step's counts read back to the host: live counts, "
                           "abm_counts_begin / abm_counts_finish, one step in flight); "
                           "steady_value excludes the creation",
               "synchronous_value": ms_e2e / (cr_s + loop_s), "synchronous_steady_value": ms_e2e / loop_s}

    sweep = None
    if args.sweep_steps > 0 and args.workload == "cascade" and not args.agents:
        sweep = run_sweep(A, torch, stream, args.sweep_steps, cpu=not args.no_cpu_baseline and world == 1)

    served = served_sub = None
    if args.serve_seconds > 0 and args.workload == "cascade" and not args.agents:
        sim.close()
        served = run_serve(A, args.serve_seconds, groups=args.serve_groups, rate=args.serve_rate,
                           admission=args.serve_admission)
        if args.serve_sub_rate > 0:
            served_sub = run_serve(A, args.serve_seconds, groups=args.serve_groups, rate=args.serve_sub_rate,
                                   drain=True, admission=args.serve_admission)
        sim = None

    sizes = None
    if args.size_steps > 0 and args.workload == "cascade" and not args.agents:
        if sim is not None:
            sim.close()
            sim = None
        import workloads as W
        sizes = []
        for n_big in (4_000_000, 16_000_000):
            big = W.mapk(n_big)
            bs = A.Sim(big, W.MAPK_SEED, stream=stream)
            bs.step(5)
            bs.sync()
            t_ms = []
            for _ in range(args.size_steps):
                if flush is not None:
                    flush_l2()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                bs.step(1)
                e1.record(stream)
                t_ms.append((e0, e1))
            torch.cuda.synchronize()
            ms = sorted(a.elapsed_time(b) for a, b in t_ms)
            live = molecules(bs.counts(), big)
            rate = live * len(ms) / (sum(ms) / 1e3)
            sizes.append({"agents": n_big, "steps": len(ms), "value": rate, "unit": UNIT,
                          "ms_per_step": sum(ms) / len(ms), "p50_step_ms": ms[len(ms) // 2],
                          "step_roofline_frac": rate * STEP_BYTES_PER_AGENT / 1e9 / hbm,
                          "l2": "flushed between steps"})
            bs.close()

    births = None
    if args.births_steps > 0 and args.workload == "cascade" and not args.agents:
        import workloads as W
        bm = W.births(50_000)
        bsim = A.Sim(bm, 31, capacity=1_000_000, births_per_step=80_000, stream=stream)
        bsim.step(5)
        c0 = bsim.counts()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bsim.step(args.births_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        c1 = bsim.counts()
        ms = e0.elapsed_time(e1) / args.births_steps
        births = {"model": "births(50,000 expressors, p_emit 1; children emit and degrade)",
                  "steps": args.births_steps, "ms_per_step": ms,
                  "births_per_step": float(c1[-1] - c0[-1]) / args.births_steps,
                  "agents_live": molecules(c1, bm), "l2": "not flushed (state below L2)"}
        bsim.close()

    volume = None
    if args.volume_steps > 0 and args.workload == "cascade" and not args.agents:
        from paper_2606_14603_b300.experiments import volume_invariance
        import workloads as W
        volume = volume_invariance(lambda n, d: W.mapk(n, d), [0.0, 0.02, 0.05, 0.10], 1_000_000,
                                   factor=10, steps=args.volume_steps, stream=stream)
        volume["note"] = ("cascade at 1x (1M agents per dose) and 10x volume (10M) at the same "
                          "concentrations, one batch per volume; change_pct = final vs initial "
                          "pERK+ppERK (free + in complexes), percent")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(model, seed, name)

    clocks = clk.summary()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": total_ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": config_of(args, model, name, {"parallelism": f"replicas x{world}",
                                                    "seed": seed - rank}),
            "p50_step_ms": per_step[len(per_step) // 2], "p99_step_ms": per_step[int(0.99 * (len(per_step) - 1))],
            "roofline": roof, "step_roofline": step_roof,
            "kernel_share": share, "kernel_ms_per_step": {k: v / P for k, v in prof.items()},
            "gpu_launches": launches_per_step(sim_cells) * K, "e2e": e2e, "cpu_baseline": cpu, "sweep": sweep,
            "serve": served, "serve_subcapacity": served_sub, "sizes": sizes, "births": births, "volume": volume,
            "clocks": clocks, "wall_s_timed_region": wall}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if sim is not None:
        sim.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
