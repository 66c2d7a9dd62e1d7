"""Python binding of the B300 molecule-agent step engine (C ABI in include/abm.h).

Argument marshalling only: every step runs in the CUDA kernels of libabm.so.
PyTorch may supply the device arena (a uint8 CUDA tensor) and the stream;
otherwise the library allocates its own.  There is no CPU fallback: if the
library cannot be loaded or no sm_103 device is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libabm.so")
READ_SLOTS = 4  # pinned slots of the pipelined counts reads (ABM_READ_SLOTS)

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ECAPACITY, EDEVICE, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
_NAMES = {0: "ABM_OK", -1: "ABM_EINVAL", -2: "ABM_ENOMEM", -3: "ABM_ECUDA", -4: "ABM_ETIMEOUT",
          -5: "ABM_ECAPACITY", -6: "ABM_EDEVICE", -7: "ABM_ESTATE"}

RECORD_DTYPE = np.dtype([("id", "<u4"), ("sp", "u1"), ("comp", "u1"), ("flags", "u1"),
                         ("rxn", "u1"), ("x", "<i4"), ("y", "<i4"), ("z", "<i4"),
                         ("partner", "<u4")])


class AbmError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        super().__init__(f"{_NAMES.get(status, status)}: {msg}")
        self.status = status


class Species(C.Structure):
    _fields_ = [("initial_count", C.c_uint32), ("D_um2_s", C.c_double), ("compartment", C.c_int32),
                ("p_cross", C.c_double), ("p_uni", C.c_double), ("uni_to", C.c_int32),
                ("p_emit", C.c_double), ("emit_species", C.c_int32)]


class Reaction(C.Structure):
    _fields_ = [("a", C.c_int32), ("b", C.c_int32), ("kind", C.c_int32), ("prod_a", C.c_int32),
                ("prod_b", C.c_int32), ("radius_nm", C.c_double), ("p_bind", C.c_double),
                ("p_release", C.c_double)]


class Compartment(C.Structure):
    _fields_ = [("shape", C.c_int32), ("size_um", C.c_double), ("parent", C.c_int32),
                ("center_um", C.c_double * 3)]


class Model(C.Structure):
    _fields_ = [("species", C.POINTER(Species)), ("n_species", C.c_uint32),
                ("reactions", C.POINTER(Reaction)), ("n_reactions", C.c_uint32),
                ("compartments", C.POINTER(Compartment)), ("n_compartments", C.c_uint32),
                ("dt_s", C.c_double), ("unit_nm", C.c_double)]


class Options(C.Structure):
    _fields_ = [("capacity_agents", C.c_uint64), ("cell_log2", C.c_uint32),
                ("births_per_step", C.c_uint32), ("arena", C.c_void_p), ("arena_bytes", C.c_size_t),
                ("stream", C.c_void_p), ("ncdf_table", C.c_void_p)]


class BatchOptions(C.Structure):
    _fields_ = [("capacity_agents", C.c_uint64), ("capacity_cells", C.c_uint64),
                ("max_sims", C.c_uint32), ("births_per_step", C.c_uint32), ("arena", C.c_void_p),
                ("arena_bytes", C.c_size_t), ("stream", C.c_void_p), ("ncdf_table", C.c_void_p),
                ("blocks_per_sm", C.c_uint32), ("threads_per_block", C.c_uint32),
                ("propose_chunk", C.c_uint32)]


class Monitor(C.Structure):
    _fields_ = [("step_begin", C.c_uint32), ("step_end", C.c_uint32), ("period", C.c_uint32),
                ("above", C.c_int32), ("threshold", C.c_int64)]


class MonitorStateC(C.Structure):
    _fields_ = [("value", C.c_int64), ("last_step", C.c_uint32), ("first_pass", C.c_uint32),
                ("n_evaluated", C.c_uint32), ("n_passed", C.c_uint32), ("state", C.c_int32),
                ("reserved", C.c_uint32)]


@dataclasses.dataclass
class MonitorState:
    """A threshold monitor's state: the last evaluated value and step, the
    first step that passed (None if none), counts, the last outcome (True /
    False / None before any evaluation) and the evaluated values, oldest
    first (the last 1024 at most)."""
    value: int
    last_step: int
    first_pass: Optional[int]
    n_evaluated: int
    n_passed: int
    state: Optional[bool]
    trace: np.ndarray


_lib = None


def lib():
    """Load libabm.so (built in-tree by build.py); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2606_14603_b300/build.py")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        sig = {
            "abm_arena_bytes": (C.c_size_t, [C.POINTER(Model), C.POINTER(Options)]),
            "abm_create": (C.c_int, [C.POINTER(Model), C.c_uint64, C.POINTER(Options), C.POINTER(P)]),
            "abm_restore": (C.c_int, [C.POINTER(Model), C.c_uint64, C.POINTER(Options), P, C.c_size_t,
                                      C.c_uint32, C.c_uint32, C.POINTER(P)]),
            "abm_batch_restore": (C.c_int, [P, C.POINTER(Model), C.c_uint64, C.c_uint32, P, C.c_size_t,
                                            C.c_uint32, C.c_uint32, C.POINTER(C.c_int32)]),
            "abm_step": (C.c_int, [P, C.c_uint32]),
            "abm_counts": (C.c_int, [P, P, C.c_size_t, C.POINTER(C.c_size_t)]),
            "abm_counts_begin": (C.c_int, [P, C.c_uint32]),
            "abm_live_counts": (C.c_int, [P, C.c_int]),
            "abm_counts_finish": (C.c_int, [P, C.c_uint32, P, C.c_size_t, C.POINTER(C.c_size_t)]),
            "abm_digest": (C.c_int, [P, C.POINTER(C.c_uint64)]),
            "abm_dump": (C.c_int, [P, P, C.c_size_t, C.POINTER(C.c_size_t)]),
            "abm_sync": (C.c_int, [P]),
            "abm_step_index": (C.c_int, [P, C.POINTER(C.c_uint32)]),
            "abm_last_error": (C.c_char_p, [P]),
            "abm_destroy": (None, [P]),
            "abm_batch_arena_bytes": (C.c_size_t, [C.POINTER(BatchOptions)]),
            "abm_batch_create": (C.c_int, [C.POINTER(BatchOptions), C.POINTER(P)]),
            "abm_batch_add": (C.c_int, [P, C.POINTER(Model), C.c_uint64, C.c_uint32, C.POINTER(C.c_int32)]),
            "abm_batch_remove": (C.c_int, [P, C.c_int32]),
            "abm_batch_set_max_step": (C.c_int, [P, C.c_int32, C.c_uint32]),
            "abm_batch_step": (C.c_int, [P, C.c_uint32]),
            "abm_batch_counts": (C.c_int, [P, C.c_int32, P, C.c_size_t, C.POINTER(C.c_size_t)]),
            "abm_batch_counts_begin": (C.c_int, [P, C.c_int32, C.c_uint32]),
            "abm_batch_live_counts": (C.c_int, [P, C.c_int]),
            "abm_batch_counts_finish": (C.c_int, [P, C.c_uint32, P, C.c_size_t, C.POINTER(C.c_size_t)]),
            "abm_batch_digest": (C.c_int, [P, C.c_int32, C.POINTER(C.c_uint64)]),
            "abm_batch_dump": (C.c_int, [P, C.c_int32, P, C.c_size_t, C.POINTER(C.c_size_t)]),
            "abm_batch_sync": (C.c_int, [P]),
            "abm_batch_sim_status": (C.c_int, [P, C.c_int32]),
            "abm_batch_live_agents": (C.c_int, [P, C.POINTER(C.c_uint64)]),
            "abm_batch_last_error": (C.c_char_p, [P]),
            "abm_batch_destroy": (None, [P]),
            "abm_ncdf_table": (None, [P]),
            "abm_debug_philox": (C.c_int, [P, P, P, C.c_size_t]),
            "abm_version": (C.c_char_p, []),
            "abm_profile_step": (C.c_int, [P, C.c_uint32, P, C.c_uint32]),
            "abm_batch_profile_step": (C.c_int, [P, C.c_uint32, P, C.c_uint32]),
            "abm_kernel_name": (C.c_char_p, [C.c_uint32]),
            "abm_grid_cells": (C.c_int, [P, C.POINTER(C.c_uint64)]),
            "abm_model_grid": (C.c_int, [C.POINTER(Model), C.c_uint32, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)]),
            "abm_debug_inject_launch_error": (None, [C.c_int]),
            "abm_monitor_set": (C.c_int, [P, C.POINTER(Monitor), P, C.c_size_t]),
            "abm_monitor_clear": (C.c_int, [P]),
            "abm_monitor_read": (C.c_int, [P, C.POINTER(MonitorStateC), P, C.c_size_t, C.POINTER(C.c_size_t)]),
            "abm_batch_monitor_set": (C.c_int, [P, C.c_int32, C.POINTER(Monitor), P, C.c_size_t]),
            "abm_batch_monitor_clear": (C.c_int, [P, C.c_int32]),
            "abm_batch_monitor_read": (C.c_int, [P, C.c_int32, C.POINTER(MonitorStateC), P, C.c_size_t,
                                                 C.POINTER(C.c_size_t)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return [n for n in dir(lib()) if n.startswith("abm_")]


class _ModelStructs:
    """C structs for a model description (any object with .species,
    .reactions, .compartments, .dt_s, .unit_nm in the workloads layout)."""

    def __init__(self, model):
        sp = (Species * len(model.species))()
        for i, s in enumerate(model.species):
            sp[i] = Species(s.count, s.D, s.comp, s.p_cross, s.p_uni, s.uni_to, s.p_emit, s.emit)
        n_rx = len(model.reactions)
        rx = (Reaction * max(1, n_rx))()
        for i, r in enumerate(model.reactions):
            rx[i] = Reaction(r.a, r.b, r.kind, r.prod_a, r.prod_b, r.radius_nm, r.p_bind, r.p_release)
        cm = (Compartment * len(model.compartments))()
        for i, c in enumerate(model.compartments):
            cm[i] = Compartment(c.shape, c.size_um, c.parent, (C.c_double * 3)(*c.center_um))
        self._keep = (sp, rx, cm)
        self.model = Model(sp, len(model.species), rx, n_rx, cm, len(model.compartments),
                           model.dt_s, model.unit_nm)
        self.n_counts = len(model.species) * len(model.compartments) + n_rx + 1


def _check(st, err_fn=None, handle=None):
    if st != OK:
        msg = ""
        if err_fn is not None and handle is not None:
            m = err_fn(handle)
            msg = m.decode() if m else ""
        raise AbmError(st, msg)


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream) or None
    return int(stream) or None


def arena_bytes(model, capacity: int = 0, cell_log2: int = 0, births_per_step: int = 0) -> int:
    ms = _ModelStructs(model)
    o = Options(capacity, cell_log2, births_per_step, None, 0, None, None)
    return lib().abm_arena_bytes(C.byref(ms.model), C.byref(o))


def model_grid(model, cell_log2: int = 0):
    """(cell_log2, cells) of a model's grid, without touching the device."""
    ms = _ModelStructs(model)
    sh, cells = C.c_uint32(), C.c_uint64()
    _check(lib().abm_model_grid(C.byref(ms.model), cell_log2, C.byref(sh), C.byref(cells)))
    return sh.value, cells.value


def monitor_weights(model, species, include_bound: bool = True, compartments=None) -> np.ndarray:
    """Weights over the counts vector that add up the given species (names or
    indices): their free agents in the given compartments (all by default)
    and, with include_bound, one per bound complex that contains one of them."""
    names = [s.name for s in model.species]
    idx = {names.index(s) if isinstance(s, str) else int(s) for s in species}
    n_comp = len(model.compartments)
    comps = range(n_comp) if compartments is None else compartments
    w = np.zeros(len(model.species) * n_comp + len(model.reactions), dtype=np.int32)
    for sp in idx:
        for c in comps:
            w[sp * n_comp + c] = 1
    if include_bound:
        for r, rx in enumerate(model.reactions):
            w[len(model.species) * n_comp + r] = int(rx.a in idx) + int(rx.b in idx)
    return w


def _monitor_args(weights, threshold, above, begin, end, period):
    w = np.ascontiguousarray(weights, dtype=np.int32)
    m = Monitor(begin, 0xFFFFFFFF if end is None else end, period, 1 if above else 0, int(threshold))
    return m, w


def _monitor_state(st: MonitorStateC, trace: np.ndarray, n: int) -> MonitorState:
    return MonitorState(int(st.value), int(st.last_step),
                        None if st.first_pass == 0xFFFFFFFF else int(st.first_pass),
                        int(st.n_evaluated), int(st.n_passed), None if st.state < 0 else bool(st.state),
                        trace[:n].copy())


def batch_capacity(models, headroom: float = 1.25, cell_log2_delta: int = 0):
    """(capacity_agents, capacity_cells) for a batch of these models."""
    agents = sum(m.n_agents for m in models)
    cells = 0
    for m in models:
        sh, _ = model_grid(m)
        cells += model_grid(m, max(1, sh + cell_log2_delta))[1] if cell_log2_delta else model_grid(m)[1]
    return int(agents * headroom) + 65536, cells


class Sim:
    """One simulation on the GPU.  `arena` may be a torch uint8 CUDA tensor of
    at least arena_bytes(...) bytes (kept alive by this object); `stream` a
    torch.cuda.Stream or a raw cudaStream_t."""

    def __init__(self, model, seed: int, capacity: int = 0, cell_log2: int = 0,
                 births_per_step: int = 0, arena=None, stream=None, ncdf_table=None, restore=None):
        """restore=(records, step, next_id) resumes from a checkpoint (see
        checkpoint()) instead of placing the model's initial agents."""
        L = lib()
        ms = _ModelStructs(model)
        self.n_counts = ms.n_counts
        self._arena = arena
        self._table = None
        tptr = None
        if ncdf_table is not None:
            self._table = np.ascontiguousarray(ncdf_table, dtype=np.int16)
            tptr = self._table.ctypes.data
        aptr, abytes = (None, 0)
        if arena is not None:
            aptr, abytes = arena.data_ptr(), arena.numel() * arena.element_size()
        o = Options(capacity, cell_log2, births_per_step, aptr, abytes, _stream_ptr(stream), tptr)
        h = C.c_void_p()
        if restore is None:
            st = L.abm_create(C.byref(ms.model), seed, C.byref(o), C.byref(h))
        else:
            rec, step, next_id = restore
            rec = np.ascontiguousarray(rec, dtype=RECORD_DTYPE)
            st = L.abm_restore(C.byref(ms.model), seed, C.byref(o), rec.ctypes.data if len(rec) else None,
                               len(rec), step, next_id, C.byref(h))
        if st != OK:
            raise AbmError(st, "abm_create failed" if restore is None else "abm_restore failed")
        self._h = h

    def step(self, n: int = 1) -> None:
        _check(lib().abm_step(self._h, n), lib().abm_last_error, self._h)

    def sync(self) -> None:
        _check(lib().abm_sync(self._h), lib().abm_last_error, self._h)

    def counts(self) -> np.ndarray:
        out = np.zeros(self.n_counts, dtype=np.uint64)
        n = C.c_size_t()
        _check(lib().abm_counts(self._h, out.ctypes.data, out.size, C.byref(n)), lib().abm_last_error, self._h)
        return out

    def live_counts(self, on: bool = True) -> None:
        """Every step also keeps the counts of its result (counts_begin then
        needs no pass over the agents)."""
        _check(lib().abm_live_counts(self._h, 1 if on else 0), lib().abm_last_error, self._h)

    def counts_begin(self, slot: int = 0) -> None:
        """Queue a counts read of the state after the steps issued so far into
        pinned slot `slot` (0..READ_SLOTS-1); returns at once."""
        _check(lib().abm_counts_begin(self._h, slot), lib().abm_last_error, self._h)

    def counts_finish(self, slot: int = 0) -> np.ndarray:
        """Wait for the counts read queued in `slot` and return them."""
        out = np.zeros(self.n_counts, dtype=np.uint64)
        n = C.c_size_t()
        _check(lib().abm_counts_finish(self._h, slot, out.ctypes.data, out.size, C.byref(n)),
               lib().abm_last_error, self._h)
        return out

    def digest(self) -> int:
        v = C.c_uint64()
        _check(lib().abm_digest(self._h, C.byref(v)), lib().abm_last_error, self._h)
        return v.value

    def dump(self) -> np.ndarray:
        n = C.c_size_t()
        _check(lib().abm_dump(self._h, None, 0, C.byref(n)), lib().abm_last_error, self._h)
        out = np.zeros(n.value, dtype=RECORD_DTYPE)
        m = C.c_size_t()
        _check(lib().abm_dump(self._h, out.ctypes.data, out.size, C.byref(m)), lib().abm_last_error, self._h)
        return out[: m.value]

    def checkpoint(self):
        """(records, step, next_id): everything needed to resume this simulation."""
        return self.dump(), self.t, int(self.counts()[-1])

    def profile_step(self, n: int = 1) -> dict:
        """n un-graphed steps with CUDA events around each kernel: ms per kernel."""
        ms = np.zeros(8, dtype=np.float32)
        _check(lib().abm_profile_step(self._h, n, ms.ctypes.data, 8), lib().abm_last_error, self._h)
        return {kernel_name(k): float(ms[k]) for k in range(N_STEP_KERNELS)}

    def monitor(self, weights, threshold: int, above: bool = True, begin: int = 0,
                end: Optional[int] = None, period: int = 1) -> None:
        """Install a threshold monitor: sum(weights * counts) against threshold
        at steps begin, begin + period, ... below end (None = open)."""
        m, w = _monitor_args(weights, threshold, above, begin, end, period)
        _check(lib().abm_monitor_set(self._h, C.byref(m), w.ctypes.data if w.size else None, w.size),
               lib().abm_last_error, self._h)

    def monitor_clear(self) -> None:
        _check(lib().abm_monitor_clear(self._h), lib().abm_last_error, self._h)

    def monitor_read(self) -> MonitorState:
        st, tr, n = MonitorStateC(), np.zeros(1024, dtype=np.int64), C.c_size_t()
        _check(lib().abm_monitor_read(self._h, C.byref(st), tr.ctypes.data, tr.size, C.byref(n)),
               lib().abm_last_error, self._h)
        return _monitor_state(st, tr, n.value)

    def grid_cells(self) -> int:
        """Cells of this simulation's grid."""
        v = C.c_uint64()
        _check(lib().abm_grid_cells(self._h, C.byref(v)), lib().abm_last_error, self._h)
        return v.value

    @property
    def t(self) -> int:
        v = C.c_uint32()
        _check(lib().abm_step_index(self._h, C.byref(v)), lib().abm_last_error, self._h)
        return v.value

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().abm_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many simulations stepped together in one set of launches (per-sim offset
    tables on the device).  Simulations may be added and removed between steps."""

    def __init__(self, capacity_agents: int, capacity_cells: int, max_sims: int,
                 births_per_step: int = 0, arena=None, stream=None, blocks_per_sm: int = 0,
                 threads_per_block: int = 0, propose_chunk: int = 0):
        L = lib()
        aptr, abytes = (None, 0)
        if arena is not None:
            aptr, abytes = arena.data_ptr(), arena.numel() * arena.element_size()
        self._arena = arena
        o = BatchOptions(capacity_agents, capacity_cells, max_sims, births_per_step, aptr, abytes,
                         _stream_ptr(stream), None, blocks_per_sm, threads_per_block, propose_chunk)
        h = C.c_void_p()
        st = L.abm_batch_create(C.byref(o), C.byref(h))
        if st != OK:
            raise AbmError(st, "abm_batch_create failed")
        self._h = h
        self._n_counts = {}
        self._read_sims = {}  # pipelined counts reads in flight: slot -> simulation

    @staticmethod
    def arena_bytes(capacity_agents: int, capacity_cells: int, max_sims: int, births_per_step: int = 0) -> int:
        o = BatchOptions(capacity_agents, capacity_cells, max_sims, births_per_step, None, 0, None, None, 0, 0, 0)
        return lib().abm_batch_arena_bytes(C.byref(o))

    def add(self, model, seed: int, cell_log2: int = 0) -> int:
        ms = _ModelStructs(model)
        sid = C.c_int32(-1)
        _check(lib().abm_batch_add(self._h, C.byref(ms.model), seed, cell_log2, C.byref(sid)),
               lib().abm_batch_last_error, self._h)
        self._n_counts[sid.value] = ms.n_counts
        return sid.value

    def set_max_step(self, sim: int, max_step: int) -> None:
        """Freeze `sim` once its step counter reaches max_step."""
        _check(lib().abm_batch_set_max_step(self._h, sim, max_step), lib().abm_batch_last_error, self._h)

    def remove(self, sim: int) -> None:
        _check(lib().abm_batch_remove(self._h, sim), lib().abm_batch_last_error, self._h)
        self._n_counts.pop(sim, None)

    def step(self, n: int = 1) -> None:
        _check(lib().abm_batch_step(self._h, n), lib().abm_batch_last_error, self._h)

    def sync(self) -> None:
        _check(lib().abm_batch_sync(self._h), lib().abm_batch_last_error, self._h)

    def live_agents(self) -> int:
        v = C.c_uint64()
        _check(lib().abm_batch_live_agents(self._h, C.byref(v)), lib().abm_batch_last_error, self._h)
        return v.value

    def sim_status(self, sim: int) -> tuple:
        """(status, message) of one simulation: (OK, "") or, for a simulation
        stopped by its own error (births of one step beyond its limit), the
        status and the library's message; the batch itself stays usable."""
        st = lib().abm_batch_sim_status(self._h, sim)
        if st == OK:
            return OK, ""
        msg = lib().abm_batch_last_error(self._h).decode()
        if st == ESTATE and "simulation" not in msg:
            raise AbmError(st, msg)
        return st, msg

    def counts(self, sim: int) -> np.ndarray:
        out = np.zeros(self._n_counts[sim], dtype=np.uint64)
        n = C.c_size_t()
        _check(lib().abm_batch_counts(self._h, sim, out.ctypes.data, out.size, C.byref(n)),
               lib().abm_batch_last_error, self._h)
        return out

    def live_counts(self, on: bool = True) -> None:
        """Every step also keeps the counts of its result (counts_begin then
        needs no pass over the agents)."""
        _check(lib().abm_batch_live_counts(self._h, 1 if on else 0), lib().abm_batch_last_error, self._h)

    def counts_begin(self, sim: int, slot: int = 0) -> None:
        """Queue a counts read of simulation `sim` into pinned slot `slot`."""
        _check(lib().abm_batch_counts_begin(self._h, sim, slot), lib().abm_batch_last_error, self._h)
        self._read_sims[slot] = sim

    def counts_finish(self, slot: int = 0) -> np.ndarray:
        """Wait for the counts read queued in `slot` and return them."""
        sim = self._read_sims.pop(slot, None)
        out = np.zeros(self._n_counts.get(sim, 512), dtype=np.uint64)  # (the sim may be gone since)
        n = C.c_size_t()
        _check(lib().abm_batch_counts_finish(self._h, slot, out.ctypes.data, out.size, C.byref(n)),
               lib().abm_batch_last_error, self._h)
        return out[: n.value]

    def digest(self, sim: int) -> int:
        v = C.c_uint64()
        _check(lib().abm_batch_digest(self._h, sim, C.byref(v)), lib().abm_batch_last_error, self._h)
        return v.value

    def dump(self, sim: int) -> np.ndarray:
        n = C.c_size_t()
        _check(lib().abm_batch_dump(self._h, sim, None, 0, C.byref(n)), lib().abm_batch_last_error, self._h)
        out = np.zeros(n.value, dtype=RECORD_DTYPE)
        m = C.c_size_t()
        _check(lib().abm_batch_dump(self._h, sim, out.ctypes.data, out.size, C.byref(m)),
               lib().abm_batch_last_error, self._h)
        return out[: m.value]

    def monitor(self, sim: int, weights, threshold: int, above: bool = True, begin: int = 0,
                end: Optional[int] = None, period: int = 1) -> None:
        m, w = _monitor_args(weights, threshold, above, begin, end, period)
        _check(lib().abm_batch_monitor_set(self._h, sim, C.byref(m), w.ctypes.data if w.size else None, w.size),
               lib().abm_batch_last_error, self._h)

    def monitor_clear(self, sim: int) -> None:
        _check(lib().abm_batch_monitor_clear(self._h, sim), lib().abm_batch_last_error, self._h)

    def monitor_read(self, sim: int) -> MonitorState:
        st, tr, n = MonitorStateC(), np.zeros(1024, dtype=np.int64), C.c_size_t()
        _check(lib().abm_batch_monitor_read(self._h, sim, C.byref(st), tr.ctypes.data, tr.size, C.byref(n)),
               lib().abm_batch_last_error, self._h)
        return _monitor_state(st, tr, n.value)

    def profile_step(self, n: int = 1) -> dict:
        ms = np.zeros(8, dtype=np.float32)
        _check(lib().abm_batch_profile_step(self._h, n, ms.ctypes.data, 8), lib().abm_batch_last_error, self._h)
        return {kernel_name(k): float(ms[k]) for k in range(N_STEP_KERNELS)}

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().abm_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


N_STEP_KERNELS = 6


def kernel_name(k: int) -> str:
    return lib().abm_kernel_name(k).decode()


def ncdf_table() -> np.ndarray:
    out = np.zeros(65536, dtype=np.int16)
    lib().abm_ncdf_table(out.ctypes.data)
    return out


def inject_launch_error(cuda_error: int) -> None:
    """Testing hook: the next step call fails as if its launch had returned
    this CUDA error (host side only; see include/abm.h)."""
    lib().abm_debug_inject_launch_error(cuda_error)


def device_philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """The engine's device Philox4x32-10 on rows of ctr (n,4) and key (n,2)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(ctr)
    _check(lib().abm_debug_philox(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, ctr.shape[0]))
    return out
