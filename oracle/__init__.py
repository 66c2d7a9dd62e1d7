"""ctypes binding of the serial CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py.  The product package never imports
it, and it never imports the product package.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

RECORD_DTYPE = np.dtype([("id", "<u4"), ("sp", "u1"), ("comp", "u1"), ("flags", "u1"),
                         ("rxn", "u1"), ("x", "<i4"), ("y", "<i4"), ("z", "<i4"),
                         ("partner", "<u4")])


class _Species(C.Structure):
    _fields_ = [("initial_count", C.c_uint32), ("D_um2_s", C.c_double), ("compartment", C.c_int32),
                ("p_cross", C.c_double), ("p_uni", C.c_double), ("uni_to", C.c_int32),
                ("p_emit", C.c_double), ("emit_species", C.c_int32)]


class _Reaction(C.Structure):
    _fields_ = [("a", C.c_int32), ("b", C.c_int32), ("kind", C.c_int32), ("prod_a", C.c_int32),
                ("prod_b", C.c_int32), ("radius_nm", C.c_double), ("p_bind", C.c_double),
                ("p_release", C.c_double)]


class _Compartment(C.Structure):
    _fields_ = [("shape", C.c_int32), ("size_um", C.c_double), ("parent", C.c_int32),
                ("center_um", C.c_double * 3)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Species), C.c_uint32, C.POINTER(_Reaction), C.c_uint32,
                                 C.POINTER(_Compartment), C.c_uint32, C.c_double, C.c_double,
                                 C.c_uint64, C.c_int, C.c_char_p, C.c_size_t]
        L.orc_step.argtypes = [C.c_void_p, C.c_uint32]
        L.orc_counts.restype = C.c_size_t
        L.orc_counts.argtypes = [C.c_void_p, C.POINTER(C.c_uint64), C.c_size_t]
        L.orc_digest.restype = C.c_uint64
        L.orc_digest.argtypes = [C.c_void_p]
        L.orc_dump.restype = C.c_size_t
        L.orc_dump.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
        L.orc_n_agents.restype = C.c_size_t
        L.orc_n_agents.argtypes = [C.c_void_p]
        L.orc_step_index.restype = C.c_uint32
        L.orc_step_index.argtypes = [C.c_void_p]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_set_table.restype = C.c_int
        L.orc_set_table.argtypes = [C.c_void_p, C.POINTER(C.c_int16)]
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.orc_ncdf_table.argtypes = [C.POINTER(C.c_int16)]
        L.orc_gauss_step.restype = C.c_int64
        L.orc_gauss_step.argtypes = [C.c_int16, C.c_uint64]
        L.orc_threshold.restype = C.c_uint64
        L.orc_threshold.argtypes = [C.c_double]
        L.orc_mult.restype = C.c_uint64
        L.orc_mult.argtypes = [C.c_double, C.c_double, C.c_double]
        _lib = L
    return _lib


def _structs(model):
    sp = (_Species * len(model.species))()
    for i, s in enumerate(model.species):
        sp[i] = _Species(s.count, s.D, s.comp, s.p_cross, s.p_uni, s.uni_to, s.p_emit, s.emit)
    n_rx = len(model.reactions)
    rx = (_Reaction * max(1, n_rx))()
    for i, r in enumerate(model.reactions):
        rx[i] = _Reaction(r.a, r.b, r.kind, r.prod_a, r.prod_b, r.radius_nm, r.p_bind, r.p_release)
    cm = (_Compartment * len(model.compartments))()
    for i, c in enumerate(model.compartments):
        cm[i] = _Compartment(c.shape, c.size_um, c.parent, (C.c_double * 3)(*c.center_um))
    return sp, rx, cm


class OracleError(ValueError):
    pass


class OracleSim:
    """Serial simulator of one model; ids ascending, every phase a plain loop."""

    def __init__(self, model, seed: int, brute_force: bool = False, table=None):
        L = lib()
        sp, rx, cm = _structs(model)
        err = C.create_string_buffer(256)
        h = L.orc_create(sp, len(model.species), rx, len(model.reactions), cm,
                         len(model.compartments), model.dt_s, model.unit_nm, seed,
                         1 if brute_force else 0, err, 256)
        if not h:
            raise OracleError(err.value.decode())
        self._h = h
        if table is not None:  # a caller's Gaussian table (data, like the default one)
            self._table = np.ascontiguousarray(table, dtype=np.int16)
            assert self._table.shape == (65536,)
            if L.orc_set_table(h, self._table.ctypes.data_as(C.POINTER(C.c_int16))) != 0:
                L.orc_destroy(h)
                self._h = None
                raise OracleError("diffusion step exceeds the domain with this table")
        self.model = model
        self.n_species = len(model.species)
        self.n_comp = len(model.compartments)
        self.n_rx = len(model.reactions)

    def step(self, n: int = 1) -> None:
        lib().orc_step(self._h, n)

    @property
    def t(self) -> int:
        return lib().orc_step_index(self._h)

    @property
    def n_agents(self) -> int:
        return lib().orc_n_agents(self._h)

    def counts(self) -> np.ndarray:
        need = self.n_species * self.n_comp + self.n_rx + 1
        out = (C.c_uint64 * need)()
        lib().orc_counts(self._h, out, need)
        return np.frombuffer(out, dtype=np.uint64).copy()

    def digest(self) -> int:
        return lib().orc_digest(self._h)

    def dump(self) -> np.ndarray:
        n = self.n_agents
        out = np.zeros(n, dtype=RECORD_DTYPE)
        lib().orc_dump(self._h, out.ctypes.data, n)
        return out

    def close(self) -> None:
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return list(o)


def ncdf_table() -> np.ndarray:
    out = np.zeros(65536, dtype=np.int16)
    lib().orc_ncdf_table(out.ctypes.data_as(C.POINTER(C.c_int16)))
    return out


def gauss_step(z: int, m: int) -> int:
    return lib().orc_gauss_step(z, m)


def threshold(p: float) -> int:
    return lib().orc_threshold(p)


def mult(D: float, dt: float, unit_nm: float) -> int:
    return lib().orc_mult(D, dt, unit_nm)
