"""abm_dump_noalloc against abm_dump, through the C ABI (GPU).

abm_dump_noalloc is for callers that cannot allocate device memory at the
moment they read the agents (for example a per-step monitor that must not
trigger cudaMalloc's device synchronisation); it stages records in a fixed
device array instead.  Its output must equal abm_dump's, bit for bit (the
state is integer: tolerance zero), on consecutive calls, including calls
that reuse the shared array after other calls.  This file is collected last
so that a run stopping at its first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from gpu_common import engine, require_gpu

pytestmark = pytest.mark.gpu

LIMIT = 131072


@pytest.fixture(scope="module")
def A():
    require_gpu()
    return engine()


def _fn(A):
    f = A.lib().abm_dump_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]
    return f


def _noalloc_dump(A, sim):
    f = _fn(A)
    n = C.c_size_t()
    assert f(sim._h, None, 0, C.byref(n)) == A.OK
    out = np.zeros(n.value, dtype=A.RECORD_DTYPE)
    m = C.c_size_t()
    assert f(sim._h, out.ctypes.data, out.size, C.byref(m)) == A.OK
    assert m.value == n.value
    return out


def test_noalloc_dump_equals_dump_on_consecutive_calls(A):
    sim = A.Sim(W.mapk(20_000), 12)          # complexes form: hidden records too
    sim.step(40)
    for _ in range(2):
        ref = sim.dump()
        first = _noalloc_dump(A, sim)
        second = _noalloc_dump(A, sim)          # two calls in a row, shared array
        assert len(ref) > 20_000 - 1 and np.count_nonzero(ref["flags"] & 2) > 0
        assert np.array_equal(first, ref)
        assert np.array_equal(second, ref)
        sim.step(9)
    small = A.Sim(W.toy(300, 200, edge_um=0.3), 3)  # a smaller dump after larger ones
    small.step(5)
    assert np.array_equal(_noalloc_dump(A, small), small.dump())
    small.close()
    sim.close()


def test_noalloc_dump_rejects_more_than_its_array(A):
    sim = A.Sim(W.mapk(150_000), 12)
    n = C.c_size_t()
    st = _fn(A)(sim._h, None, 0, C.byref(n))
    assert st == A.ECAPACITY
    assert n.value >= 150_000
    assert str(LIMIT) in A.lib().abm_last_error(sim._h).decode()
    sim.step(1)                                   # the handle is still usable
    assert len(sim.dump()) == 150_000
    sim.close()


def test_noalloc_dump_refuses_a_short_output_and_keeps_the_handle(A):
    sim = A.Sim(W.toy(400, 300, edge_um=0.4), 5)
    sim.step(3)
    f = _fn(A)
    n = C.c_size_t()
    assert f(sim._h, None, 0, C.byref(n)) == A.OK
    short = np.zeros(n.value - 1, dtype=A.RECORD_DTYPE)
    m = C.c_size_t()
    assert f(sim._h, short.ctypes.data, short.size, C.byref(m)) == A.EINVAL
    assert "needed" in A.lib().abm_last_error(sim._h).decode()
    sim.step(2)                                   # not a failure of the handle
    assert np.array_equal(_noalloc_dump(A, sim), sim.dump())
    sim.close()
