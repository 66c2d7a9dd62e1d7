"""The C ABI without a GPU: the library loads, exports every declared entry
point, validates models before touching the device, and its host-side
building blocks agree with independent computations."""
import re
import os

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def A():
    import paper_2606_14603_b300 as A
    from paper_2606_14603_b300 import build
    build.build()
    A.lib()
    return A


def declared_functions():
    src = open(os.path.join(ROOT, "include", "abm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(abm_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(A):
    import ctypes
    lib = ctypes.CDLL(A.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n


def test_read_slots_match_the_header(A):
    src = open(os.path.join(ROOT, "include", "abm.h")).read()
    assert int(re.search(r"#define ABM_READ_SLOTS (\d+)", src).group(1)) == A.READ_SLOTS


def test_version(A):
    assert b"sm_103a" in A.lib().abm_version()


def test_builtin_table_equals_oracle_table(A, oracle_mod):
    assert np.array_equal(A.ncdf_table(), oracle_mod.ncdf_table())


def _bad(kind):
    m = W.toy()
    if kind == "aa":
        m.reactions = [W.Reaction(0, 0, W.CONVERT, 2, 2, 5.0, 1.0)]
    elif kind == "dup":
        m.reactions = m.reactions * 2
    elif kind == "rev":
        m.reactions = m.reactions + [W.Reaction(1, 0, W.CONVERT, 2, 2, 5.0, 1.0)]
    elif kind == "prob":
        m.reactions[0].p_bind = 1.5
    elif kind == "prob_neg":
        m.species[0].p_uni = -0.1
    elif kind == "radius":
        m.reactions[0].radius_nm = 0.0
    elif kind == "product":
        m.reactions[0].prod_a = 7
    elif kind == "emit":
        m.species[0].emit = 9
    elif kind == "comp":
        m.species[0].comp = 3
    elif kind == "child_out":
        m.compartments = [W.Compartment(W.CUBE, 1.0), W.Compartment(W.SPHERE, 2.0, parent=0)]
    elif kind == "child_overlap":
        m.compartments = [W.Compartment(W.SPHERE, 4.0), W.Compartment(W.SPHERE, 1.0, parent=0),
                          W.Compartment(W.SPHERE, 1.0, parent=0, center_um=(0.5, 0, 0))]
    elif kind == "dt":
        m.dt_s = 0.0
    elif kind == "huge_step":
        m.dt_s = 10.0
    elif kind == "no_species":
        m.species = []
    elif kind == "extent":  # 2,100,000 units of 0.1 nm: positions need 21 bits at most
        m.compartments = [W.Compartment(W.CUBE, 210.0)]
    return m


@pytest.mark.parametrize("kind", ["aa", "dup", "rev", "prob", "prob_neg", "radius", "product", "emit",
                                  "comp", "child_out", "child_overlap", "dt", "huge_step", "extent"])
def test_invalid_model_is_einval_without_device(A, kind):
    with pytest.raises(A.AbmError) as e:
        A.Sim(_bad(kind), 1)
    assert e.value.status == A.EINVAL
    assert A.arena_bytes(_bad(kind)) == 0


def test_largest_extent_is_accepted(A):
    """The root edge may reach 2^21 - 1 position units (209.7 um at 0.1 nm)."""
    m = W.toy()
    m.compartments = [W.Compartment(W.CUBE, 209.7)]
    assert A.arena_bytes(m) > 0


def test_cell_smaller_than_radius_is_einval(A):
    with pytest.raises(A.AbmError) as e:
        A.Sim(W.toy(), 1, cell_log2=5)            # 32 units < R = 50 units
    assert e.value.status == A.EINVAL


def test_arena_bytes_scales(A):
    a = A.arena_bytes(W.mapk(100_000))
    b = A.arena_bytes(W.mapk(1_000_000))
    assert a > 0 and b > 5 * a
    # about 80-90 bytes per agent slot plus the cell grid
    assert b < 200 * 1_300_000 + 16 * 1_000_000


def test_batch_arena_bytes_rejects_bad_options(A):
    assert A.Batch.arena_bytes(0, 10, 1) == 0
    assert A.Batch.arena_bytes(10, 10, 0) == 0
    assert A.Batch.arena_bytes(10, 10, 5000) == 0
    assert A.Batch.arena_bytes(1000, 1000, 4) > 0


def test_no_device_is_reported(A):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(A.AbmError) as e:
        A.Sim(W.toy(), 1)
    assert e.value.status == A.EDEVICE
