"""Shared helpers of the GPU tests (engine vs oracle comparisons)."""
import numpy as np
import pytest


def require_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def engine():
    from paper_2606_14603_b300 import build
    build.build()
    import paper_2606_14603_b300 as A
    A.lib()
    return A


FIELDS = ["id", "sp", "comp", "flags", "rxn", "x", "y", "z", "partner"]


def assert_same_dump(gpu_dump, orc_dump, where=""):
    """Element-by-element equality of two id-sorted dumps (bit-exact)."""
    assert len(gpu_dump) == len(orc_dump), f"{where}: {len(gpu_dump)} vs {len(orc_dump)} agents"
    for f in FIELDS:
        a = np.asarray(gpu_dump[f])
        b = np.asarray(orc_dump[f])
        bad = np.nonzero(a != b)[0]
        if len(bad):
            i = bad[0]
            raise AssertionError(f"{where}: field {f} differs at {len(bad)} agents; first id "
                                 f"{orc_dump['id'][i]}: gpu {gpu_dump[i]} oracle {orc_dump[i]}")
