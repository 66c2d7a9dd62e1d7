"""Autotuner knobs do not change results (GPU): every (cell size, CTAs per
SM, block size, proposal chunk, concurrent batches) candidate yields
identical digests, equal to the oracle's; the tuner returns its fastest
candidate, over a product of axes or axis by axis."""
import pytest

import workloads as W
from gpu_common import engine, require_gpu

pytestmark = pytest.mark.gpu


def test_tuner_candidates_agree_and_match_oracle(oracle_mod):
    require_gpu()
    engine()
    from paper_2606_14603_b300 import autotune
    sims = [(W.mapk(9_000, drug_frac=0.03), 21), (W.nuclear(8_000, boost=50.0, n_genes=8, genes_on=4), 22),
            (W.toy(700, 600, edge_um=0.45), 23)]
    ref = []
    for m, s in sims:
        o = oracle_mod.OracleSim(m, s)
        o.step(25)
        ref.append(o.digest())
    for d, bps, tb, ch in [(0, 0, 0, 0), (1, 4, 0, 0), (-1, 32, 0, 0), (2, 8, 0, 0), (0, 0, 128, 1024),
                           (0, 0, 512, 4096), (1, 1, 512, 2048), (0, 16, 128, 4096)]:
        b, ids = autotune.batch_for(sims, d, bps, threads_per_block=tb, propose_chunk=ch)
        b.step(25)
        assert [b.digest(i) for i in ids] == ref, (d, bps, tb, ch)
        b.close()
    for ng in (2, 3):   # simulations split over concurrent batches on their own streams
        grp = autotune.BatchGroup(sims, 0, 0, ng)
        grp.step(25)
        grp.sync()
        assert [grp.digest(k) for k in range(len(sims))] == ref, ng
        grp.close()
    best, allc = autotune.tune(sims, cell_deltas=(0, 1), blocks=(8, 16), groups=(1, 2), steps=5, warmup=1)
    assert len(allc) == 8 and best.ms_per_step == min(c.ms_per_step for c in allc)
    best, allc = autotune.tune(sims, cell_deltas=(0, 1), blocks=(0,), groups=(1, 2), threads=(256, 128, 512),
                               chunks=(0, 1024, 4096), steps=5, warmup=1, search="axes")
    assert len(allc) == 2 + 1 + 2 + 2 and best.ms_per_step == min(c.ms_per_step for c in allc)
    with pytest.raises(A_error()):
        autotune.batch_for(sims, 0, 0, threads_per_block=300)


def A_error():
    import paper_2606_14603_b300 as A
    return A.AbmError
