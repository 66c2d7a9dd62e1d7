"""Volume invariance of the dose readout (the paper's criterion: the final
relative change of pERK + ppERK agrees within about one percentage point
between a volume and ten times that volume, at every dose), at 200k vs 2M
agents per dose."""
import pytest

import workloads as W
from gpu_common import engine, require_gpu

pytestmark = pytest.mark.gpu


def test_readout_volume_invariant():
    require_gpu()
    A = engine()
    from paper_2606_14603_b300.experiments import volume_invariance
    r = volume_invariance(lambda n, d: W.mapk(n, d), [0.0, 0.05, 0.10], 200_000, factor=10,
                          steps=2000, period=100)
    assert r["agents"][1] == pytest.approx(10 * r["agents"][0], rel=1e-6)
    for small, large in zip(*r["change_pct"]):
        assert small < 0 and large < 0          # the readout falls over the run at every dose
    assert r["max_diff_pp"] <= 1.0, r
