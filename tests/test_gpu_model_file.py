"""A model file on the engine against the oracle (GPU, bit-exact).

Sec. 2: a model can be given as a JSON file instead of through the GUI, and
is checked for consistency before it runs.  The file here describes a cell
with a nucleus (Sec. 3.4): species with molecular weights (diffusion from
Stokes-Einstein), concentrations, localisations, translocation, degradation
and expression (a gene expressor that makes mRNA, which makes protein), and
bind / convert reactions with turnover numbers.  model_json.load turns it
into the engine's inputs; the engine and the oracle run the loaded model
from the same seed.  Digests are compared after every step, counts every
10 steps and the full id-sorted dumps at the end."""
import os

import numpy as np
import pytest

from gpu_common import assert_same_dump, engine, require_gpu
from paper_2606_14603_b300 import model_json as MJ

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
MODEL = os.path.join(HERE, "golden", "nucleus_expressor.json")


def test_loaded_model_file_equals_the_oracle(oracle_mod):
    require_gpu()
    A = engine()
    m = MJ.load(MODEL)
    assert len(m.compartments) == 2 and any(s.p_emit > 0 for s in m.species)
    seed, steps = 77, 300
    sim = A.Sim(m, seed)
    o = oracle_mod.OracleSim(m, seed)
    for t in range(1, steps + 1):
        sim.step(1)
        o.step(1)
        assert sim.digest() == o.digest(), f"step {t}"
        if t % 10 == 0:
            assert np.array_equal(sim.counts(), o.counts()), f"step {t}"
    c = o.counts()
    n_sp, n_c = len(m.species), len(m.compartments)
    names = [s.name for s in m.species]
    assert c[-1] > m.n_agents + 1000                                  # births happened
    assert c[names.index("mRNA") * n_c + 0] > 0                       # mRNA left the nucleus
    assert c[names.index("ppERK") * n_c + 1] > 0                      # ppERK entered it
    assert c[n_sp * n_c: -1].sum() > 0                                # complexes formed
    assert_same_dump(sim.dump(), o.dump(), f"after {steps} steps")
    o.close()
    sim.close()
