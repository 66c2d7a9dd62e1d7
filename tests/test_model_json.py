"""Model files: conversion of physical inputs and the consistency checks."""
import copy
import json
import math
import os

import pytest

from paper_2606_14603_b300 import model_json as MJ

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE1 = os.path.join(HERE, "golden", "table1_mapk.json")


def _doc():
    with open(TABLE1) as f:
        return json.load(f)


def test_table1_counts_at_point_three_picolitres():
    """Agent counts at the paper's multi-seed volume (3e-13 L, Sec. 3.2) from
    the Table 1 concentrations: round(c V N_A)."""
    m = MJ.load(TABLE1)
    counts = {s.name: s.count for s in m.species}
    assert counts["BRAF"] == 542                 # 3 nM: the low-abundance species of Sec. 3.3
    assert counts["MEK"] == 216_797
    assert counts["pERK"] == 14_467
    assert counts["ppERK"] == 202_073
    assert counts["phosphatase 1"] == 54
    assert counts["phosphatase 2"] == 21_680
    assert counts["dabrafenib"] == 347_706         # 1000 ng/mL = 1.9246e-6 M (Sec. 3.1)
    assert counts["ERK"] == counts["pMEK"] == counts["ppMEK"] == 0


def test_cube_edges_match_the_papers_volumes():
    """Sec. 3.2: 3e-12 L is about a 14.4 um cube, 3e-13 L about 6.7 um."""
    for vol, edge in ((3e-12, 14.4), (3e-13, 6.7)):
        d = _doc()
        d["cell"]["volume_l"] = vol
        m = MJ.load(d)
        assert abs(m.compartments[0].size_um - edge) < 0.05


def test_stokes_einstein_and_radius_scaling():
    r1, r8 = MJ.radius_nm(10.0), MJ.radius_nm(80.0)
    assert abs(r8 / r1 - 2.0) < 1e-12                      # r ~ M^(1/3)
    # 100 kDa at 1.35 g/cm3: r = (3 * 1e5 / (4 pi 1.35 N_A))^(1/3) cm = 3.085 nm
    assert abs(MJ.radius_nm(100.0) - 3.0851) < 1e-3
    d1 = MJ.stokes_einstein_um2_s(3.0, 298.15, 0.00089)
    assert abs(d1 - 81.8) < 0.2                              # k_B T / (6 pi eta r)
    assert abs(MJ.stokes_einstein_um2_s(6.0, 298.15, 0.00089) * 2 - d1) < 1e-9
    assert abs(MJ.per_step(50.0, 1e-6) - (1 - math.exp(-5e-5))) < 1e-15


def test_loaded_model_runs_in_the_oracle(oracle_mod):
    d = _doc()
    d["cell"]["volume_l"] = 3e-15                           # small: 5 BRAF, ~3.5k agents in all
    d["species"][1]["concentration_m"] = 1e-7
    for s in d["species"]:
        if s["name"] == "phosphatase 1":
            s["concentration_m"] = 3e-9
    m = MJ.load(d)
    sim = oracle_mod.OracleSim(m, 5)
    sim.step(20)
    assert sim.n_agents == m.n_agents


@pytest.mark.parametrize("case,needle", [
    ("unknown_product", "product 'pppERK'"),
    ("unknown_partner", "partner 'RAS'"),
    ("non_reciprocal", "does not list it back"),
    ("duplicate_pair", "second reaction"),
    ("self_reaction", "itself"),
    ("zero_agents", "rounds to none"),
    ("nucleus_missing", "nucleus the model does not define"),
    ("no_kcat", "turnover number"),
    ("bad_mw", "molecular weight missing"),
    ("expressor_without_rate", "expression block"),
])
def test_consistency_errors(case, needle):
    d = _doc()
    if case == "unknown_product":
        d["reactions"][4]["products"][1] = "pppERK"
    elif case == "unknown_partner":
        d["species"][0]["partners"].append("RAS")
    elif case == "non_reciprocal":
        d["species"][5]["partners"].remove("BRAF")
    elif case == "duplicate_pair":
        d["reactions"].append(copy.deepcopy(d["reactions"][0]))
    elif case == "self_reaction":
        d["reactions"][0]["b"] = "BRAF"
    elif case == "zero_agents":
        d["cell"]["volume_l"] = 3e-16                        # 3 nM BRAF: 0.18 molecules
    elif case == "nucleus_missing":
        d["species"][0]["localisation"] = "nucleus"
    elif case == "no_kcat":
        del d["reactions"][0]["kcat_per_s"]
    elif case == "bad_mw":
        d["species"][2]["mw_kda"] = 0
    else:
        d["species"][2]["class"] = "expressor"
    issues = MJ.check(d)
    errors = [str(i) for i in issues if i.level == "error"]
    assert any(needle in e for e in errors), errors
    with pytest.raises(MJ.ModelError):
        MJ.load(d)


def test_warnings_do_not_block():
    d = _doc()
    d["species"][0]["mw_kda"] = 9000.0                      # implausible, warned
    issues = MJ.check(d)
    assert any(i.level == "warning" and "implausible" in i.message for i in issues)
    MJ.load(d)


def test_reference_model_is_consistent():
    assert [i for i in MJ.check(_doc()) if i.level == "error"] == []
