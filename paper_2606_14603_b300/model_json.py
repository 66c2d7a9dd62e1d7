"""Model files (JSON) and their consistency checks.

The paper defines a model by its species and reactions (Sec. 2): for each
species a molecular weight, an initial concentration, a localisation and a
functional class (active, inactive, expressor; inhibited species emerge and
are not declared), and for each interaction the partners, the turnover number
and the products; compartment volumes and translocation rates when
compartments are modelled, expression rates when genes are.  It also names a
consistency check run before a simulation: reciprocal interaction
definitions, referenced molecules that exist, plausible molecular weights,
and volumes compatible with the concentrations.

This module reads such a description and turns the physical quantities into
the engine's parameters:
  radius      sphere of the protein's mass at protein density 1.35 g/cm^3
  D           Stokes-Einstein, k_B T / (6 pi eta r)
  contact     sum of the two radii (unless given)
  per step    p = 1 - exp(-rate * dt) for turnover (release), degradation and
              expression rates
  counts      round(concentration * compartment volume * N_A)

Schema (keys in brackets are optional):
{
  "name": str, "dt_s": float, ["unit_nm": 0.1], ["temperature_k": 310.15],
  ["viscosity_pa_s": 0.0032],
  "cell":    {"shape": "cube", "volume_l": float} | {"shape": "sphere", "diameter_um": float},
  ["nucleus": {"diameter_um": float}],
  "species": [{"name", "class": "active"|"inactive"|"expressor"|"product",
               "mw_kda", "concentration_m", ["localisation": "cytosol"|"nucleus"],
               ["partners": [names]], ["translocation_p": float],
               ["degradation_per_s": float], ["converts_to": name],
               ["expression": {"product": name, "rate_per_s": float}],
               ["diffusion_um2_s": float (overrides Stokes-Einstein)]}],
  "reactions": [{"a": name, "b": name, "kind": "bind"|"convert",
                 "products": [name|null, name|null], ["kcat_per_s": float],
                 ["p_bind": 1.0], ["radius_nm": float]}]
}
"""
from __future__ import annotations

import dataclasses
import json
import math
from typing import List, Tuple

AVOGADRO = 6.02214076e23
BOLTZMANN = 1.380649e-23
PROTEIN_DENSITY_G_CM3 = 1.35

CLASSES = ("active", "inactive", "expressor", "product", "inhibited")


@dataclasses.dataclass
class Issue:
    level: str          # "error" or "warning"
    where: str
    message: str

    def __str__(self):
        return f"{self.level}: {self.where}: {self.message}"


class ModelError(ValueError):
    def __init__(self, issues: List[Issue]):
        super().__init__("; ".join(str(i) for i in issues if i.level == "error"))
        self.issues = issues


def radius_nm(mw_kda: float) -> float:
    """Radius (nm) of a sphere of mass mw_kda kDa at protein density."""
    grams = mw_kda * 1000.0 / AVOGADRO
    volume_cm3 = grams / PROTEIN_DENSITY_G_CM3
    r_cm = (3.0 * volume_cm3 / (4.0 * math.pi)) ** (1.0 / 3.0)
    return r_cm * 1e7


def stokes_einstein_um2_s(r_nm: float, temperature_k: float, viscosity_pa_s: float) -> float:
    """Diffusion coefficient (um^2/s) of a sphere of radius r_nm."""
    d_m2_s = BOLTZMANN * temperature_k / (6.0 * math.pi * viscosity_pa_s * r_nm * 1e-9)
    return d_m2_s * 1e12


def per_step(rate_per_s: float, dt_s: float) -> float:
    """Probability that a first-order event of this rate happens in dt."""
    return 1.0 - math.exp(-rate_per_s * dt_s)


def _volumes_l(doc) -> Tuple[float, float]:
    """(cell volume, nucleus volume) in litres."""
    cell = doc["cell"]
    if cell.get("shape") == "cube":
        v_cell = float(cell["volume_l"])
    else:
        d_um = float(cell["diameter_um"])
        v_cell = math.pi / 6.0 * d_um ** 3 * 1e-15
    v_nuc = 0.0
    if "nucleus" in doc:
        v_nuc = math.pi / 6.0 * float(doc["nucleus"]["diameter_um"]) ** 3 * 1e-15
    return v_cell, v_nuc


def check(doc) -> List[Issue]:
    """Consistency checks of a model description; returns every issue found."""
    issues: List[Issue] = []

    def err(where, msg):
        issues.append(Issue("error", where, msg))

    def warn(where, msg):
        issues.append(Issue("warning", where, msg))

    species = doc.get("species", [])
    names = [s.get("name") for s in species]
    known = set(names)
    for n in set(names):
        if names.count(n) > 1:
            err(f"species {n}", "defined more than once")
    if not isinstance(doc.get("dt_s"), (int, float)) or doc["dt_s"] <= 0:
        err("model", "dt_s must be a positive number")
    if "cell" not in doc:
        err("model", "no cell geometry")
        return issues
    v_cell, v_nuc = _volumes_l(doc)
    if v_cell <= 0:
        err("cell", "volume must be positive")
    if v_nuc >= v_cell:
        err("nucleus", "nucleus is not smaller than the cell")
    for s in species:
        w = f"species {s.get('name')}"
        cls = s.get("class")
        if cls not in CLASSES:
            err(w, f"unknown class {cls!r}")
        if cls == "inhibited" and s.get("concentration_m", 0) > 0:
            warn(w, "inhibited molecules emerge by binding an inhibitor and need no initial amount")
        mw = s.get("mw_kda")
        if not isinstance(mw, (int, float)) or mw <= 0:
            err(w, "molecular weight missing or not positive")
        elif not 0.1 <= mw <= 5000.0:
            warn(w, f"molecular weight {mw} kDa is implausible for a molecule of a signalling pathway")
        c = s.get("concentration_m", 0.0)
        if c < 0:
            err(w, "negative concentration")
        loc = s.get("localisation", "cytosol")
        if loc not in ("cytosol", "nucleus"):
            err(w, f"unknown localisation {loc!r}")
        elif loc == "nucleus" and "nucleus" not in doc:
            err(w, "localised in a nucleus the model does not define")
        vol = v_nuc if loc == "nucleus" else v_cell - v_nuc
        n = c * vol * AVOGADRO
        if 0 < n < 0.5:
            err(w, f"{c:g} M in {vol:g} L is {n:.3g} molecules: rounds to none (enlarge the volume)")
        elif 0.5 <= n < 10:
            warn(w, f"only {round(n)} molecules at this volume: results will be noisy")
        if n > 2 ** 31:
            err(w, f"{n:.3g} molecules exceed the engine's agent capacity")
        for ref_key in ("converts_to",):
            if s.get(ref_key) is not None and s[ref_key] not in known:
                err(w, f"{ref_key} names unknown species {s[ref_key]!r}")
        e = s.get("expression")
        if cls == "expressor" and not e:
            err(w, "an expressor needs an expression block")
        if e:
            if e.get("product") not in known:
                err(w, f"expression product {e.get('product')!r} is not a defined species")
            if e.get("rate_per_s", 0) < 0:
                err(w, "negative expression rate")
        for p in s.get("partners", []):
            if p not in known:
                err(w, f"partner {p!r} is not a defined species")
    # reciprocal partner lists
    by_name = {s.get("name"): s for s in species}
    for s in species:
        for p in s.get("partners", []):
            if p in by_name and "partners" in by_name[p] and s["name"] not in by_name[p]["partners"]:
                err(f"species {s['name']}", f"lists {p} as a partner but {p} does not list it back")
    pairs = set()
    for k, r in enumerate(doc.get("reactions", [])):
        w = f"reaction {k} ({r.get('a')}+{r.get('b')})"
        a, b = r.get("a"), r.get("b")
        for nm in (a, b):
            if nm not in known:
                err(w, f"reactant {nm!r} is not a defined species")
        if a == b:
            err(w, "a species reacting with itself is not supported")
        key = frozenset((a, b))
        if key in pairs:
            err(w, "a second reaction for the same pair of species")
        pairs.add(key)
        if r.get("kind") not in ("bind", "convert"):
            err(w, f"unknown kind {r.get('kind')!r}")
        prods = r.get("products", [])
        if len(prods) != 2:
            err(w, "products must list two entries (null for a molecule that is consumed)")
        for p in prods:
            if p is not None and p not in known:
                err(w, f"product {p!r} is not a defined species")
        if r.get("kind") == "bind" and r.get("kcat_per_s") is None:
            err(w, "a bind reaction needs its turnover number kcat_per_s")
        if not 0.0 <= r.get("p_bind", 1.0) <= 1.0:
            err(w, "p_bind outside [0, 1]")
        for nm, other in ((a, b), (b, a)):
            s = by_name.get(nm)
            if s is not None and "partners" in s and other not in s["partners"]:
                err(w, f"{nm} does not list {other} as a partner")
    return issues


def load(doc_or_path):
    """A workloads.Model for the engine and the oracle; raises ModelError
    when the consistency check finds an error."""
    import workloads as W  # the neutral model description shared by both sides
    doc = doc_or_path
    if isinstance(doc_or_path, str):
        with open(doc_or_path) as f:
            doc = json.load(f)
    issues = check(doc)
    if any(i.level == "error" for i in issues):
        raise ModelError(issues)
    dt = float(doc["dt_s"])
    temp = float(doc.get("temperature_k", 310.15))
    eta = float(doc.get("viscosity_pa_s", 0.0032))
    v_cell, v_nuc = _volumes_l(doc)
    species = doc["species"]
    index = {s["name"]: i for i, s in enumerate(species)}
    radii = [radius_nm(s["mw_kda"]) for s in species]
    out_sp = []
    for s, r in zip(species, radii):
        loc = s.get("localisation", "cytosol")
        vol = v_nuc if loc == "nucleus" else v_cell - v_nuc
        count = int(round(s.get("concentration_m", 0.0) * vol * AVOGADRO))
        D = s.get("diffusion_um2_s")
        if D is None:
            D = 0.0 if s["class"] == "expressor" else stokes_einstein_um2_s(r, temp, eta)
        e = s.get("expression") or {}
        deg = s.get("degradation_per_s", 0.0)
        out_sp.append(W.Species(
            s["name"], count, float(D), comp=1 if loc == "nucleus" else 0,
            p_cross=float(s.get("translocation_p", 0.0)),
            p_uni=per_step(deg, dt) if deg else 0.0,
            uni_to=index[s["converts_to"]] if s.get("converts_to") else -1,
            p_emit=per_step(e.get("rate_per_s", 0.0), dt) if e else 0.0,
            emit=index[e["product"]] if e else -1))
    out_rx = []
    for r in doc.get("reactions", []):
        a, b = index[r["a"]], index[r["b"]]
        pa, pb = r["products"]
        radius = r.get("radius_nm") or radii[a] + radii[b]
        kind = W.BIND if r["kind"] == "bind" else W.CONVERT
        out_rx.append(W.Reaction(a, b, kind, index[pa] if pa is not None else -1,
                                 index[pb] if pb is not None else -1, float(radius),
                                 float(r.get("p_bind", 1.0)),
                                 per_step(r["kcat_per_s"], dt) if kind == W.BIND else 0.0))
    cell = doc["cell"]
    if cell.get("shape") == "cube":
        comps = [W.Compartment(W.CUBE, (v_cell * 1e15) ** (1.0 / 3.0))]
    else:
        comps = [W.Compartment(W.SPHERE, float(cell["diameter_um"]))]
    if "nucleus" in doc:
        comps.append(W.Compartment(W.SPHERE, float(doc["nucleus"]["diameter_um"]), parent=0))
    return W.Model(doc.get("name", "model"), out_sp, out_rx, comps, dt_s=dt,
                   unit_nm=float(doc.get("unit_nm", 0.1)))
