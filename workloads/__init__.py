"""Seeded synthetic workloads shared by the tests, the bench and the oracle.

This module only *describes* models (species, reactions, compartments, time
step, seeds) as plain dataclasses.  It holds none of the simulation's
arithmetic: no thresholds, no random draws, no positions.  Both the CUDA
engine's binding and the oracle's binding turn these descriptions into their
own C structs.

The paper's own parameter sets (its MAPK/ERK tables, the cFos network of its
Sec. 3.4, clinical data) are not available, so every model here is synthetic.
The proportions of the cascade follow the species list of the paper's Table 1
(BRAF, dabrafenib, the MEK and ERK phosphorylation states, phosphatases); the
reaction radii, probabilities and diffusion coefficients are chosen by us
within the ranges stated next to each builder.
"""
from __future__ import annotations

import dataclasses
import math
import random
from typing import List, Sequence, Tuple

CONVERT = 0
BIND = 1
CUBE = 0
SPHERE = 1


@dataclasses.dataclass
class Species:
    name: str
    count: int
    D: float                     # um^2/s
    comp: int = 0                # initial compartment
    p_cross: float = 0.0         # per attempted membrane crossing
    p_uni: float = 0.0           # first-order convert/death per step
    uni_to: int = -1             # -1 = death
    p_emit: float = 0.0          # expressor birth probability per step
    emit: int = -1               # child species, -1 = none


@dataclasses.dataclass
class Reaction:
    a: int                       # proposer species
    b: int                       # acceptor species
    kind: int                    # CONVERT or BIND
    prod_a: int                  # species of a afterwards (-1 dies)
    prod_b: int                  # species of b afterwards (-1 dies)
    radius_nm: float
    p_bind: float
    p_release: float = 0.0


@dataclasses.dataclass
class Compartment:
    shape: int                   # CUBE or SPHERE
    size_um: float               # edge (cube) or diameter (sphere)
    parent: int = -1
    center_um: Tuple[float, float, float] = (0.0, 0.0, 0.0)


@dataclasses.dataclass
class Model:
    name: str
    species: List[Species]
    reactions: List[Reaction]
    compartments: List[Compartment]
    dt_s: float = 1e-6
    unit_nm: float = 0.1

    @property
    def n_agents(self) -> int:
        return sum(s.count for s in self.species)

    def with_counts(self, counts: Sequence[int]) -> "Model":
        sp = [dataclasses.replace(s, count=int(c)) for s, c in zip(self.species, counts)]
        return dataclasses.replace(self, species=sp)


# --------------------------------------------------------------------------
# Workload 1: toy A + B -> C in a 1 um cube (2,500 A + 2,500 B, D = 1 um^2/s,
# contact radius 5 nm, bind probability 1, dt = 1 us, 200 steps, seed 1).
def toy(n_a: int = 2500, n_b: int = 2500, edge_um: float = 1.0, radius_nm: float = 5.0,
        D: float = 1.0, dt_s: float = 1e-6) -> Model:
    return Model(
        name="toy_A+B->C",
        species=[Species("A", n_a, D), Species("B", n_b, D), Species("C", 0, D)],
        reactions=[Reaction(0, 1, CONVERT, 2, -1, radius_nm, 1.0)],
        compartments=[Compartment(CUBE, edge_um)],
        dt_s=dt_s,
    )


TOY_SEED = 1
TOY_STEPS = 200

# --------------------------------------------------------------------------
# Workload 2: MAPK-like cascade in one cubic compartment.  Composition at
# 1,000,000 agents (drug fraction 10% at the top dose): BRAF* 2%, drug 0-10%,
# MEK 20%, ERK 40%, ppERK 20%, phosphatase 8%; pMEK, ppMEK, pERK start at 0.
# 12 reactions: enzyme-substrate complexes formed by BIND and released as
# products (radii 2-8 nm, bind probability 0.01-1, release 0.001-0.1 per step).
MAPK_SPECIES = ["BRAF*", "D", "MEK", "pMEK", "ppMEK", "ERK", "pERK", "ppERK", "PPase"]
_BRAF, _D, _MEK, _PMEK, _PPMEK, _ERK, _PERK, _PPERK, _PPASE = range(9)
MAPK_D = [1.0, 10.0, 3.0, 3.0, 3.0, 4.0, 4.0, 4.0, 2.0]


def mapk_reactions() -> List[Reaction]:
    return [
        Reaction(_BRAF, _MEK, BIND, _BRAF, _PMEK, 5.0, 0.5, 0.05),
        Reaction(_BRAF, _PMEK, BIND, _BRAF, _PPMEK, 5.0, 0.5, 0.05),
        Reaction(_PPMEK, _ERK, BIND, _PPMEK, _PERK, 4.0, 0.3, 0.05),
        Reaction(_PPMEK, _PERK, BIND, _PPMEK, _PPERK, 4.0, 0.3, 0.05),
        Reaction(_PMEK, _ERK, BIND, _PMEK, _PERK, 4.0, 0.01, 0.02),
        Reaction(_PMEK, _PERK, BIND, _PMEK, _PPERK, 4.0, 0.01, 0.02),
        Reaction(_PPASE, _PPERK, BIND, _PPASE, _PERK, 6.0, 0.2, 0.1),
        Reaction(_PPASE, _PERK, BIND, _PPASE, _ERK, 6.0, 0.2, 0.1),
        Reaction(_PPASE, _PPMEK, BIND, _PPASE, _PMEK, 6.0, 0.1, 0.1),
        Reaction(_PPASE, _PMEK, BIND, _PPASE, _MEK, 6.0, 0.1, 0.1),
        Reaction(_BRAF, _D, BIND, _BRAF, _D, 8.0, 1.0, 0.001),      # inhibition by the drug
        Reaction(_PPERK, _BRAF, BIND, _PPERK, _BRAF, 2.0, 0.05, 0.01),  # feedback sequestration
    ]


def mapk(n_total: int = 1_000_000, drug_frac: float = 0.10, edge_um: float | None = None,
         dt_s: float = 1e-6) -> Model:
    """The cascade at n_total agents (before the drug) at the density of
    1,000,000 agents per (10 um)^3, plus round(drug_frac * n_total) drug agents
    within that total (drug_frac = 0.1 is the top dose)."""
    n_d = int(round(drug_frac * n_total))
    base = n_total - n_d
    frac = {_BRAF: 0.02, _MEK: 0.20, _ERK: 0.40, _PPERK: 0.20, _PPASE: 0.08}
    scale = base / 0.90
    counts = [0] * 9
    for k, f in frac.items():
        counts[k] = int(round(f * scale))
    counts[_ERK] += base - sum(counts)          # rounding remainder to ERK
    counts[_D] = n_d
    if edge_um is None:
        edge_um = 10.0 * (n_total / 1_000_000) ** (1.0 / 3.0)
    species = [Species(name, counts[i], MAPK_D[i]) for i, name in enumerate(MAPK_SPECIES)]
    return Model(name="mapk", species=species, reactions=mapk_reactions(),
                 compartments=[Compartment(CUBE, edge_um)], dt_s=dt_s)


MAPK_SEED = 12
MAPK_STEPS = 10_000

# --------------------------------------------------------------------------
# Workload 3: two compartments.  A 12 um spherical cell with a concentric
# 5 um nucleus (diameters), 4,000,000 agents.  ERK/ppERK (and phosphatase)
# cross the nuclear membrane with probability 1e-3 per attempt; 64 immobile
# gene sites are activated by pElk1 and emit mRNA; mRNA emits cFos; ppERK
# phosphorylates cFos; pcFos emits the repressor F, which binds active genes
# (hidden inside the gene while bound, blocking emission); mRNA, cFos, pcFos
# and F degrade.
NUC_SPECIES = ["ppMEK", "ERK", "ppERK", "PPase", "Elk1", "pElk1", "GENE_off", "GENE_on",
               "mRNA", "cFos", "pcFos", "F"]
(_N_PPMEK, _N_ERK, _N_PPERK, _N_PPASE, _N_ELK, _N_PELK, _N_GOFF, _N_GON, _N_MRNA, _N_CFOS,
 _N_PCFOS, _N_F) = range(12)


def nuclear(n_total: int = 4_000_000, cell_um: float | None = None, boost: float = 1.0,
            n_genes: int = 64, genes_on: int = 0, dt_s: float = 1e-6) -> Model:
    """The two-compartment network.  `boost` multiplies the first-order,
    emission and membrane-crossing probabilities (capped at 1) so that small
    parity cases see many events; boost = 1 is the nominal model.  `genes_on`
    of the gene sites start active (the nominal model starts with all off)."""
    if cell_um is None:
        cell_um = 12.0 * (n_total / 4_000_000) ** (1.0 / 3.0)
    nuc_um = cell_um * 5.0 / 12.0
    scale = n_total / 4_000_000
    b = lambda p: min(1.0, p * boost)
    counts = {
        _N_PPMEK: int(round(400_000 * scale)),
        _N_ERK: int(round(1_600_000 * scale)),
        _N_PPERK: int(round(400_000 * scale)),
        _N_PPASE: int(round(1_400_000 * scale)),
        _N_GOFF: n_genes - genes_on,
        _N_GON: genes_on,
    }
    counts[_N_ELK] = n_total - sum(counts.values())
    sp = [
        Species("ppMEK", counts[_N_PPMEK], 3.0, 0),
        Species("ERK", counts[_N_ERK], 4.0, 0, p_cross=b(1e-3)),
        Species("ppERK", counts[_N_PPERK], 4.0, 0, p_cross=b(1e-3)),
        Species("PPase", counts[_N_PPASE], 2.0, 0, p_cross=b(1e-3)),
        Species("Elk1", counts[_N_ELK], 3.0, 1),
        Species("pElk1", 0, 3.0, 1),
        Species("GENE_off", counts[_N_GOFF], 0.0, 1),
        Species("GENE_on", counts[_N_GON], 0.0, 1, p_uni=b(1e-4), uni_to=_N_GOFF, p_emit=b(1e-2), emit=_N_MRNA),
        Species("mRNA", 0, 1.0, 1, p_cross=b(1e-2), p_uni=b(1e-4), uni_to=-1, p_emit=b(1e-3), emit=_N_CFOS),
        Species("cFos", 0, 3.0, 1, p_cross=b(1e-3), p_uni=b(2e-5), uni_to=-1),
        Species("pcFos", 0, 3.0, 1, p_cross=b(1e-3), p_uni=b(5e-6), uni_to=-1, p_emit=b(1e-4), emit=_N_F),
        Species("F", 0, 2.0, 1, p_cross=b(1e-3), p_uni=b(1e-5), uni_to=-1),
    ]
    rx = [
        Reaction(_N_PPMEK, _N_ERK, BIND, _N_PPMEK, _N_PPERK, 4.0, 0.3, 0.05),
        Reaction(_N_PPASE, _N_PPERK, BIND, _N_PPASE, _N_ERK, 6.0, 0.2, 0.1),
        Reaction(_N_PPERK, _N_ELK, BIND, _N_PPERK, _N_PELK, 5.0, 0.5, 0.05),
        Reaction(_N_PPASE, _N_PELK, BIND, _N_PPASE, _N_ELK, 6.0, 0.2, 0.1),
        Reaction(_N_PELK, _N_GOFF, CONVERT, _N_PELK, _N_GON, 8.0, 1.0),
        Reaction(_N_F, _N_GON, BIND, _N_F, _N_GON, 8.0, 1.0, 5e-4),
        Reaction(_N_PPERK, _N_CFOS, BIND, _N_PPERK, _N_PCFOS, 5.0, 0.5, 0.05),
        Reaction(_N_PPASE, _N_PCFOS, BIND, _N_PPASE, _N_CFOS, 6.0, 0.05, 0.1),
    ]
    comps = [Compartment(SPHERE, cell_um), Compartment(SPHERE, nuc_um, parent=0)]
    return Model(name="nuclear", species=sp, reactions=rx, compartments=comps, dt_s=dt_s)


NUCLEAR_SEED = 42
NUCLEAR_STEPS = 20_000

# --------------------------------------------------------------------------
# Workload 4: dose-response sweep, 8 doses (log-spaced 0.1-1000) x 8 seeds =
# 64 cascade sims of uneven sizes N_k = round(50,000 * 10^(k/63)), k = 0..63,
# assigned to (dose, seed) by a shuffle seeded with 2024; volume scales with N
# at the cascade's density; 5,000 steps each.
SWEEP_SEEDS = [12, 42, 314, 101010, 1, 2, 3, 4]
SWEEP_STEPS = 5_000


def sweep_doses() -> List[float]:
    return [0.1 * 10 ** (4.0 * j / 7.0) for j in range(8)]


def sweep(scale: float = 1.0) -> List[Tuple[Model, int]]:
    """[(model, seed)] for the 64 sims; `scale` shrinks every size (parity)."""
    sizes = [int(round(50_000 * 10 ** (k / 63.0) * scale)) for k in range(64)]
    rng = random.Random(2024)
    rng.shuffle(sizes)
    out = []
    for j, dose in enumerate(sweep_doses()):
        for i, seed in enumerate(SWEEP_SEEDS):
            n = sizes[j * 8 + i]
            out.append((mapk(n, drug_frac=0.1 * dose / 1000.0), seed))
    return out


# --------------------------------------------------------------------------
# Workload 5: served jobs.  Poisson arrivals (mean 20/s, seed 7); each job is
# a cascade or a two-compartment sim (probability 1/2 each) with N
# log-uniform in [10k, 2M] agents and a step count log-uniform in [1k, 20k].
@dataclasses.dataclass
class Job:
    job_id: int
    arrival_s: float
    model: Model
    seed: int
    steps: int


def served_jobs(duration_s: float = 600.0, rate_per_s: float = 20.0, seed: int = 7,
                n_range: Tuple[float, float] = (1e4, 2e6),
                steps_range: Tuple[float, float] = (1e3, 2e4)) -> List[Job]:
    rng = random.Random(seed)
    t = 0.0
    jobs = []
    while True:
        t += rng.expovariate(rate_per_s)
        if t >= duration_s:
            break
        kind = rng.random() < 0.5
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        steps = int(round(math.exp(rng.uniform(math.log(steps_range[0]), math.log(steps_range[1])))))
        job_seed = rng.randrange(1, 2 ** 31)
        model = mapk(n, drug_frac=0.05) if kind else nuclear(n, n_genes=max(1, n // 62_500))
        jobs.append(Job(len(jobs), t, model, job_seed, steps))
    return jobs


# --------------------------------------------------------------------------
# Birth-heavy model (expression, Sec. 2 and Sec. 3.4: expressors produce new
# molecules at a fixed rate; degradation removes them).  n_emit expressors E
# (p_emit per step, child C); C degrades with p 0.5 per step and itself
# emits G with p 0.2; G degrades at its first step; bystanders X bind C
# (BIND, released with p 0.2), so some parents are immune while bound.  At
# p_emit = 1 a step sees about 1.4 * n_emit births.  Density about that of
# the cascade (1,000 agents per um^3 at the start).
def births(n_emit: int = 1000, p_emit: float = 1.0, n_bystanders: int | None = None,
           edge_um: float | None = None) -> Model:
    nx = n_emit if n_bystanders is None else n_bystanders
    if edge_um is None:
        edge_um = ((n_emit + nx) / 1000.0) ** (1.0 / 3.0)
    sp = [
        Species("E", n_emit, 0.5, p_emit=p_emit, emit=1),
        Species("C", 0, 2.0, p_uni=0.5, uni_to=-1, p_emit=0.2, emit=2),
        Species("G", 0, 3.0, p_uni=1.0, uni_to=-1),
        Species("X", nx, 1.0),
    ]
    rx = [Reaction(3, 1, BIND, 3, 1, 30.0, 0.5, 0.2)]
    return Model(name="births", species=sp, reactions=rx, compartments=[Compartment(CUBE, edge_um)])
