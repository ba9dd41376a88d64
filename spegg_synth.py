"""Seeded synthetic inputs for the sPEGG per-generation update.

This module only *describes workloads*: it draws the allelic effects, builds the
caller-supplied lookup tables (viability thresholds, attack rates), lays out
special starting genotypes and lists the workload configurations.  It holds none
of the update's arithmetic (mate sampling, transmission, mutation, phenotype,
survival decisions, compaction, ecology); both the CUDA library and the CPU
oracle consume what it returns as plain inputs.

Conventions shared by every consumer (they are the library's input format, not
its computation):

* ``L`` loci per haplotype, ``W = L // 32`` uint32 words per haplotype; an
  individual is a record of ``2W`` words: haplotype 0 words then haplotype 1
  words; locus ``l`` is bit ``l % 32`` of word ``l // 32``.
* Allelic effects are int16 in Q8 fixed point (value / 256 in trait units).  The
  integer phenotype ``raw`` of an individual is the sum over loci of
  ``effect * (allele count)`` and the trait is ``z = raw / 512`` (the offspring's
  genetic value is the midpoint of its two gametes' allelic values, S2
  "Genetics", eq. S2-phenval).
* Phenotype bins: ``bin = clamp((raw + bias) >> shift, 0, 4095)``; tables are
  uint32[4096] indexed by bin.  A viability entry ``t`` means survival with
  probability ``t / 2**32``; ``0xFFFFFFFF`` means certain survival.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

N_BINS = 4096
CERTAIN = 0xFFFFFFFF


# --------------------------------------------------------------------------
# allelic effects and the phenotype-bin map
# --------------------------------------------------------------------------
def effects_q8(n_loci: int, sd: float = 0.1, seed: int = 0) -> np.ndarray:
    """Allelic effects drawn once from N(0, sd) (sd = standard deviation),
    quantised to Q8 with round-half-even and clamped to int16."""
    x = np.random.default_rng(seed).normal(0.0, sd, size=n_loci)
    q = np.rint(x * 256.0)
    return np.clip(q, -32768, 32767).astype(np.int16)


def bin_map(effects: np.ndarray) -> tuple[int, int]:
    """(bias, shift) such that every reachable raw phenotype maps into [0, 4096).

    raw ranges over [2*sum(min(e,0)), 2*sum(max(e,0))]; bias = -raw_min and
    shift is the smallest shift with (raw_max - raw_min) >> shift < 4096."""
    e = effects.astype(np.int64)
    raw_min = 2 * int(np.minimum(e, 0).sum())
    raw_max = 2 * int(np.maximum(e, 0).sum())
    span = raw_max - raw_min
    shift = 0
    while (span >> shift) >= N_BINS:
        shift += 1
    return -raw_min, shift


def bin_centre_trait(bias: int, shift: int) -> np.ndarray:
    """Trait value z at the centre of each of the 4096 bins."""
    b = np.arange(N_BINS, dtype=np.float64)
    raw_c = b * float(1 << shift) - float(bias) + (float(1 << shift) - 1.0) / 2.0
    return raw_c / 512.0


def stabilizing_table(bias: int, shift: int, s: float, theta: float = 0.0) -> np.ndarray:
    """Gaussian stabilising viability w(z) = exp(-s (z - theta)^2) as uint32
    thresholds: floor(w * 2^32) capped at 0xFFFFFFFE, and 0xFFFFFFFF exactly
    where w == 1."""
    z = bin_centre_trait(bias, shift)
    w = np.exp(-s * (z - theta) ** 2)
    t = np.floor(w * 4294967296.0)
    t = np.minimum(t, 4294967294.0).astype(np.uint64)
    t[w >= 1.0] = CERTAIN
    return t.astype(np.uint32)


def constant_table(value: int) -> np.ndarray:
    return np.full(N_BINS, value, dtype=np.uint32)


def attack_table(bias: int, shift: int, base: float = 1.0, amp: float = 0.5) -> np.ndarray:
    """Trait-dependent attack rate a(z) = base + amp * tanh(z) in Q16 (uint32)."""
    z = bin_centre_trait(bias, shift)
    a = np.rint((base + amp * np.tanh(z)) * 65536.0)
    return np.clip(a, 0, 2 ** 32 - 1).astype(np.uint32)


def genotype_table(bias: int, shift: int, effects: np.ndarray,
                   w_by_copies: List[float]) -> np.ndarray:
    """Viability table for a one-locus model: locus 0 carries the only nonzero
    effect; genotypes with 0/1/2 copies get viabilities w_by_copies[0..2]
    (given as probabilities; 1.0 means certain)."""
    t = constant_table(CERTAIN)
    e0 = int(effects[0])
    for copies, w in enumerate(w_by_copies):
        raw = copies * e0
        v = raw + bias
        b = 0 if v < 0 else min(v >> shift, N_BINS - 1)
        t[b] = CERTAIN if w >= 1.0 else min(int(math.floor(w * 4294967296.0)), 0xFFFFFFFE)
    return t


def p0_threshold(p0: float) -> int:
    """Q32 threshold for initial allele frequency p0 (allele 1 iff u < thr)."""
    return int(min(max(math.floor(p0 * 4294967296.0), 0), 0xFFFFFFFF))


# --------------------------------------------------------------------------
# special starting genotypes (packed records, uint32[n, 2W])
# --------------------------------------------------------------------------
def genotypes_uniform(n: int, n_loci: int, hap0_word: int, hap1_word: int) -> np.ndarray:
    w = n_loci // 32
    g = np.empty((n, 2 * w), dtype=np.uint32)
    g[:, :w] = np.uint32(hap0_word)
    g[:, w:] = np.uint32(hap1_word)
    return g


def genotypes_random_haplotype_pairs(n: int, n_loci: int, seed: int) -> np.ndarray:
    """Each haplotype is independently all-0 or all-1 with probability 1/2:
    allele frequency 1/2 at every locus, Hardy-Weinberg pairing of haplotypes,
    and maximal linkage disequilibrium D = 1/4 between every pair of loci."""
    w = n_loci // 32
    rng = np.random.default_rng(seed)
    which = rng.integers(0, 2, size=(n, 2))
    g = np.empty((n, 2 * w), dtype=np.uint32)
    g[:, :w] = np.where(which[:, :1] == 1, np.uint32(0xFFFFFFFF), np.uint32(0))
    g[:, w:] = np.where(which[:, 1:] == 1, np.uint32(0xFFFFFFFF), np.uint32(0))
    return g


def genotypes_bernoulli(n: int, n_loci: int, p: float, seed: int) -> np.ndarray:
    w = n_loci // 32
    rng = np.random.default_rng(seed)
    bits = (rng.random((n, 2, n_loci)) < p).astype(np.uint64)
    bits = bits.reshape(n, 2, w, 32)
    words = (bits << np.arange(32, dtype=np.uint64)).sum(axis=3).astype(np.uint32)
    return words.reshape(n, 2 * w)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    """One population's inputs.  All tables are uint32[4096]."""
    name: str
    n: int
    n_loci: int
    n_gen: int
    seed: int
    replicate: int
    effects: np.ndarray
    bias: int
    shift: int
    surv_table: np.ndarray
    mu: float
    p0_q32: int = 0x80000000
    init_genotypes: Optional[np.ndarray] = None
    # ecology (consumer-resource); None when the population has no resource
    eco_r: Optional[float] = None
    eco_K: Optional[float] = None
    eco_R0: Optional[float] = None
    eco_R_half: Optional[float] = None
    attack: Optional[np.ndarray] = None
    eco_model: int = 0      # 0 logistic resource, 1 Beverton-Holt
    eco_r_sd: float = 0.0   # Beverton-Holt: standard deviation of the growth rate
    s: float = 0.0
    # linkage map (None: free recombination): distance in Morgans between loci
    # l-1 and l, negative where locus l starts a new chromosome
    map_morgans: Optional[np.ndarray] = None
    # weighted parents (None: uniform): uint32 weights over the phenotype bins
    mother_weights: Optional[np.ndarray] = None
    father_weights: Optional[np.ndarray] = None
    # dominance deviations (None: additive): int16 Q8 per locus, added at
    # heterozygous loci; bias/shift then cover the widened phenotype range
    dominance: Optional[np.ndarray] = None
    # continuous allelic values (allele_model 1): int16 Q8 per allele copy,
    # Gaussian mutation steps (sd mut_sd) and environmental deviations (sd
    # env_sd), trait units; founders = biallelic draws mapped to effect * allele
    allele_model: int = 0
    mut_sd: float = 0.0
    env_sd: float = 0.0
    init_values: Optional[np.ndarray] = None

    @property
    def words(self) -> int:
        return self.n_loci // 32

    @property
    def has_ecology(self) -> bool:
        return self.attack is not None


def linkage_map(n_loci: int, chromosomes: int, morgans: float) -> np.ndarray:
    """Evenly spaced map: the loci split into `chromosomes` runs of equal
    length (in record order), each `morgans` long with equal intervals
    between adjacent loci; -1 marks each chromosome's first locus."""
    per = n_loci // chromosomes
    assert per * chromosomes == n_loci and per >= 1
    m = np.empty(n_loci, np.float64)
    for c in range(chromosomes):
        m[c * per] = -1.0
        if per > 1:
            m[c * per + 1:(c + 1) * per] = morgans / (per - 1)
    return m


def with_linkage(w: "Workload", chromosomes: int = 4, morgans: float = 1.0) -> "Workload":
    """The same workload with an evenly spaced linkage map."""
    import dataclasses
    return dataclasses.replace(w, map_morgans=linkage_map(w.n_loci, chromosomes, morgans),
                               name=w.name + f"+map{chromosomes}x{morgans:g}M")


def continuous_trait(n: int = 10_000, n_loci: int = 64, n_gen: int = 100, mu: float = 1e-3,
                     mut_sd: float = 0.05, env_sd: float = 0.2, s: float = 0.5, seed: int = 0,
                     replicate: int = 0, effects_seed: int = 0, name: str = "continuous") -> "Workload":
    """The paper's continuous genetic model (S2 "Genetics"): allelic values
    start at effect * allele of biallelic founders (p0 = 1/2), mutate by
    Gaussian steps of sd `mut_sd` and the phenotype carries an environmental
    deviation of sd `env_sd` (trait units); Gaussian stabilising viability
    exp(-s z^2) over a bin map wide enough for the drift of the values."""
    import dataclasses
    w = single_species(n=n, n_loci=n_loci, n_gen=n_gen, mu=mu, s=s, seed=seed, replicate=replicate,
                       effects_seed=effects_seed, name=name)
    span = 2 * int(np.abs(w.effects.astype(np.int64)).sum()) + 4096 * 4
    shift = 0
    while ((2 * span) >> shift) >= N_BINS:
        shift += 1
    bias = span
    return dataclasses.replace(w, allele_model=1, mut_sd=mut_sd, env_sd=env_sd, bias=bias, shift=shift,
                               surv_table=stabilizing_table(bias, shift, s))


def with_dominance(w: "Workload", sd: float = 0.1, seed: int = 99) -> "Workload":
    """The same workload with dominance deviations d_l = Q8(N(0, sd)) and the
    bin map and viability table rebuilt over the widened phenotype range
    (raw = sum e_l (a0 + a1) + sum d_l [a0 != a1])."""
    import dataclasses
    d = effects_q8(w.n_loci, sd, seed)
    e = w.effects.astype(np.int64)
    # per locus the genotype values are 0, e + d, 2e: bounds over them
    vals = np.stack([np.zeros_like(e), e + d.astype(np.int64), 2 * e])
    raw_min, raw_max = int(vals.min(axis=0).sum()), int(vals.max(axis=0).sum())
    bias = -raw_min
    shift = 0
    while ((raw_max - raw_min) >> shift) >= N_BINS:
        shift += 1
    table = stabilizing_table(bias, shift, w.s if w.s else 0.5)
    out = dataclasses.replace(w, dominance=d, bias=bias, shift=shift, surv_table=table, name=w.name + "+dominance")
    if w.attack is not None:
        out.attack = attack_table(bias, shift)
    return out


def fecundity_weights(bias: int, shift: int, slope: float = 1.0, theta: float = 0.0) -> np.ndarray:
    """Parent weights rising with the trait: w(z) = 2^16 (1 + tanh(slope (z -
    theta))) + 1 at each bin centre (always positive), as uint32."""
    z = bin_centre_trait(bias, shift)
    w = np.floor(65536.0 * (1.0 + np.tanh(slope * (z - theta)))) + 1.0
    return w.astype(np.uint32)


def with_beverton_holt(w: "Workload", r: float = 2.0, r_sd: float = 0.2) -> "Workload":
    """The same consumer-resource workload with a Beverton-Holt resource whose
    growth rate is r + r_sd z each generation (z: Irwin-Hall(12) normal)."""
    import dataclasses
    assert w.has_ecology
    return dataclasses.replace(w, eco_model=1, eco_r=r, eco_r_sd=r_sd, name=w.name + f"+BH{r:g}sd{r_sd:g}")


def with_weights(w: "Workload", slope: float = 1.0) -> "Workload":
    """The same workload with trait-dependent mother and father weights
    (fathers twice as steep, as for size-dependent male success)."""
    import dataclasses
    return dataclasses.replace(w, mother_weights=fecundity_weights(w.bias, w.shift, slope),
                               father_weights=fecundity_weights(w.bias, w.shift, 2.0 * slope),
                               name=w.name + f"+weights{slope:g}")


def single_species(n: int = 10_000, n_loci: int = 32, n_gen: int = 100, mu: float = 1e-4,
                   s: float = 0.5, seed: int = 0, replicate: int = 0,
                   effects_seed: int = 0, name: str = "single-species") -> Workload:
    """Single species, additive trait, Gaussian stabilising viability, random
    mating, free recombination, per-locus mutation; defaults are the
    N=10,000 / L=32 / 100-generation workload."""
    e = effects_q8(n_loci, 0.1, effects_seed)
    bias, shift = bin_map(e)
    return Workload(name=name, n=n, n_loci=n_loci, n_gen=n_gen, seed=seed, replicate=replicate,
                    effects=e, bias=bias, shift=shift,
                    surv_table=stabilizing_table(bias, shift, s), mu=mu, s=s)


def consumer_resource(n: int = 1_000_000, n_loci: int = 128, n_gen: int = 1000, mu: float = 1e-5,
                      s: float = 0.5, r: float = 0.5, K: float = 1e7, seed: int = 0,
                      replicate: int = 0, effects_seed: int = 1,
                      name: str = "consumer-resource") -> Workload:
    """One consumer species feeding on a logistic resource (r, K); survival =
    stabilising viability x resource factor R/(R + K/10); trait-dependent
    attack rate; defaults are the N=1,000,000 / L=128 / 1,000-generation
    workload with R0 = K/2."""
    w = single_species(n, n_loci, n_gen, mu, s, seed, replicate, effects_seed, name)
    w.eco_r, w.eco_K, w.eco_R0, w.eco_R_half = r, K, K / 2.0, K / 10.0
    w.attack = attack_table(w.bias, w.shift)
    return w


def batch_replicates(count: int = 4096, n_gen: int = 500, n_min: int = 1_000, n_max: int = 200_000,
                     loci_choices=(32, 64, 128), s_max: float = 0.5, mu: float = 1e-5,
                     seed: int = 0, spec_seed: int = 12345) -> List[Workload]:
    """Independent single-species replicates: N log-uniform in [n_min, n_max],
    L uniform over loci_choices, selection strength uniform in [0, s_max];
    replicate r uses Philox seed `seed` and replicate id r."""
    rng = np.random.default_rng(spec_seed)
    out = []
    for r in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        L = int(rng.choice(loci_choices))
        s = float(rng.uniform(0.0, s_max))
        out.append(single_species(n, L, n_gen, mu, s, seed, r, effects_seed=1000 + r,
                                  name=f"replicate-{r}"))
    return out


def served_trace(count: int = 200, rate: float = 200.0, n_min: int = 1_000, n_max: int = 2_000_000,
                 loci_choices=(64, 256), gen_min: int = 100, gen_max: int = 2000, mu: float = 1e-5,
                 s_max: float = 0.5, seed: int = 0, trace_seed: int = 2024):
    """Parameter-sweep jobs arriving as a Poisson stream: returns (workloads,
    generation counts, arrival times in seconds).  N log-uniform in
    [n_min, n_max], L uniform over loci_choices, generations uniform in
    [gen_min, gen_max], selection strength uniform in [0, s_max]; job i uses
    replicate id i."""
    rng = np.random.default_rng(trace_seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    arrivals = np.cumsum(gaps) - gaps[0]
    ws, gens = [], []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        L = int(rng.choice(loci_choices))
        g = int(rng.integers(gen_min, gen_max + 1))
        s = float(rng.uniform(0.0, s_max))
        ws.append(single_species(n, L, g, mu, s, seed, i, effects_seed=5000 + i, name=f"job-{i}"))
        gens.append(g)
    return ws, gens, arrivals


# --------------------------------------------------------------------------
# spatial community (species on a torus of patches, age classes 0/1/2)
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Species:
    """One species of a spatial community.  tables: uint32[3, 4096] viability
    by age class; D, A: survival interaction; G, P, E, C, beta_q16, bmax:
    recruitment (see the library header for the integer formulas)."""
    effects: np.ndarray
    bias: int
    shift: int
    tables: np.ndarray
    mu: float
    n0: int
    p0_q32: int
    D: int
    A: List[int]
    G: int
    P: List[int]
    E: int
    C: List[int]
    beta_q16: int
    bmax: int


@dataclasses.dataclass
class Community:
    X: int
    Y: int
    n_loci: int
    seed: int
    disp_q32: int
    species: List[Species]
    n_gen: int = 200

    @property
    def patches(self) -> int:
        return self.X * self.Y


def spatial_community(X: int = 64, Y: int = 64, n0: int = 814, n_loci: int = 256, n_gen: int = 200,
                      disp: float = 0.05, mu: float = 1e-5, s: float = 0.3, seed: int = 0,
                      effects_seed: int = 77) -> Community:
    """Three species (prey, competitor, predator) on an X x Y torus, n0 founders
    per species and patch (10^7 individuals at the defaults), L loci, dispersal
    probability `disp` to one of the four neighbours.  Viabilities are Gaussian
    stabilising in the trait around the founders' mean, scaled per age class
    (newborn, juvenile, adult);
    recruitment falls with the species' own local density, the predator's
    rises with local prey; all three depress the prey's and competitor's
    survival, the predator only its own."""
    rng_seeds = [effects_seed + k for k in range(3)]
    age_scale = [[0.80, 0.90, 0.82], [0.80, 0.90, 0.82], [0.85, 0.92, 0.85]]
    inter_A = [[1, 1, 3], [1, 1, 3], [0, 0, 1]]
    D = [400000, 400000, 400000]
    G = [1500, 1500, 0]
    P = [[0, 0, 0], [0, 0, 0], [1, 1, 0]]
    E = [0, 0, 500]
    C = [[2, 0, 0], [0, 2, 0], [0, 0, 2]]
    beta = [int(0.7 * 65536), int(0.7 * 65536), int(0.65 * 65536)]
    out = []
    for k in range(3):
        e = effects_q8(n_loci, 0.1, rng_seeds[k])
        bias, shift = bin_map(e)
        # optimum at the founders' mean trait (allele frequency 1/2: raw = sum e)
        theta = float(e.astype(np.float64).sum()) / 512.0
        w = stabilizing_table(bias, shift, s, theta).astype(np.float64)
        tabs = np.stack([np.minimum(np.floor(w * a), 4294967294.0) for a in age_scale[k]]).astype(np.uint32)
        out.append(Species(effects=e, bias=bias, shift=shift, tables=tabs, mu=mu, n0=n0, p0_q32=0x80000000,
                           D=D[k], A=list(inter_A[k]), G=G[k], P=list(P[k]), E=E[k], C=list(C[k]),
                           beta_q16=beta[k], bmax=2 * n0))
    return Community(X=X, Y=Y, n_loci=n_loci, seed=seed, disp_q32=p0_threshold(disp), species=out, n_gen=n_gen)
