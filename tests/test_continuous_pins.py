"""Pins for the oracle's continuous allelic values (S2 "Genetics": values vary
continuously, a mutation moves a value by a normal step, the phenotype is
normal around the genetic value), read with int16 Q8 values and Irwin-Hall(12)
normal steps in exact integer arithmetic."""
import dataclasses
import math

import numpy as np
from scipy import stats as sps

import oracle
import spegg_synth as S

L = 64


def population(n, mu, mut_sd, env_sd, values, seed=1):
    w = S.continuous_trait(n=n, n_loci=L, mu=mu, mut_sd=mut_sd, env_sd=env_sd, seed=seed)
    w = dataclasses.replace(w, surv_table=S.constant_table(S.CERTAIN), init_values=values)
    return w, oracle.OraclePopulation.from_workload(w)


def test_founder_values_are_effect_times_allele():
    w = S.continuous_trait(n=500, n_loci=L, seed=4)
    v = oracle.OraclePopulation.from_workload(w).values()
    b = dataclasses.replace(w, allele_model=0)
    g = oracle.OraclePopulation.from_workload(b).genotypes()
    bits = ((g.reshape(500, 2, 2)[..., None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(500, 2, L)
    assert np.array_equal(v, (bits * w.effects.astype(np.int64)).astype(np.int16))


def test_mutation_steps_follow_the_irwin_hall_normal():
    n, mu, sd = 20000, 0.05, 0.2
    _, p = population(n, mu, sd, 0.0, np.zeros((n, 2, L), np.int16))
    p.step(1)
    steps = p.values().astype(np.int64).ravel()
    copies = steps.size
    nz = steps[steps != 0]
    expect = copies * mu
    assert abs(len(nz) - expect) < 5 * math.sqrt(expect * (1 - mu)) + 0.01 * expect  # a few steps are 0
    s = sd * 256.0
    assert np.abs(nz).max() <= 6 * s + 1
    # floor rounding: mean -1/2; sd s; excess kurtosis of Irwin-Hall(12) = -0.1
    m = len(nz)
    assert abs(nz.mean() + 0.5) < 5 * s / math.sqrt(m) + 0.5
    assert abs(nz.std() / s - 1) < 0.02
    assert abs(sps.kurtosis(nz) + 0.1) < 0.06


def test_inheritance_takes_one_parental_value_per_copy():
    n = 20000
    v = np.zeros((n, 2, L), np.int16)
    v[:, 0, :], v[:, 1, :] = 100, -100
    _, p = population(n, 0.0, 0.0, 0.0, v)
    p.step(1)
    c = p.values()
    assert np.all(np.abs(c) == 100)
    frac = (c == 100).mean(axis=0)  # per haplotype and locus
    assert np.all(np.abs(frac - 0.5) < 5 * math.sqrt(0.25 / n))
    het = (c[:, 0, :] != c[:, 1, :]).mean()
    assert abs(het - 0.5) < 5 * math.sqrt(0.25 / (n * L))


def test_phenotype_is_values_plus_environmental_deviation():
    n, env = 40000, 0.3
    w, p = population(n, 0.0, 0.0, 0.0, None)
    st = p.step(1)[-1]
    g = p.values().astype(np.int64).sum(axis=(1, 2))
    assert st["sum_raw"] == g.sum() and st["sum_raw2"] == (g * g).sum()
    w2, p2 = population(n, 0.0, 0.0, env, None)
    st2 = p2.step(1)[-1]
    g2 = p2.values().astype(np.int64).sum(axis=(1, 2))
    se = env * 512.0
    mean_e = float(st2["sum_raw"]) / n - g2.mean()
    var_raw = float(st2["sum_raw2"]) / n - (float(st2["sum_raw"]) / n) ** 2
    assert abs(mean_e + 0.5) < 5 * se / math.sqrt(n)
    assert abs((var_raw - g2.var()) / se ** 2 - 1) < 0.05
