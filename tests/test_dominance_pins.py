"""Pins for the oracle's dominance deviations (the non-additive genotype-
phenotype maps of the paper's Main text): the genetic value is
sum_l e_l (a0 + a1) + sum_l d_l [a0 != a1]."""
import dataclasses
import math

import numpy as np

import oracle
import spegg_synth as S


def unpack(g, L):
    n, w = g.shape[0], L // 32
    bits = (g.reshape(n, 2, w)[..., None] >> np.arange(32, dtype=np.uint32)) & 1
    return bits.reshape(n, 2, L).astype(np.int64)


def brute_raw(g, L, e, d):
    a = unpack(g, L)
    return (a.sum(axis=1) * e.astype(np.int64)).sum(axis=1) + ((a[:, 0] != a[:, 1]) * d.astype(np.int64)).sum(axis=1)


def test_statistics_equal_the_brute_force_genetic_value():
    for L in (32, 128):
        w = S.with_dominance(S.single_species(n=3000, n_loci=L, mu=1e-3, seed=L), sd=0.2)
        p = oracle.OraclePopulation.from_workload(w)
        st = p.step(3)[-1]
        raw = brute_raw(p.genotypes(), L, w.effects, w.dominance)
        assert st["sum_raw"] == raw.sum()
        assert st["sum_raw2"] == (raw * raw).sum()
        assert st["min_raw"] == raw.min() and st["max_raw"] == raw.max()


def test_zero_dominance_is_the_additive_model():
    w = S.single_species(n=2000, n_loci=64, mu=1e-3, seed=4)
    wd = dataclasses.replace(w, dominance=np.zeros(64, np.int16))
    a, b = oracle.OraclePopulation.from_workload(w), oracle.OraclePopulation.from_workload(wd)
    sa, sb = a.step(5), b.step(5)
    for name in sa.dtype.names:
        assert np.array_equal(sa[name], sb[name]), name
    assert np.array_equal(a.genotypes(), b.genotypes())


def test_mean_and_variance_at_half_frequency():
    """Hardy-Weinberg at p = 1/2 (neutral offspring of founders drawn at
    p0 = 1/2): per locus the genotype values 0, e + d, 2e have probabilities
    1/4, 1/2, 1/4, so E[raw] = sum (e + d/2) and Var[raw] = sum (e^2/2 +
    d^2/4) (additive plus dominance variance)."""
    L, n = 64, 40000
    w = S.with_dominance(S.single_species(n=n, n_loci=L, mu=0.0, seed=1), sd=0.3)
    w.surv_table = S.constant_table(S.CERTAIN)
    p = oracle.OraclePopulation.from_workload(w)
    st = p.step(1)[-1]
    e, d = w.effects.astype(np.float64), w.dominance.astype(np.float64)
    mean = float(st["sum_raw"]) / n
    var = float(st["sum_raw2"]) / n - mean * mean
    exp_mean = (e + d / 2).sum()
    exp_var = (e * e / 2 + d * d / 4).sum()
    assert abs(mean - exp_mean) < 5 * math.sqrt(exp_var / n)
    assert abs(var / exp_var - 1) < 5 * math.sqrt(2 / n) + 0.02
