"""Pins for the oracle's linkage maps (the "variable linkage maps" of the
paper's Main text, read as Haldane's no-interference model): what the model
fixes in closed form, checked on gametes of parents heterozygous at every
locus (haplotype 0 all allele 0, haplotype 1 all allele 1), so an offspring
haplotype spells out the origin of every locus of its gamete."""
import math

import numpy as np
import pytest
from scipy import stats as sps

import oracle
import spegg_synth as S

N = 20000


def het_founders(n, L):
    w = L // 32
    rec = np.zeros((n, 2 * w), np.uint32)
    rec[:, w:] = 0xFFFFFFFF
    return rec


def gametes(map_morgans, L, n=N, seed=11):
    """Both gametes of n offspring of all-heterozygous founders: an array
    [2n, L] of origins (0: the parent's haplotype 0, 1: haplotype 1)."""
    e = np.zeros(L, np.int16)
    bias, shift = S.bin_map(e)
    p = oracle.OraclePopulation(n, L, seed, 0, e, S.constant_table(S.CERTAIN), bias, shift, 0.0,
                                init_genotypes=het_founders(n, L))
    p.set_linkage(map_morgans)
    p.step(1)
    g = p.genotypes()
    w = L // 32
    bits = (g[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1  # [n, 2w, 32]
    hap0 = bits[:, :w, :].reshape(n, L)
    hap1 = bits[:, w:, :].reshape(n, L)
    return np.concatenate([hap0, hap1]).astype(np.int64)


def haldane(d):
    return 0.5 * (1.0 - math.exp(-2.0 * d))


def test_recombination_fraction_per_interval_follows_haldane():
    L = 64
    m = np.full(L, 0.02)
    m[0] = -1.0
    m[32] = -1.0  # a second chromosome
    probe = {3: 0.0, 6: 0.01, 9: 0.05, 12: 0.1, 15: 0.3, 18: 0.7, 21: 1.5, 24: 3.0, 40: 0.2}
    for l, d in probe.items():
        m[l] = d
    o = gametes(m, L)
    rec = (o[:, 1:] != o[:, :-1])  # interval l is column l-1
    n2 = o.shape[0]
    for l, d in probe.items():
        r = rec[:, l - 1].mean()
        if d == 0.0:
            assert rec[:, l - 1].sum() == 0, "a zero-length interval never recombines"
            continue
        exp = haldane(d)
        sd = math.sqrt(exp * (1 - exp) / n2)
        assert abs(r - exp) < 5 * sd + 1e-4, (l, d, r, exp)
    # across the chromosome boundary: free recombination
    r = rec[:, 31].mean()
    assert abs(r - 0.5) < 5 * math.sqrt(0.25 / n2)


def test_no_interference_between_intervals():
    """Haldane: recombination in two intervals of one chromosome is
    independent (no crossover interference)."""
    L = 32
    m = np.full(L, 0.05)
    m[0] = -1.0
    m[8], m[20] = 0.35, 0.5
    o = gametes(m, L, seed=5)
    a = o[:, 8] != o[:, 7]
    b = o[:, 20] != o[:, 19]
    table = np.array([[np.sum(~a & ~b), np.sum(~a & b)], [np.sum(a & ~b), np.sum(a & b)]])
    assert sps.chi2_contingency(table, correction=False)[1] > 1e-4
    assert abs(a.mean() - haldane(0.35)) < 5 * math.sqrt(0.25 / len(a))
    assert abs(b.mean() - haldane(0.5)) < 5 * math.sqrt(0.25 / len(b))


def test_chromosomes_start_from_independent_fair_coins():
    L = 64
    m = S.linkage_map(L, 8, 0.5)  # 8 chromosomes of 8 loci
    o = gametes(m, L, seed=7)
    starts = o[:, ::8]  # origin of each chromosome's first locus
    n2 = starts.shape[0]
    assert np.all(np.abs(starts.mean(axis=0) - 0.5) < 5 * math.sqrt(0.25 / n2))
    for c in range(7):
        t = np.array([[np.sum((starts[:, c] == x) & (starts[:, c + 1] == y)) for y in (0, 1)] for x in (0, 1)])
        assert sps.chi2_contingency(t, correction=False)[1] > 1e-4


def test_zero_length_map_transmits_whole_haplotypes():
    L = 32
    m = np.zeros(L)
    m[0] = -1.0
    o = gametes(m, L, n=4000, seed=3)
    assert np.all((o == 0).all(axis=1) | (o == 1).all(axis=1))
    frac = o[:, 0].mean()
    assert abs(frac - 0.5) < 5 * math.sqrt(0.25 / o.shape[0])


def test_every_locus_its_own_chromosome_is_free_recombination():
    """A map that starts a chromosome at every locus has no linked interval:
    every adjacent pair recombines with probability 1/2, independently."""
    L = 32
    m = np.full(L, -1.0)
    o = gametes(m, L, n=8000, seed=9)
    rec = (o[:, 1:] != o[:, :-1]).mean(axis=0)
    assert np.all(np.abs(rec - 0.5) < 5 * math.sqrt(0.25 / o.shape[0]))


def test_crossover_count_table_is_binomial():
    """The crossover-count table is the Binomial(2^16, D/2^16) CDF (the
    Poisson(D) limit of Haldane's model), within 2 units of Q32."""
    for D in (0.5, 2.0, 6.0):
        cdf = oracle.mutation_cdf(D / 65536.0, 65536)
        ks = np.arange(len(cdf))
        exact = np.floor(sps.binom.cdf(ks, 65536, D / 65536.0) * 2.0 ** 32)
        assert np.all(np.abs(cdf.astype(np.float64) - exact) <= 2)
        assert abs(sps.binom.cdf(ks[-1], 65536, D / 65536.0) - sps.poisson.cdf(ks[-1], D)) < 1e-3


def test_map_validation():
    e = np.zeros(32, np.int16)
    bias, shift = S.bin_map(e)
    p = oracle.OraclePopulation(10, 32, 1, 0, e, S.constant_table(S.CERTAIN), bias, shift, 0.0)
    with pytest.raises(ValueError):
        p.set_linkage(np.full(32, 1.0))  # 31 Morgans: beyond the 16-Morgan limit
    with pytest.raises(ValueError):
        p.set_linkage(np.full(32, np.nan))
