"""Pins of the oracle's per-locus allele counts (allele-1 copies of each locus
over both haplotypes of the current generation; S2 "Genetics", biallelic
diploid loci): the packed records unpacked independently, the total against
the oracle's own allele statistic, and populations fixed for one allele."""
import numpy as np
import pytest

import oracle
import spegg_synth as S


def unpacked_counts(geno: np.ndarray, n_loci: int) -> np.ndarray:
    """Per-locus counts from packed records [n, 2W]: bit l % 32 of word
    l // 32 of each haplotype."""
    n = geno.shape[0]
    words = geno.reshape(n, 2, n_loci // 32).astype(np.uint64)
    bits = (words[..., None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)
    return bits.reshape(n, 2, n_loci).sum(axis=(0, 1)).astype(np.uint32)


@pytest.mark.parametrize("n,n_loci,mu", [(1, 32, 1e-2), (333, 64, 1e-3), (2049, 128, 5e-3), (700, 256, 1e-2)])
def test_locus_counts_match_packed_records_each_generation(n, n_loci, mu):
    w = S.consumer_resource(n=n, n_loci=n_loci, mu=mu, s=1.0, K=max(4.0 * n, 50.0), seed=12)
    orc = oracle.OraclePopulation.from_workload(w)
    assert np.array_equal(orc.locus_counts(), unpacked_counts(orc.genotypes(), n_loci))  # founders
    for _ in range(4):
        orc.step(1)
        c = orc.locus_counts()
        assert c.shape == (n_loci,) and c.dtype == np.uint32
        assert np.array_equal(c, unpacked_counts(orc.genotypes(), n_loci))
        assert c.max() <= 2 * n


@pytest.mark.parametrize("n_loci", [32, 128, 256])
def test_locus_counts_total_is_the_allele_statistic(n_loci):
    w = S.single_species(n=1500, n_loci=n_loci, mu=2e-3, s=1.5, seed=4)
    orc = oracle.OraclePopulation.from_workload(w)
    for _ in range(5):
        st = orc.step(1)
        assert int(orc.locus_counts().sum()) == int(st[-1]["allele"])


@pytest.mark.parametrize("fill,expect", [(0, 0), (0xFFFFFFFF, 2)])
def test_locus_counts_of_a_fixed_population(fill, expect):
    """Founders all 0 (or all 1) and no mutation: every gamete is 0 (or 1)
    at every locus whatever the recombination, so every generation counts
    0 (or 2N) copies at every locus."""
    n, n_loci = 400, 64
    w = S.single_species(n=n, n_loci=n_loci, mu=0.0, seed=6)
    w.init_genotypes = np.full((n, 2 * (n_loci // 32)), fill, np.uint32)
    w.surv_table = S.constant_table(S.CERTAIN)
    orc = oracle.OraclePopulation.from_workload(w)
    for _ in range(3):
        orc.step(1)
        assert np.array_equal(orc.locus_counts(), np.full(n_loci, expect * n, np.uint32))


def test_locus_counts_refuse_continuous_populations():
    orc = oracle.OraclePopulation.from_workload(S.continuous_trait(n=50, n_loci=32))
    with pytest.raises(ValueError):
        orc.locus_counts()


def test_locus_counts_follow_binomial_sampling_under_neutrality():
    """Wright-Fisher with certain survival and no mutation: each of the next
    generation's 2N copies of a locus is a copy of a uniformly drawn parental
    copy, so given c the next count is Binomial(2N, c / 2N).  Pooled over 256
    loci and 30 generations, the changes have mean 0 (z within 5) and their
    squares average 2N p(1 - p) (ratio within 10 %)."""
    n, n_loci = 500, 256
    w = S.single_species(n=n, n_loci=n_loci, mu=0.0, seed=17)
    w.surv_table = S.constant_table(S.CERTAIN)
    orc = oracle.OraclePopulation.from_workload(w)
    prev = orc.locus_counts().astype(np.float64)
    dsum = var = sq = 0.0
    for _ in range(30):
        orc.step(1)
        cur = orc.locus_counts().astype(np.float64)
        p = prev / (2 * n)
        v = 2 * n * p * (1 - p)
        dsum += (cur - prev).sum()
        var += v.sum()
        sq += ((cur - prev) ** 2).sum()
        prev = cur
    assert abs(dsum) / np.sqrt(var) < 5.0
    assert abs(sq / var - 1.0) < 0.10
