"""Pins for the oracle's weighted parents (S2 "Reproduction": the chance that
an individual parents an egg grows with its size relative to the others'):
each parent is drawn with probability proportional to its weight, checked on
founders of two marked classes whose offspring reveal their parents' class."""
import math

import numpy as np

import oracle
import spegg_synth as S

L = 32


def two_class_population(n_a, n_b, mother_w, father_w, seed=1):
    """Founders: n_a of class A (allele 1 everywhere) then n_b of class B
    (allele 0 everywhere); effects +10 at every locus, so A and B fall in
    different phenotype bins; certain survival, no mutation."""
    e = np.full(L, 10, np.int16)
    bias, shift = S.bin_map(e)
    rec = np.zeros((n_a + n_b, 2), np.uint32)
    rec[:n_a] = 0xFFFFFFFF
    p = oracle.OraclePopulation(n_a + n_b, L, seed, 0, e, S.constant_table(S.CERTAIN), bias, shift, 0.0,
                                init_genotypes=rec)
    bins = np.arange(4096)
    bin_a, bin_b = (2 * L * 10 + bias) >> shift, bias >> shift
    mw = np.ones(4096, np.uint32)
    fw = np.ones(4096, np.uint32)
    mw[bin_a], mw[bin_b] = mother_w
    fw[bin_a], fw[bin_b] = father_w
    assert bin_a != bin_b and 0 <= bin_b < bin_a < len(bins)
    p.set_weights(mw, fw)
    return p


def parent_classes(p):
    """Fraction of offspring whose mother (haplotype 0) and father
    (haplotype 1) belong to class A."""
    p.step(1)
    g = p.genotypes()
    mom_a = g[:, 0] == 0xFFFFFFFF
    dad_a = g[:, 1] == 0xFFFFFFFF
    assert np.all(mom_a | (g[:, 0] == 0)) and np.all(dad_a | (g[:, 1] == 0))
    return mom_a, dad_a


def test_parents_drawn_in_proportion_to_weight():
    n_a, n_b = 5000, 15000
    p = two_class_population(n_a, n_b, mother_w=(3, 1), father_w=(1, 5))
    mom_a, dad_a = parent_classes(p)
    n = len(mom_a)
    for obs, exp in ((mom_a.mean(), n_a * 3 / (n_a * 3 + n_b * 1)), (dad_a.mean(), n_a * 1 / (n_a * 1 + n_b * 5))):
        assert abs(obs - exp) < 5 * math.sqrt(exp * (1 - exp) / n), (obs, exp)


def test_zero_weight_class_does_not_parent():
    n_a, n_b = 8000, 8000
    p = two_class_population(n_a, n_b, mother_w=(7, 0), father_w=(0, 2))
    mom_a, dad_a = parent_classes(p)
    # a zero-weight parent appears only if all 64 proposals are rejected:
    # probability 2^-64 per offspring here
    assert mom_a.all()
    assert not dad_a.any()


def test_equal_weights_keep_wright_fisher_drift():
    """Equal weights accept the first proposal: heterozygosity decays as
    E[H_t] = H_0 (1 - 1/2N)^t, as with uniform mating."""
    n, t, reps = 50, 30, 240
    H = []
    for rep in range(reps):
        w = S.single_species(n=n, n_loci=L, mu=0.0, seed=rep)
        w.surv_table = S.constant_table(S.CERTAIN)
        w.mother_weights = np.full(4096, 9, np.uint32)
        w.father_weights = np.full(4096, 9, np.uint32)
        p = oracle.OraclePopulation.from_workload(w)
        g0 = p.genotypes()
        p.step(t)
        g = p.genotypes()

        def het(g):
            bits = (g[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1
            freq = bits.reshape(n, 2 * 32).reshape(n, 2, 32).mean(axis=(0, 1))
            return (2 * freq * (1 - freq)).mean()

        H.append((het(g0), het(g)))
    H = np.array(H)
    expect = H[:, 0].mean() * (1 - 1 / (2 * n)) ** t
    se = H[:, 1].std() / math.sqrt(reps)
    assert abs(H[:, 1].mean() - expect) < 4 * se + 0.01
