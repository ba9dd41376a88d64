"""Pins for the spatial-community oracle: checks against what the model's
statement fixes (neighbour geometry on the torus, per-age survival
probabilities, the interaction factor, the integer recruitment rule,
Mendelian transmission from adults only, conservation, layout order)."""
import math

import numpy as np
import pytest
from scipy import stats as sps

import oracle
import spegg_synth as S

CERT = S.CERTAIN


def species(L=32, n0=0, tables=None, mu=0.0, D=1, A=(0, 0, 0), G=0, P=(0, 0, 0), E=0, C=(0, 0, 0),
            beta=0, bmax=0, p0=0x80000000, effects=None):
    e = np.zeros(L, np.int16) if effects is None else effects
    bias, shift = S.bin_map(e)
    t = np.full((3, 4096), CERT, np.uint32) if tables is None else tables
    return S.Species(effects=e, bias=bias, shift=shift, tables=t, mu=mu, n0=n0, p0_q32=p0, D=D, A=list(A), G=G,
                     P=list(P), E=E, C=list(C), beta_q16=beta, bmax=bmax)


def community(X, Y, sps_, disp=0.0, L=32, seed=1):
    return S.Community(X=X, Y=Y, n_loci=L, seed=seed, disp_q32=S.p0_threshold(disp) if disp < 1 else 0xFFFFFFFF,
                       species=sps_)


def tagged(n, L, word, ages):
    w = L // 32
    rec = np.full((n, 2 * w), np.uint32(word), dtype=np.uint32)
    return rec, np.asarray(ages, dtype=np.uint8)


def test_dispersal_reaches_exactly_the_four_neighbours_uniformly():
    """Everyone moves (probability 1), survival certain, no births: a tagged
    deme at the centre of a 5 x 5 torus ends up only in its N/S/E/W
    neighbours, in multinomial(1/4 each) proportions; all ages advance."""
    X = Y = 5
    c = community(X, Y, [species()], disp=1.0)
    o = oracle.OracleSpace(c)
    n = 4000
    centre = 2 * X + 2
    o.set_deme(0, centre, *tagged(n, 32, 0xFFFFFFFF, [2] * 2000 + [1] * 1000 + [0] * 1000))
    st = o.step(1)[0][0]
    sizes = o.sizes()[0]
    expect = {centre - X: "N", centre + X: "S", centre + 1: "E", centre - 1: "W"}
    assert sizes.sum() == n and st["n_after"] == n and st["movers"] == n
    assert set(np.nonzero(sizes)[0]) == set(expect)
    counts = np.array([sizes[p] for p in expect])
    assert sps.chisquare(counts).pvalue > 1e-4
    for p in expect:
        rec, age = o.deme(0, p)
        assert np.all(rec == 0xFFFFFFFF) and np.all(age >= 1)
        assert np.all(np.diff(age.astype(int)) <= 0)


def test_torus_wraps_at_the_edges():
    X, Y = 4, 3
    c = community(X, Y, [species()], disp=1.0)
    o = oracle.OracleSpace(c)
    o.set_deme(0, 0, *tagged(2000, 32, 7, [2] * 2000))
    o.step(1)
    sizes = o.sizes()[0]
    assert set(np.nonzero(sizes)[0]) == {(Y - 1) * X, X, 1, X - 1}


def test_movers_are_binomial():
    c = community(6, 6, [species(n0=500)], disp=0.05)
    o = oracle.OracleSpace(c)
    st = o.step(1)[0][0]
    n = 36 * 500
    assert abs(st["movers"] - 0.05 * n) < 5 * math.sqrt(n * 0.05 * 0.95)
    assert st["n_after"] == n


def test_survival_probability_by_age_class():
    q = [0.3, 0.6, 0.9]
    tabs = np.stack([np.full(4096, int(x * 2 ** 32), np.uint32) for x in q])
    c = community(1, 1, [species(tables=tabs)])
    o = oracle.OracleSpace(c)
    n_age = [6000, 5000, 4000]
    ages = [2] * n_age[2] + [1] * n_age[1] + [0] * n_age[0]
    o.set_deme(0, 0, *tagged(len(ages), 32, 0, ages))
    o.step(1)
    _, age = o.deme(0, 0)
    now2, now1 = int((age == 2).sum()), int((age == 1).sum())
    # age-1 and age-2 survivors become adults, age-0 survivors become age 1
    m1 = n_age[1] * q[1] + n_age[2] * q[2]
    v1 = n_age[1] * q[1] * (1 - q[1]) + n_age[2] * q[2] * (1 - q[2])
    assert abs(now2 - m1) < 5 * math.sqrt(v1)
    assert abs(now1 - n_age[0] * q[0]) < 5 * math.sqrt(n_age[0] * q[0] * (1 - q[0]))
    assert int((age == 0).sum()) == 0


def test_interaction_factor_scales_survival():
    """Certain viability times the factor D / (D + A n): survival probability
    is D / (D + A n) for n individuals of the species in the patch."""
    n, D, A = 8000, 4000, 2
    c = community(1, 1, [species(D=D, A=(A, 0, 0))])
    o = oracle.OracleSpace(c)
    o.set_deme(0, 0, *tagged(n, 32, 0, [2] * n))
    st = o.step(1)[0][0]
    p = D / (D + A * n)
    assert abs(st["survivors"] - n * p) < 5 * math.sqrt(n * p * (1 - p))


def test_recruitment_rule_counts():
    """Births = min(bmax, floor(m * beta * g / 2^48)), g = floor(2^32 num / den),
    num = G + sum P n, den = num + E + sum C n, for two interacting species."""
    sp0 = species(G=300, P=(0, 2, 0), E=50, C=(1, 3, 0), beta=int(1.7 * 65536), bmax=100000)
    sp1 = species(G=10, P=(1, 0, 0), E=0, C=(0, 1, 0), beta=int(0.6 * 65536), bmax=250)
    c = community(1, 1, [sp0, sp1])
    o = oracle.OracleSpace(c)
    a0 = [2] * 700 + [1] * 300 + [0] * 200
    a1 = [2] * 900 + [0] * 100
    o.set_deme(0, 0, *tagged(len(a0), 32, 0, a0))
    o.set_deme(1, 0, *tagged(len(a1), 32, 0, a1))
    st = o.step(1)[0]
    n = [len(a0), len(a1)]
    for k, sp, m in ((0, sp0, 700), (1, sp1, 900)):
        num = sp.G + sum(pk * nk for pk, nk in zip(sp.P, n))
        den = num + sp.E + sum(ck * nk for ck, nk in zip(sp.C, n))
        g = (num << 32) // den
        expect = min(sp.bmax, (m * sp.beta_q16 * g) >> 48)
        assert st[k]["births"] == expect, (k, st[k]["births"], expect)


def test_newborns_inherit_from_adults_only_in_mendelian_proportions():
    """Adults heterozygous at every locus (hap0 = 0, hap1 = 1), juveniles all-1,
    no mutation: newborn genotype classes follow 1:2:1 at every locus and no
    newborn carries a juvenile-only haplotype pattern beyond that."""
    L, n_ad = 32, 3000
    sp = species(L=L, G=1, beta=int(2.0 * 65536), bmax=20000)
    c = community(1, 1, [sp])
    o = oracle.OracleSpace(c)
    rec = np.zeros((n_ad + 500, 2), np.uint32)
    rec[:n_ad, 1] = 0xFFFFFFFF
    rec[n_ad:, :] = 0xFFFFFFFF
    age = np.array([2] * n_ad + [1] * 500, np.uint8)
    o.set_deme(0, 0, rec, age)
    st = o.step(1)[0][0]
    B = int(st["births"])
    assert B > 5000
    r, a = o.deme(0, 0)
    newborn = r[a == 0]
    assert len(newborn) == B
    bits = (newborn[:, :, None].astype(np.uint64) >> np.arange(32, dtype=np.uint64)) & 1
    copies = bits.sum(axis=1)  # [B, 32]
    chi2 = 0.0
    for l in range(L):
        obs = np.bincount(copies[:, l].astype(int), minlength=3)
        exp = B * np.array([0.25, 0.5, 0.25])
        chi2 += ((obs - exp) ** 2 / exp).sum()
    assert sps.chi2.sf(chi2, 2 * L) > 1e-4
    # juveniles (all-1 on both haplotypes) never parent: a newborn with both
    # haplotypes all-1 at every locus would have probability 4^-32 from adults
    assert not np.any((newborn[:, 0] == 0xFFFFFFFF) & (newborn[:, 1] == 0xFFFFFFFF))


def test_layout_is_adults_first_and_stable_without_moves():
    """No dispersal, certain survival, no births: each deme keeps its members
    in their previous order with ages advanced; ages stay sorted."""
    c = community(3, 2, [species(n0=300, p0=0x40000000), species(n0=200)])
    o = oracle.OracleSpace(c)
    before = {(s, p): o.deme(s, p) for s in range(2) for p in range(6)}
    st = o.step(1)[0]
    assert all(int(x["n_after"]) == int(x["n_before"]) for x in st)
    for (s, p), (rec0, age0) in before.items():
        rec1, age1 = o.deme(s, p)
        assert np.array_equal(rec0, rec1)
        assert np.array_equal(age1, np.minimum(age0.astype(int) + 1, 2))


def test_community_runs_and_layout_invariants_hold():
    c = S.spatial_community(X=4, Y=4, n0=200, n_loci=64, mu=1e-3)
    o = oracle.OracleSpace(c)
    for st in o.step(8):
        for x in st:
            assert x["n_after"] == x["survivors"] + x["births"]
            assert x["survivors"] <= x["n_before"]
    for s in range(3):
        for p in range(16):
            _, age = o.deme(s, p)
            assert np.all(np.diff(age.astype(int)) <= 0)
