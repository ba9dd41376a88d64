"""Pins for the CPU oracle: each test checks it against something the paper or
the mathematics fixes, never against a retyped copy of its own code.

Model facts used (paper, Supplementary S2 "Genetics" and Fig. 1):
  * free recombination among all loci and gametes carrying half the parent's
    alleles  -> Hardy-Weinberg proportions after one generation of random
    mating, linkage disequilibrium halving every generation;
  * per-locus mutation with probability mu -> Binomial mutation counts, the
    two-way mutation expectation 1/2 (1 - (1 - 2 mu)^t);
  * random mating in a finite population -> Wright-Fisher drift, expected
    heterozygosity decaying by (1 - 1/2N) per generation;
  * survival against the selective environment, removal of the dead and
    environment update from the survivors (Fig. 1 D-F) -> exact Markov chain
    of a one-locus viability-selection model, per-bin survival frequencies,
    the fixed point of the resource's deterministic skeleton.
"""
import json
import math
import os
import subprocess
import sys
from collections import defaultdict

import numpy as np
import pytest
from scipy import stats as sps

import oracle
import spegg_synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def unpack(g: np.ndarray, n_loci: int) -> np.ndarray:
    """Packed records uint32[n, 2W] -> alleles int64[n, 2, L]."""
    n = g.shape[0]
    w = n_loci // 32
    words = g.reshape(n, 2, w).astype(np.uint64)
    bits = (words[..., None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)
    return bits.reshape(n, 2, n_loci).astype(np.int64)


def neutral_pop(n, n_loci, seed=0, rep=0, mu=0.0, init=None, p0_q32=0x80000000, effects=None):
    e = np.zeros(n_loci, np.int16) if effects is None else effects
    bias, shift = S.bin_map(e)
    return oracle.OraclePopulation(n, n_loci, seed, rep, e, S.constant_table(S.CERTAIN), bias, shift,
                                   mu, init, p0_q32)


# --------------------------------------------------------------------------
# Philox4x32-10 against an independent library implementation
# --------------------------------------------------------------------------
_TRITON_PHILOX = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
cases = json.loads(sys.stdin.read())
@triton.jit
def k(c_ptr, out_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c_ptr + i * 4 + 0); c1 = tl.load(c_ptr + i * 4 + 1)
    c2 = tl.load(c_ptr + i * 4 + 2); c3 = tl.load(c_ptr + i * 4 + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + i * 4 + 0, a); tl.store(out_ptr + i * 4 + 1, b)
    tl.store(out_ptr + i * 4 + 2, c); tl.store(out_ptr + i * 4 + 3, d)
res = []
for seed, ctrs in cases:
    c = torch.tensor([[x - (1 << 32) if x >= (1 << 31) else x for x in row] for row in ctrs], dtype=torch.int32)
    out = torch.zeros_like(c)
    k[(1,)](c, out, seed, N=c.shape[0])
    res.append([[v & 0xFFFFFFFF for v in row] for row in out.tolist()])
print(json.dumps(res))
"""


def test_philox_matches_independent_library():
    """Philox4x32-10 (Salmon et al., SC'11) vs Triton's implementation of the
    same published generator (run in its CPU interpreter)."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(99)
    cases = []
    for seed in [0, 1, 0xFFFFFFFFFFFFFFFF, 0x299F31D0A4093822, int(rng.integers(0, 2 ** 63))]:
        ctrs = [[0, 0, 0, 0], [0xFFFFFFFF] * 4] + rng.integers(0, 2 ** 32, size=(14, 4)).tolist()
        cases.append([seed, ctrs])
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _TRITON_PHILOX], input=json.dumps(cases), env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lib_out = json.loads(r.stdout.strip().splitlines()[-1])
    for (seed, ctrs), expect in zip(cases, lib_out):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for ctr, e in zip(ctrs, expect):
            assert list(oracle.philox4x32_10(ctr, key)) == e, (seed, ctr)


def test_philox_lanes_are_uniform():
    """Each output lane is uniform on [0, 2^32): top-byte histogram of 64k draws."""
    out = np.array([oracle.philox4x32_10([i, 7, 3, 2 << 24], [5, 9]) for i in range(16384)])
    for lane in range(4):
        hist = np.bincount(out[:, lane] >> 24, minlength=256)
        assert sps.chisquare(hist).pvalue > 1e-4


# --------------------------------------------------------------------------
# mutation-count distribution
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mu,n", [(1e-4, 64), (1e-5, 256), (1e-5, 512), (1e-3, 128), (0.05, 64), (0.2, 64)])
def test_mutation_cdf_is_binomial(mu, n):
    cdf = oracle.mutation_cdf(mu, n)
    k = np.arange(len(cdf))
    exact = sps.binom.cdf(k, n, mu) * 4294967296.0
    assert np.all(np.abs(cdf.astype(np.float64) - np.floor(exact)) <= 2.0)
    assert np.all(np.diff(cdf.astype(np.int64)) >= 0)
    # counts above len(cdf) are capped; the table stops where that tail,
    # P(K > len(cdf)), is below 2^-32 (or at 32 entries)
    if len(cdf) < 32:
        assert sps.binom.sf(len(cdf), n, mu) < 2.0 ** -31


def test_mutation_cdf_zero_rate():
    assert len(oracle.mutation_cdf(0.0, 64)) == 0


# --------------------------------------------------------------------------
# genotype -> phenotype map (brute force)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n_loci", [32, 64, 128, 256])
def test_phenotype_brute_force(n_loci):
    rng = np.random.default_rng(n_loci)
    e = rng.integers(-32768, 32768, size=n_loci).astype(np.int16) // 64
    recs = rng.integers(0, 2 ** 32, size=(50, 2 * (n_loci // 32)), dtype=np.uint64).astype(np.uint32)
    bits = unpack(recs, n_loci)
    expect = (bits.sum(axis=1) * e.astype(np.int64)[None, :]).sum(axis=1)
    got = [oracle.phenotype(e, r) for r in recs]
    assert got == expect.tolist()


@pytest.mark.parametrize("n_loci", [32, 128, 256])
def test_statistics_match_genotypes(n_loci):
    """Every integer statistic of a generation recomputed with numpy from the
    offspring genotypes and survivor list the oracle returns."""
    w = S.consumer_resource(n=3000, n_loci=n_loci, n_gen=3, mu=1e-3, s=2.0, K=2e5)
    p = oracle.OraclePopulation.from_workload(w)
    st = p.step(3)[-1]
    g = p.genotypes()
    surv = p.survivors()
    bits = unpack(g, n_loci)
    raw = (bits.sum(axis=1) * w.effects.astype(np.int64)[None, :]).sum(axis=1)
    v = raw + w.bias
    bins = np.where(v < 0, 0, np.minimum(v >> w.shift, 4095))
    assert st["n"] == w.n and st["s"] == len(surv)
    assert st["sum_raw"] == raw.sum() and st["sum_raw2"] == (raw * raw).sum()
    assert st["min_raw"] == raw.min() and st["max_raw"] == raw.max()
    assert st["sum_raw_surv"] == raw[surv].sum()
    assert st["het"] == (bits[:, 0] != bits[:, 1]).sum()
    assert st["allele"] == bits.sum()
    assert st["consumption"] == w.attack[bins[surv]].astype(np.uint64).sum()
    # FP32 summaries within 1e-6 relative of float64 numpy values
    summ = oracle.summarize(np.array([st]), n_loci)[0]
    z = raw / 512.0
    ref = [z.mean(), z.var(), len(surv) / w.n, (bits[:, 0] != bits[:, 1]).mean(), bits.mean()]
    for a, b in zip(summ, ref):
        assert abs(float(a) - b) <= 1e-6 * max(abs(b), 1e-30) + 1e-12


# --------------------------------------------------------------------------
# survivors, counts, extremes
# --------------------------------------------------------------------------
def test_survivor_list_is_ordered_and_conserved():
    w = S.single_species(n=5000, n_loci=64, n_gen=5, s=3.0)
    p = oracle.OraclePopulation.from_workload(w)
    for st in p.step(5):
        assert st["n"] == 5000
    surv = p.survivors()
    assert len(surv) == p.state()["S"] == st["s"]
    assert np.all(np.diff(surv.astype(np.int64)) > 0) and surv[-1] < 5000


def test_all_zero_table_goes_extinct_in_one_generation():
    e = S.effects_q8(32)
    bias, shift = S.bin_map(e)
    p = oracle.OraclePopulation(100, 32, 0, 0, e, S.constant_table(0), bias, shift, 1e-4)
    st = p.step(5)
    assert len(st) == 1 and st[0]["s"] == 0 and st[0]["status"] == oracle.EXTINCT
    assert p.state()["status"] == oracle.EXTINCT and len(p.step(3)) == 0


def test_certain_table_keeps_everyone():
    p = neutral_pop(777, 64, mu=1e-3)
    st = p.step(10)
    assert np.all(st["s"] == 777)


def test_survival_frequency_per_bin():
    """Empirical survival in each phenotype bin equals table[bin] / 2^32."""
    L = 32
    e = np.zeros(L, np.int16)
    e[:4] = [1, 2, 4, 8]  # raw = 2*(sum of copies*effect): bins spread over 0..30
    bias, shift = S.bin_map(e)
    table = S.constant_table(0)
    levels = np.linspace(0.05, 0.95, 31)
    for b in range(31):
        table[b] = int(levels[b] * 2 ** 32)
    n = 40000
    p = oracle.OraclePopulation(n, L, 3, 0, e, table, bias, shift, 0.0, None, 0x80000000)
    p.step(1)
    g = p.genotypes()
    alive = np.zeros(n, bool)
    alive[p.survivors()] = True
    bits = unpack(g, L)
    raw = (bits.sum(axis=1) * e.astype(np.int64)).sum(axis=1)
    bins = raw + bias
    chi2 = 0.0
    dof = 0
    for b in np.unique(bins):
        m = bins == b
        k, cnt, pr = alive[m].sum(), m.sum(), table[b] / 2 ** 32
        chi2 += (k - cnt * pr) ** 2 / (cnt * pr * (1 - pr))
        dof += 1
    assert sps.chi2.sf(chi2, dof) > 1e-4


# --------------------------------------------------------------------------
# transmission: Hardy-Weinberg, linkage equilibrium, initial frequencies
# --------------------------------------------------------------------------
def test_hardy_weinberg_after_one_generation():
    """All parents heterozygous at every locus: offspring genotype classes
    0/1/2 copies occur in proportions 1/4, 1/2, 1/4 at every locus."""
    n, L = 20000, 64
    init = S.genotypes_uniform(n, L, 0x00000000, 0xFFFFFFFF)
    p = neutral_pop(n, L, seed=11, init=init)
    p.step(1)
    copies = unpack(p.genotypes(), L).sum(axis=1)  # [n, L]
    chi2 = 0.0
    for l in range(L):
        obs = np.bincount(copies[:, l], minlength=3)
        exp = n * np.array([0.25, 0.5, 0.25])
        chi2 += ((obs - exp) ** 2 / exp).sum()
    pv = sps.chi2.sf(chi2, 2 * L)
    assert 1e-4 < pv < 1 - 1e-4
    # and no association between loci (linkage equilibrium in the offspring)
    c = np.corrcoef(copies.T.astype(np.float64))
    off = c[~np.eye(L, dtype=bool)]
    assert np.abs(off).max() < 5.0 / math.sqrt(n) * 1.5


def test_linkage_disequilibrium_halves_each_generation():
    """Free recombination (r = 1/2): D_t = D_0 / 2^t.  Start from haplotypes
    that are all-0 or all-1 (p = 1/2, D_0 = 1/4 for every pair of loci)."""
    n, L = 40000, 64
    init = S.genotypes_random_haplotype_pairs(n, L, seed=5)
    p = neutral_pop(n, L, seed=21, init=init)
    for t in range(1, 6):
        p.step(1)
        hap = unpack(p.genotypes(), L).reshape(2 * n, L).astype(np.float64)
        pf = hap.mean(axis=0)
        pair = (hap.T @ hap) / (2 * n)
        D = pair - np.outer(pf, pf)
        off = D[~np.eye(L, dtype=bool)]
        within = D[:32, :32][~np.eye(32, dtype=bool)].mean()  # same 32-bit word
        across = D[:32, 32:].mean()                              # different words
        expect = 0.25 / 2 ** t
        for val in (off.mean(), within, across):
            assert abs(val - expect) < 0.003, (t, val, expect)


def test_initial_allele_frequency_and_hwe():
    n, L = 20000, 32
    for p0 in (0.0, 0.1, 0.5):
        p = neutral_pop(n, L, seed=4, p0_q32=S.p0_threshold(p0))
        bits = unpack(p.genotypes(), L)
        freq = bits.mean()
        assert abs(freq - p0) < 5 * math.sqrt(max(p0 * (1 - p0), 1e-12) / (2 * n * L)) + 1e-12
        if p0 == 0.0:
            assert bits.sum() == 0
        if p0 == 0.5:
            copies = bits.sum(axis=1).ravel()
            obs = np.bincount(copies, minlength=3)
            assert sps.chisquare(obs, len(copies) * np.array([0.25, 0.5, 0.25])).pvalue > 1e-4


# --------------------------------------------------------------------------
# mutation
# --------------------------------------------------------------------------
def test_mutation_counts_are_binomial_and_uniform_over_positions():
    n, L, mu = 20000, 64, 1e-3
    init = S.genotypes_uniform(n, L, 0, 0)
    p = neutral_pop(n, L, seed=8, mu=mu, init=init)
    p.step(1)
    bits = unpack(p.genotypes(), L)  # every 1 is a mutation
    total = bits.sum()
    mean, sd = 2 * n * L * mu, math.sqrt(2 * n * L * mu * (1 - mu))
    assert abs(total - mean) < 5 * sd
    per_pos = bits.sum(axis=0).ravel()  # 2L positions
    assert sps.chisquare(per_pos).pvalue > 1e-4
    # mutations within one genome are at distinct positions: at most one flip per copy
    assert bits.max() <= 1


def test_two_way_mutation_expectation():
    """E[p_t] = 1/2 (1 - (1 - 2 mu)^t) from p_0 = 0 under neutrality."""
    n, L, mu, t = 5000, 64, 0.01, 20
    p = neutral_pop(n, L, seed=9, mu=mu, init=S.genotypes_uniform(n, L, 0, 0))
    p.step(t)
    freq = unpack(p.genotypes(), L).mean()
    expect = 0.5 * (1 - (1 - 2 * mu) ** t)
    assert abs(freq - expect) < 0.012, (freq, expect)


# --------------------------------------------------------------------------
# drift
# --------------------------------------------------------------------------
@pytest.mark.slow
def test_neutral_heterozygosity_decay():
    """Wright-Fisher with 2N gene copies: E[H_t] = H_0 (1 - 1/2N)^t, H = 2p(1-p)."""
    n, L, reps, checkpoints = 50, 32, 300, [10, 20, 40, 60]
    H = np.zeros((reps, len(checkpoints) + 1))
    for r in range(reps):
        p = neutral_pop(n, L, seed=1234, rep=r)
        def het():
            f = unpack(p.genotypes(), L).reshape(2 * n, L).mean(axis=0)
            return (2 * f * (1 - f)).mean()
        H[r, 0] = het()
        prev = 0
        for i, t in enumerate(checkpoints):
            p.step(t - prev)
            prev = t
            H[r, i + 1] = het()
    for i, t in enumerate(checkpoints):
        ratio = H[:, i + 1].mean() / H[:, 0].mean()
        se = H[:, i + 1].std(ddof=1) / math.sqrt(reps) / H[:, 0].mean()
        expect = (1 - 1 / (2 * n)) ** t
        assert abs(ratio - expect) < 4.5 * se, (t, ratio, expect, se)


# --------------------------------------------------------------------------
# selection + mutation + drift: exact Markov chain on a tiny population
# --------------------------------------------------------------------------
def _chain(N, t, mu, w, start):
    """Distribution of the survivors' genotype counts (s0, s1, s2) at one
    locus after t generations, from theory: each offspring allele is a random
    allele of a random survivor, flipped with probability mu; offspring with c
    copies survive with probability w[c]."""
    states = [(a, b, c) for a in range(N + 1) for b in range(N + 1 - a) for c in range(N + 1 - a - b)]
    dist = {start: 1.0}
    for _ in range(t):
        new = defaultdict(float)
        for (s0, s1, s2), pr in dist.items():
            Ss = s0 + s1 + s2
            if Ss == 0:
                new[(0, 0, 0)] += pr
                continue
            q = (0.5 * s1 + s2) / Ss
            qm = q * (1 - mu) + (1 - q) * mu
            pi = [(1 - qm) ** 2, 2 * qm * (1 - qm), qm ** 2]
            ps = [pi[c] * w[c] for c in range(3)]
            pdead = 1.0 - sum(ps)
            for (n0, n1, n2) in states:
                k = n0 + n1 + n2
                coef = math.factorial(N) / (math.factorial(n0) * math.factorial(n1) * math.factorial(n2)
                                            * math.factorial(N - k))
                new[(n0, n1, n2)] += pr * coef * ps[0] ** n0 * ps[1] ** n1 * ps[2] ** n2 * pdead ** (N - k)
        dist = new
    return dist


@pytest.mark.parametrize("N,t,mu,wv", [(4, 3, 0.05, (1.0, 0.7, 0.3)), (3, 4, 0.02, (0.9, 1.0, 0.5))])
def test_selection_mutation_drift_markov_chain(N, t, mu, wv):
    L = 32
    e = np.zeros(L, np.int16)
    e[0] = 256
    bias, shift = S.bin_map(e)
    table = S.genotype_table(bias, shift, e, list(wv))
    w_exact = [1.0 if table[c * 256 + bias] == S.CERTAIN else table[c * 256 + bias] / 2 ** 32 for c in range(3)]
    init = S.genotypes_uniform(N, L, 0x0, 0x1)  # heterozygous at locus 0
    reps = 20000
    counts = defaultdict(int)
    for r in range(reps):
        p = oracle.OraclePopulation(N, L, 77, r, e, table, bias, shift, mu, init)
        p.step(t)
        g = p.genotypes()
        surv = p.survivors()
        c = (g[surv, 0] & 1) + (g[surv, 1] & 1)
        counts[(int((c == 0).sum()), int((c == 1).sum()), int((c == 2).sum()))] += 1
    dist = _chain(N, t, mu, w_exact, (0, N, 0))
    keys = sorted(set(dist) | set(counts))
    exp = np.array([dist.get(k, 0.0) * reps for k in keys])
    obs = np.array([counts.get(k, 0) for k in keys], dtype=np.float64)
    assert obs[exp == 0].sum() == 0
    big = exp >= 5
    e_b = np.append(exp[big], exp[~big].sum())
    o_b = np.append(obs[big], obs[~big].sum())
    if e_b[-1] == 0:
        e_b, o_b = e_b[:-1], o_b[:-1]
    chi2 = ((o_b - e_b) ** 2 / e_b).sum()
    assert sps.chi2.sf(chi2, len(e_b) - 1) > 1e-4


# --------------------------------------------------------------------------
# ecology
# --------------------------------------------------------------------------
def test_resource_without_consumption_tends_to_carrying_capacity():
    w = S.single_species(n=500, n_loci=32, s=0.0)
    p = oracle.OraclePopulation.from_workload(w)
    K = 1e6
    p.set_ecology(0.5, K, K / 2, K / 10, S.constant_table(0))
    st = p.step(60)
    R = st["R"]
    assert np.all(np.diff(R) >= 0) and np.all(R <= K)
    assert R[0] == 0.625 * K  # K/2 + r * K/2 * (1 - 1/2): exact in binary
    assert abs(R[-1] - K) < 1e-6 * K
    assert np.all(st["consumption"] == 0)


def test_resource_fixed_point_under_trait_independent_harvest():
    """Constant attack rate a, certain viability: survival probability is the
    resource factor f(R) = R/(R+R_h), so the deterministic skeleton is
    R' = R + rR(1-R/K) - a N f(R); the simulated R settles at its stable
    fixed point r(1-R/K)(R+R_h) = a N."""
    n, K, r, Rh, a = 20000, 1e6, 0.5, 1e5, 4.0
    p = neutral_pop(n, 32, seed=3)
    p.set_ecology(r, K, K / 2, Rh, S.constant_table(int(a * 65536)))
    st = p.step(300)
    assert np.all(st["consumption"] == st["s"].astype(np.uint64) * np.uint64(a * 65536))
    # r(1 - x)(xK + Rh) = aN  ->  -rK x^2 + r(K - Rh) x + r Rh - aN = 0
    roots = np.roots([-r * K, r * (K - Rh), r * Rh - a * n])
    xstar = roots.real.max()
    Rbar = st["R"][100:].mean()
    assert abs(Rbar / (xstar * K) - 1) < 2e-3, (Rbar, xstar * K)
    fbar = st["f"][100:].mean() / 2 ** 32
    assert abs(fbar - xstar * K / (xstar * K + Rh)) < 1e-3


def test_resource_collapse_drives_extinction():
    p = neutral_pop(1000, 32)
    p.set_ecology(0.5, 1e5, 5e4, 1e4, S.constant_table(2 ** 30))
    st = p.step(10)
    assert st[-1]["status"] == oracle.EXTINCT and st[-1]["s"] == 0
    assert 0.0 in st["R"]


# --------------------------------------------------------------------------
# determinism of the counter-based draws
# --------------------------------------------------------------------------
def test_same_inputs_same_run_and_replicates_differ():
    w = S.single_species(n=2000, n_loci=64, n_gen=5, mu=1e-3)
    a = oracle.OraclePopulation.from_workload(w).step(5)
    b = oracle.OraclePopulation.from_workload(w).step(5)
    assert a.tobytes() == b.tobytes()
    w.replicate = 1
    c = oracle.OraclePopulation.from_workload(w).step(5)
    assert a.tobytes() != c.tobytes()


def test_selfing_single_parent_transmits_only_its_alleles():
    """N = 1, no mutation: every offspring allele is one of the parent's two
    alleles at that locus (homozygous loci are transmitted unchanged)."""
    L = 64
    init = S.genotypes_bernoulli(1, L, 0.5, seed=2)
    p = neutral_pop(1, L, init=init)
    par = unpack(init, L)[0]
    for _ in range(1):
        p.step(1)
        kid = unpack(p.genotypes(), L)[0]
        for l in range(L):
            for h in range(2):
                assert kid[h, l] in (par[0, l], par[1, l])
