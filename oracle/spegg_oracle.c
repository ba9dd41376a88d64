/*
 * CPU oracle for the sPEGG per-generation update -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, obviously-correct statement of what one
 * generation of the forward-time simulation computes.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the product
 * library never does, and the two share no code, headers or tables.
 *
 * What it follows (paper sections):
 *   - Fig. 1 / Main text: each step identifies parents, transmits genetic
 *     information by recombination and mutation, maps genotype to phenotype,
 *     updates survival against the selective environment, removes the dead,
 *     and updates the environment from the survivors.
 *   - S2 "Genetics": diploid, sexual, free recombination among all loci;
 *     each gamete carries half of the parent's alleles; each locus mutates
 *     with probability mu; the genetic value is the sum over loci of the
 *     midpoint of the two gametes' allelic values (eq. S2-phenval).
 *   - S2 "Resource Consumption": resource density updated from the
 *     consumers' total consumption (here a logistic resource).
 *   - Fig. S5(B): every individual updated independently from its own index.
 *
 * Deliberate readings (the paper is silent or uses a continuous model):
 *   - alleles are biallelic (0/1) with effect e_l (Q8 int16) for allele 1;
 *     the integer phenotype raw = sum_l e_l * (a0_l + a1_l); the midpoint 1/2
 *     and the Q8 scale are folded into the trait z = raw / 512;
 *   - Wright-Fisher: N offspring per generation, each parent drawn uniformly
 *     (with replacement, selfing allowed) from the previous survivors;
 *   - survival: the phenotype bin indexes a caller-built uint32 threshold table
 *     (0xFFFFFFFF = certain), optionally scaled by a Q32 resource factor;
 *   - every random number is one lane of Philox4x32-10 (Salmon et al., SC'11,
 *     "Parallel random numbers: as easy as 1, 2, 3") at a counter that names
 *     (individual, generation, replicate, purpose, sub-index);
 *   - linkage maps (the "variable linkage maps" / "arbitrary linkage
 *     patterns" of the Main text; optional, free recombination otherwise):
 *     loci lie on chromosomes in record order; between adjacent loci of one
 *     chromosome the map gives a distance d_l in Morgans; crossovers follow
 *     Haldane's no-interference model, realised as K ~ Binomial(2^16, D/2^16)
 *     crossovers per gamete (D = total map length) each falling in interval l
 *     with probability d_l / D; a locus takes the haplotype given by its
 *     chromosome's fair coin, flipped once per crossover in the intervals from
 *     the chromosome's first locus up to it;
 *   - weighted parents (S2 "Reproduction": the chance that an individual
 *     parents an egg grows with its size relative to the others; optional,
 *     uniform otherwise): caller weight tables over the phenotype bins, one
 *     for mothers and one for fathers, applied to each survivor's bin at
 *     birth; each parent is drawn by bounded rejection sampling: a uniform
 *     survivor r is proposed and accepted with probability w(bin_r) / w_max,
 *     at most 64 proposals, the last one taken if all are rejected;
 *   - dominance (the non-additive genotype-phenotype maps of the Main text;
 *     optional): a heterozygous locus l adds its dominance deviation d_l
 *     (Q8 int16) to the genetic value, raw = sum_l e_l (a0 + a1) + sum_l d_l
 *     [a0 != a1];
 *   - Beverton-Holt resource (S2 "Resource Consumption", optional instead of
 *     the logistic): R' = r' R / (1 + R/K) - C 2^-16, clamped at 0, with the
 *     growth rate r' = r + r_sd z drawn every generation; the paper draws it
 *     from a normal distribution, read here as the Irwin-Hall(12) normal
 *     z = (u_1 + ... + u_12) 2^-32 - 6 (mean 0, variance 1, tails cut at
 *     6), whose integer sum keeps both implementations exact;
 *   - continuous allelic values (S2 "Genetics": allelic values vary
 *     continuously, a mutation redraws the value from a normal centred on the
 *     old one, the phenotype is normal around the genetic value; optional):
 *     every allele copy holds an int16 value in Q8 (the biallelic model's
 *     effect scale), raw = sum_l (v0_l + v1_l) plus an environmental
 *     deviation; a mutated copy adds floor(z * s) and an offspring's phenotype
 *     adds floor(z * s_env), z the Irwin-Hall(12) normal in exact integer
 *     arithmetic (see irwin_hall_step), values clamped to the int16 range.
 *
 * Genotypes are kept UNPACKED here (one byte per allele copy) so that the
 * per-locus statement of the model is visible; packing is done only when
 * reading inputs and writing outputs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_BINS 4096
#define ORC_MAX_KMAX 32
#define ORC_MUT_DRAWS 64
#define ORC_CERTAIN 0xFFFFFFFFu

#define ORC_MAX_LOCI 256
#define ORC_MAX_CHROM 96
#define ORC_LINK_SITES 65536u /* crossover opportunities per gamete */
#define ORC_MAX_MAP 16.0      /* Morgans, total map length */

#define ORC_MATE_ATTEMPTS 64

enum { ORC_INIT = 1, ORC_MATE = 2, ORC_RECOMB = 3, ORC_MUTPOS = 4, ORC_LINK = 5, ORC_MATEW = 6, ORC_GROWTH = 7,
       ORC_MUTSIZE = 8, ORC_ENV = 9 };
enum { ORC_OK = 0, ORC_EXTINCT = 1, ORC_ERR_INVALID = -1, ORC_ERR_OOM = -2 };

/* One record per generation; same field order as the library's statistics
 * record so the tests can compare them field by field. */
typedef struct {
    uint32_t gen, n, s, status;
    int64_t sum_raw;
    uint64_t sum_raw2;
    int64_t sum_raw_surv;
    int32_t min_raw, max_raw;
    uint64_t het;
    uint64_t allele;
    uint64_t consumption;
    double R;
    uint32_t f;
    uint32_t pad;
} orc_stats;

typedef struct {
    uint32_t n, L;
    uint64_t seed;
    uint32_t rep;
    int16_t *effects;
    uint32_t table[ORC_BINS];
    int32_t bias;
    uint32_t shift;
    double mu;
    uint32_t cdf[ORC_MAX_KMAX];
    uint32_t kmax;
    /* linkage map (linked == 0: free recombination) */
    int linked;
    uint32_t link_cdf[ORC_MAX_KMAX], link_kmax; /* crossovers per gamete */
    uint32_t link_cum[ORC_MAX_LOCI];            /* crossover interval CDF */
    uint32_t chrom_of[ORC_MAX_LOCI];            /* chromosome of each locus */
    uint32_t nchrom;
    /* weighted parents (weighted == 0: uniform) */
    int weighted;
    uint32_t acc_mother[ORC_BINS], acc_father[ORC_BINS]; /* acceptance thresholds, Q32 */
    uint16_t *bin_par, *bin_chi;                       /* phenotype bin of each individual at birth */
    int16_t *dominance;                                /* [L] dominance deviations, or NULL */
    /* continuous allelic values (continuous == 0: biallelic) */
    int continuous;
    int16_t *vpar, *vchi;  /* [n][2][L] allelic values, Q8 */
    int64_t s_mut, s_env;  /* Irwin-Hall scales, Q16 (raw units per standard deviation) */
    /* ecology */
    int has_eco;
    double r, K, R, R_half;
    int eco_model;   /* 0 logistic, 1 Beverton-Holt */
    double r_sd;     /* Beverton-Holt: standard deviation of the growth rate */
    uint32_t attack[ORC_BINS];
    uint32_t f;
    /* state */
    uint32_t gen, S;
    int status;
    uint8_t *par; /* [n][2][L] alleles of the current parents' generation */
    uint8_t *chi; /* [n][2][L] offspring being formed                      */
    uint32_t *surv, *surv_next;
} orc_pop;

static int32_t phenotype_unpacked(const int16_t *effects, uint32_t L, const uint8_t *hap0,
                                  const uint8_t *hap1);
static int32_t genetic_value(const orc_pop *p, const uint8_t *hap0, const uint8_t *hap1);
static uint32_t bin_of(const orc_pop *p, int32_t raw);

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition: 10 rounds of
 * (c0,c1,c2,c3) -> (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0))
 * with the key advanced by the Weyl constants between rounds.             */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The four uint32 lanes of Philox at counter
 * (individual, generation, replicate, purpose<<24 | sub). */
static void draw4(const orc_pop *p, uint32_t individual, uint32_t generation,
                  uint32_t purpose, uint32_t sub, uint32_t out[4])
{
    uint32_t ctr[4] = { individual, generation, p->rep, (purpose << 24) | sub };
    uint32_t key[2] = { (uint32_t)(p->seed & 0xFFFFFFFFu), (uint32_t)(p->seed >> 32) };
    orc_philox4x32_10(ctr, key, out);
}

/* Uniform index in [0, n) from one uint32: floor(u * n / 2^32). */
static uint32_t scaled_index(uint32_t u, uint32_t n)
{
    return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Per-locus mutation with probability mu (S2 "Genetics").  The number of
 * mutated allele copies in one offspring genome of n = 2L copies is
 * Binomial(n, mu); its CDF is tabulated in Q32 with plain IEEE-double basic
 * operations in a fixed order:
 *   P(0) = (1-mu)^n by n successive multiplications,
 *   P(k+1) = P(k) * (n-k) / (k+1) * mu / (1-mu),
 *   cdf[k] = floor(2^32 * sum_{i<=k} P(i)), stopping at the first entry
 *   >= 0xFFFFFFFF (or after 32 entries).
 * The mutation count is the number of entries <= u for one uniform u.      */
uint32_t orc_mutation_cdf(double mu, uint32_t n_copies, uint32_t *cdf_out)
{
    double q = 1.0 - mu;
    double term = 1.0;
    for (uint32_t i = 0; i < n_copies; ++i) term = term * q;
    double cum = 0.0;
    uint32_t kmax = 0;
    for (uint32_t k = 0; k <= n_copies && kmax < ORC_MAX_KMAX; ++k) {
        cum = cum + term;
        double scaled = cum * 4294967296.0;
        if (scaled >= 4294967295.0) break;
        cdf_out[kmax++] = (uint32_t)scaled; /* truncation == floor (scaled >= 0) */
        double a = term * (double)(n_copies - k);
        double b = a / (double)(k + 1);
        double c = b * mu;
        term = c / q;
    }
    return kmax;
}

/* ------------------------------------------------------------------------ */
/* Additive genotype -> phenotype map (Fig. 1C; eq. S2-phenval): a plain
 * per-locus sum over both allele copies. */
static int32_t phenotype_unpacked(const int16_t *effects, uint32_t L, const uint8_t *hap0,
                                  const uint8_t *hap1)
{
    int32_t raw = 0;
    for (uint32_t l = 0; l < L; ++l) raw += (int32_t)effects[l] * ((int32_t)hap0[l] + (int32_t)hap1[l]);
    return raw;
}

/* Genetic value of one individual: additive part plus, with dominance, the
 * deviation of every heterozygous locus. */
static int32_t genetic_value(const orc_pop *p, const uint8_t *hap0, const uint8_t *hap1)
{
    int32_t raw = phenotype_unpacked(p->effects, p->L, hap0, hap1);
    if (p->dominance)
        for (uint32_t l = 0; l < p->L; ++l)
            if (hap0[l] != hap1[l]) raw += (int32_t)p->dominance[l];
    return raw;
}

static uint32_t bin_of(const orc_pop *p, int32_t raw)
{
    int64_t v = (int64_t)raw + (int64_t)p->bias;
    if (v < 0) return 0;
    int64_t b = v >> p->shift;
    return b > (ORC_BINS - 1) ? (ORC_BINS - 1) : (uint32_t)b;
}

static uint8_t get_bit(const uint32_t *words, uint32_t pos)
{
    return (uint8_t)((words[pos / 32] >> (pos % 32)) & 1u);
}

/* Public helper for the tests: phenotype of one packed record. */
int32_t orc_phenotype_packed(const int16_t *effects, uint32_t L, const uint32_t *record)
{
    uint32_t W = L / 32;
    int32_t raw = 0;
    for (uint32_t l = 0; l < L; ++l)
        raw += (int32_t)effects[l] * ((int32_t)get_bit(record, l) + (int32_t)get_bit(record + W, l));
    return raw;
}

/* ------------------------------------------------------------------------ */
void orc_destroy(orc_pop *p)
{
    if (!p) return;
    free(p->effects); free(p->par); free(p->chi); free(p->surv); free(p->surv_next);
    free(p->bin_par);
    free(p->bin_chi);
    free(p->dominance);
    free(p->vpar);
    free(p->vchi);
    free(p);
}

/* Generation 0 (the initial population, Fig. S4 Initialize()): either the
 * caller's packed genotypes or, per allele copy, allele 1 iff u < p0_q32 with
 * u = lane (q mod 4) of Philox(i, 0, rep, INIT<<24 | q/4), q = h*L + l.     */
orc_pop *orc_create(uint32_t n, uint32_t L, uint64_t seed, uint32_t replicate,
                    const int16_t *effects, const uint32_t *init_genotypes, uint32_t p0_q32,
                    const uint32_t *surv_table, int32_t bias, uint32_t shift, double mu)
{
    if (n == 0 || L == 0 || (L % 32) != 0 || !effects || !surv_table || shift > 31) return NULL;
    if (!(mu >= 0.0 && mu < 1.0)) return NULL;
    orc_pop *p = (orc_pop *)calloc(1, sizeof(orc_pop));
    if (!p) return NULL;
    p->n = n; p->L = L; p->seed = seed; p->rep = replicate;
    p->effects = (int16_t *)malloc(sizeof(int16_t) * L);
    p->par = (uint8_t *)malloc((size_t)n * 2 * L);
    p->chi = (uint8_t *)malloc((size_t)n * 2 * L);
    p->surv = (uint32_t *)malloc(sizeof(uint32_t) * n);
    p->surv_next = (uint32_t *)malloc(sizeof(uint32_t) * n);
    p->bin_par = (uint16_t *)malloc(sizeof(uint16_t) * n);
    p->bin_chi = (uint16_t *)malloc(sizeof(uint16_t) * n);
    if (!p->effects || !p->par || !p->chi || !p->surv || !p->surv_next || !p->bin_par || !p->bin_chi) {
        orc_destroy(p);
        return NULL;
    }
    memcpy(p->effects, effects, sizeof(int16_t) * L);
    memcpy(p->table, surv_table, sizeof(uint32_t) * ORC_BINS);
    p->bias = bias; p->shift = shift; p->mu = mu;
    p->kmax = orc_mutation_cdf(mu, 2 * L, p->cdf);
    p->has_eco = 0; p->f = ORC_CERTAIN; p->R = 0.0;
    p->gen = 0; p->status = ORC_OK;

    uint32_t W = L / 32;
    for (uint32_t i = 0; i < n; ++i) {
        for (uint32_t h = 0; h < 2; ++h) {
            for (uint32_t l = 0; l < L; ++l) {
                uint8_t a;
                if (init_genotypes) {
                    const uint32_t *rec = init_genotypes + (size_t)i * 2 * W;
                    a = get_bit(rec + h * W, l);
                } else {
                    uint32_t q = h * L + l, d[4];
                    draw4(p, i, 0, ORC_INIT, q / 4, d);
                    a = d[q % 4] < p0_q32 ? 1 : 0;
                }
                p->par[((size_t)i * 2 + h) * L + l] = a;
            }
        }
        p->surv[i] = i; /* every founder is a potential parent */
        const uint8_t *h = p->par + (size_t)i * 2 * L;
        p->bin_par[i] = (uint16_t)bin_of(p, genetic_value(p, h, h + L));
    }
    p->S = n;
    return p;
}

/* Ecology (Fig. 1F): a logistic resource R consumed by the survivors.  The
 * survival factor applied to the next generation is f = R/(R + R_half) in
 * Q32 (capped at 0xFFFFFFFE so it never reads as "certain"). */
static uint32_t factor_q32(double R, double R_half)
{
    double den = R + R_half;
    double q = R / den;
    double scaled = q * 4294967296.0;
    if (scaled >= 4294967294.0) return 0xFFFFFFFEu;
    if (!(scaled > 0.0)) return 0u;
    return (uint32_t)scaled;
}

int orc_set_ecology(orc_pop *p, double r, double K, double R0, double R_half, const uint32_t *attack)
{
    if (!p || !attack || !(K > 0.0) || !(R_half > 0.0) || !(R0 >= 0.0)) return ORC_ERR_INVALID;
    p->has_eco = 1;
    p->eco_model = 0;
    p->r_sd = 0.0;
    p->r = r; p->K = K; p->R = R0; p->R_half = R_half;
    memcpy(p->attack, attack, sizeof(uint32_t) * ORC_BINS);
    p->f = factor_q32(R0, R_half);
    return ORC_OK;
}

/* Linkage map: map_morgans[l] (l >= 1) is the distance in Morgans between
 * loci l-1 and l, or negative where locus l starts a new chromosome
 * (map_morgans[0] is ignored: locus 0 starts chromosome 0).  Tables, in a
 * fixed order of IEEE-double basic operations:
 *   w_l = map_morgans[l] for linked intervals, else 0;  D = sum of w_l;
 *   crossover count: the Binomial(2^16, D / 2^16) CDF built like the
 *     mutation CDF;
 *   interval CDF: s = s + w_l, cum_l = floor(2^32 * (s / D)), saturated at
 *     0xFFFFFFFF (all zero when D = 0).
 * A crossover with uniform u lies in interval I = #{l <= L-2 : cum_l <= u}. */
int orc_set_linkage(orc_pop *p, const double *map_morgans)
{
    if (!p || !map_morgans || p->L > ORC_MAX_LOCI) return ORC_ERR_INVALID;
    const uint32_t L = p->L;
    double w[ORC_MAX_LOCI];
    double D = 0.0;
    uint32_t c = 0;
    p->chrom_of[0] = 0;
    w[0] = 0.0;
    for (uint32_t l = 1; l < L; ++l) {
        double m = map_morgans[l];
        if (m != m) return ORC_ERR_INVALID;
        if (m < 0.0) {
            c++;
            w[l] = 0.0;
        } else {
            w[l] = m;
        }
        p->chrom_of[l] = c;
        D = D + w[l];
    }
    if (c + 1 > ORC_MAX_CHROM || !(D <= ORC_MAX_MAP)) return ORC_ERR_INVALID;
    p->nchrom = c + 1;
    p->link_kmax = orc_mutation_cdf(D / (double)ORC_LINK_SITES, ORC_LINK_SITES, p->link_cdf);
    double run = 0.0;
    for (uint32_t l = 0; l < L; ++l) {
        if (D > 0.0) {
            run = run + w[l];
            double x = (run / D) * 4294967296.0;
            p->link_cum[l] = x >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)x;
        } else {
            p->link_cum[l] = 0;
        }
    }
    p->linked = 1;
    return ORC_OK;
}

/* One gamete of a parent (haplotypes h0, h1) under the linkage map; pi = 0
 * mother, 1 father.  Draws: Philox(j, g, rep, LINK<<24 | pi<<8 | sub):
 * sub 0 lane 0 = crossover-count uniform, lanes 1..3 = the coins of
 * chromosomes 0..31, 32..63, 64..95 (bit c % 32); crossover a uses lane a % 4
 * of sub 1 + a / 4. */
static void linked_gamete(const orc_pop *p, uint32_t j, uint32_t g, uint32_t pi, const uint8_t *h0,
                          const uint8_t *h1, uint8_t *out)
{
    const uint32_t L = p->L;
    uint32_t d0[4];
    draw4(p, j, g, ORC_LINK, (pi << 8) | 0u, d0);
    uint32_t K = 0;
    for (uint32_t i = 0; i < p->link_kmax; ++i)
        if (d0[0] >= p->link_cdf[i]) K++;
    uint8_t flips[ORC_MAX_LOCI];
    memset(flips, 0, sizeof flips);
    for (uint32_t a = 0; a < K; ++a) {
        uint32_t da[4];
        draw4(p, j, g, ORC_LINK, (pi << 8) | (1u + a / 4), da);
        uint32_t u = da[a % 4], I = 0;
        for (uint32_t l = 0; l + 1 < L; ++l)
            if (p->link_cum[l] <= u) I++;
        flips[I] ^= 1u; /* crossovers in one interval cancel in pairs */
    }
    uint8_t origin = 0;
    for (uint32_t l = 0; l < L; ++l) {
        if (l == 0 || p->chrom_of[l] != p->chrom_of[l - 1]) {
            uint32_t c = p->chrom_of[l];
            origin = (uint8_t)((d0[1 + c / 32] >> (c % 32)) & 1u);
        }
        origin ^= flips[l];
        out[l] = origin ? h1[l] : h0[l];
    }
}

/* Dominance deviations d[L] (Q8); the current parents' bins are recomputed. */
int orc_set_dominance(orc_pop *p, const int16_t *d)
{
    if (!p || !d) return ORC_ERR_INVALID;
    if (!p->dominance) p->dominance = (int16_t *)malloc(sizeof(int16_t) * p->L);
    if (!p->dominance) return ORC_ERR_OOM;
    memcpy(p->dominance, d, sizeof(int16_t) * p->L);
    for (uint32_t i = 0; i < p->n; ++i) {
        const uint8_t *h = p->par + (size_t)i * 2 * p->L;
        p->bin_par[i] = (uint16_t)bin_of(p, genetic_value(p, h, h + p->L));
    }
    return ORC_OK;
}

/* Normal step in raw units from twelve Philox lanes (Irwin-Hall(12)):
 * sum = u_1 + ... + u_12 (lane k%4 of sub sub0 + k/4), t = sum - 6 * 2^32,
 * step = floor(floor(t / 2^8) * s / 2^40) for a Q16 scale s, i.e. about
 * z * s / 2^16 with z = t / 2^32 (arithmetic shifts are floors). */
static int32_t irwin_hall_step(const orc_pop *p, uint32_t j, uint32_t g, uint32_t purpose, uint32_t sub0, int64_t s)
{
    uint64_t sum = 0;
    for (uint32_t k = 0; k < 12; ++k) {
        uint32_t d[4];
        draw4(p, j, g, purpose, sub0 + k / 4, d);
        sum += d[k % 4];
    }
    int64_t t = (int64_t)sum - (int64_t)6 * 4294967296LL;
    return (int32_t)(((t >> 8) * s) >> 40);
}

static int16_t clamp16(int32_t v)
{
    return (int16_t)(v < -32768 ? -32768 : v > 32767 ? 32767 : v);
}

/* Continuous allelic values: Q16 scales from standard deviations in trait
 * units (mutation: per allele copy, 256 raw units per trait unit; phenotype:
 * 512 raw units per trait unit), s = floor(sd * units * 2^16 + 1/2); the
 * current generation's values are init_values ([n][2][L]) or the biallelic
 * founders mapped to effect[l] * allele. */
int orc_set_continuous(orc_pop *p, double mut_sd, double env_sd, const int16_t *init_values)
{
    if (!p || !(mut_sd >= 0.0 && mut_sd < 64.0) || !(env_sd >= 0.0 && env_sd < 64.0) || p->linked || p->weighted ||
        p->dominance || p->gen != 0)
        return ORC_ERR_INVALID;
    const size_t cells = (size_t)p->n * 2 * p->L;
    p->vpar = (int16_t *)malloc(sizeof(int16_t) * cells);
    p->vchi = (int16_t *)malloc(sizeof(int16_t) * cells);
    if (!p->vpar || !p->vchi) return ORC_ERR_OOM;
    if (init_values) {
        memcpy(p->vpar, init_values, sizeof(int16_t) * cells);
    } else {
        for (size_t c = 0; c < cells; ++c) p->vpar[c] = (int16_t)(p->par[c] ? p->effects[c % p->L] : 0);
    }
    p->s_mut = (int64_t)floor(mut_sd * 256.0 * 65536.0 + 0.5);
    p->s_env = (int64_t)floor(env_sd * 512.0 * 65536.0 + 0.5);
    p->continuous = 1;
    return ORC_OK;
}

/* One offspring j of generation g under continuous allelic values: gametes
 * by the free-recombination bits of the biallelic model, mutations at the
 * same K distinct positions, each adding an Irwin-Hall step (mutation t uses
 * subs 3t..3t+2 of purpose MUTSIZE), then the phenotype with its
 * environmental step (subs 0..2 of purpose ENV).  Returns raw. */
static int32_t continuous_offspring(orc_pop *p, uint32_t j, uint32_t g, uint32_t mother, uint32_t father,
                                    uint32_t u_mut, int16_t *c0, int16_t *c1)
{
    const uint32_t L = p->L, W = L / 32;
    const int16_t *m0 = p->vpar + ((size_t)mother * 2 + 0) * L, *m1 = m0 + L;
    const int16_t *f0 = p->vpar + ((size_t)father * 2 + 0) * L, *f1 = f0 + L;
    for (uint32_t w = 0; w < W; ++w) {
        uint32_t qm = 2 * w + 0, qf = 2 * w + 1, dm[4], df[4];
        draw4(p, j, g, ORC_RECOMB, qm / 4, dm);
        draw4(p, j, g, ORC_RECOMB, qf / 4, df);
        for (uint32_t bit = 0; bit < 32; ++bit) {
            uint32_t l = 32 * w + bit;
            c0[l] = ((dm[qm % 4] >> bit) & 1u) ? m1[l] : m0[l];
            c1[l] = ((df[qf % 4] >> bit) & 1u) ? f1[l] : f0[l];
        }
    }
    uint32_t k = 0;
    for (uint32_t i = 0; i < p->kmax; ++i)
        if (u_mut >= p->cdf[i]) k++;
    uint32_t chosen[ORC_MAX_KMAX];
    uint32_t n_chosen = 0;
    for (uint32_t a = 0; a < ORC_MUT_DRAWS && n_chosen < k; ++a) {
        uint32_t dp[4];
        draw4(p, j, g, ORC_MUTPOS, a / 4, dp);
        uint32_t pos = scaled_index(dp[a % 4], 2 * L);
        int dup = 0;
        for (uint32_t t = 0; t < n_chosen; ++t)
            if (chosen[t] == pos) dup = 1;
        if (!dup) chosen[n_chosen++] = pos;
    }
    for (uint32_t t = 0; t < n_chosen; ++t) {
        int16_t *v = chosen[t] < L ? &c0[chosen[t]] : &c1[chosen[t] - L];
        *v = clamp16((int32_t)*v + irwin_hall_step(p, j, g, ORC_MUTSIZE, 3 * t, p->s_mut));
    }
    int32_t raw = 0;
    for (uint32_t l = 0; l < L; ++l) raw += (int32_t)c0[l] + (int32_t)c1[l];
    if (p->s_env) raw += irwin_hall_step(p, j, g, ORC_ENV, 0, p->s_env);
    return raw;
}

/* Weighted parents: acceptance threshold of bin b = floor(2^32 * w[b] / w_max)
 * in integer arithmetic, 0xFFFFFFFF where w[b] == w_max (always accepted);
 * a NULL table means uniform (every threshold 0xFFFFFFFF). */
static int weight_thresholds(const uint32_t *w, uint32_t *acc)
{
    if (!w) {
        for (uint32_t b = 0; b < ORC_BINS; ++b) acc[b] = ORC_CERTAIN;
        return ORC_OK;
    }
    uint32_t mx = 0;
    for (uint32_t b = 0; b < ORC_BINS; ++b) if (w[b] > mx) mx = w[b];
    if (mx == 0) return ORC_ERR_INVALID;
    for (uint32_t b = 0; b < ORC_BINS; ++b)
        acc[b] = w[b] == mx ? ORC_CERTAIN : (uint32_t)(((uint64_t)w[b] << 32) / mx);
    return ORC_OK;
}

int orc_set_weights(orc_pop *p, const uint32_t *mother_w, const uint32_t *father_w)
{
    if (!p || (!mother_w && !father_w)) return ORC_ERR_INVALID;
    if (weight_thresholds(mother_w, p->acc_mother) != ORC_OK) return ORC_ERR_INVALID;
    if (weight_thresholds(father_w, p->acc_father) != ORC_OK) return ORC_ERR_INVALID;
    p->weighted = 1;
    return ORC_OK;
}

/* One weighted parent of offspring j (pi = 0 mother, 1 father): proposal k
 * (k = 0..63) uses lanes 2(k%2) (survivor rank, floor(u S / 2^32)) and
 * 2(k%2)+1 (acceptance) of Philox(j, g, rep, MATEW<<24 | pi<<8 | k/2). */
static uint32_t weighted_parent(const orc_pop *p, uint32_t j, uint32_t g, uint32_t pi, const uint32_t *acc)
{
    uint32_t r = 0;
    for (uint32_t k = 0; k < ORC_MATE_ATTEMPTS; ++k) {
        uint32_t d[4];
        draw4(p, j, g, ORC_MATEW, (pi << 8) | (k / 2), d);
        r = scaled_index(d[2 * (k % 2)], p->S);
        uint32_t a = acc[p->bin_par[p->surv[r]]];
        if (a == ORC_CERTAIN || d[2 * (k % 2) + 1] < a) break;
    }
    return p->surv[r];
}

/* Beverton-Holt resource with a growth rate drawn every generation (model 1);
 * r_sd = 0 keeps r' = r. */
int orc_set_resource_model(orc_pop *p, int model, double r_sd)
{
    if (!p || !p->has_eco || (model != 0 && model != 1) || !(r_sd >= 0.0) || (model == 0 && r_sd != 0.0))
        return ORC_ERR_INVALID;
    p->eco_model = model;
    p->r_sd = r_sd;
    return ORC_OK;
}

/* Growth rate of generation g: r' = r + r_sd * z with the Irwin-Hall(12)
 * normal z = (u_1 + ... + u_12) 2^-32 - 6, u_k = lane k%4 of
 * Philox(0, g, rep, GROWTH<<24 | k/4). */
static double growth_rate(const orc_pop *p, uint32_t g)
{
    if (p->r_sd == 0.0) return p->r;
    uint64_t sum = 0;
    for (uint32_t k = 0; k < 12; ++k) {
        uint32_t d[4];
        draw4(p, 0, g, ORC_GROWTH, k / 4, d);
        sum += d[k % 4];
    }
    double u = (double)sum * (1.0 / 4294967296.0);
    double z = u - 6.0;
    double dev = p->r_sd * z;
    return p->r + dev;
}

/* Beverton-Holt update with consumption C (Q16): R' = (r' R) / (1 + R/K) -
 * C 2^-16, clamped at 0. */
static double resource_update_bh(double R, double rg, double K, uint64_t C)
{
    double grown_num = rg * R;
    double ratio = R / K;
    double den = 1.0 + ratio;
    double grown = grown_num / den;
    double eaten = (double)C * (1.0 / 65536.0);
    double next = grown - eaten;
    if (!(next > 0.0)) next = 0.0;
    return next;
}

/* Logistic update with consumption C (attack units in Q16):
 *   R' = (R + (r*R) * (1 - R/K)) - C * 2^-16, clamped at 0. */
static double resource_update(double R, double r, double K, uint64_t C)
{
    double ratio = R / K;
    double room = 1.0 - ratio;
    double rR = r * R;
    double growth = rR * room;
    double grown = R + growth;
    double eaten = (double)C * (1.0 / 65536.0);
    double next = grown - eaten;
    if (!(next > 0.0)) next = 0.0;
    return next;
}

/* ------------------------------------------------------------------------ */
/* One generation g = gen + 1, in the order of Fig. 1 (A-F). */
static void one_generation(orc_pop *p, orc_stats *st)
{
    const uint32_t n = p->n, L = p->L, W = L / 32, g = p->gen + 1;
    const uint32_t S = p->S;

    memset(st, 0, sizeof(*st));
    st->gen = g; st->n = n;
    st->min_raw = INT32_MAX; st->max_raw = INT32_MIN;

    uint32_t survivors = 0;
    for (uint32_t j = 0; j < n; ++j) {
        uint8_t *c0 = p->chi + ((size_t)j * 2 + 0) * L;
        uint8_t *c1 = p->chi + ((size_t)j * 2 + 1) * L;

        /* (A) parents: two uniform draws over the previous survivors */
        uint32_t d[4];
        draw4(p, j, g, ORC_MATE, 0, d);
        uint32_t mother, father;
        if (p->weighted) {
            mother = weighted_parent(p, j, g, 0, p->acc_mother);
            father = weighted_parent(p, j, g, 1, p->acc_father);
        } else {
            mother = p->surv[scaled_index(d[0], S)];
            father = p->surv[scaled_index(d[1], S)];
        }
        uint32_t u_surv = d[2];
        uint32_t u_mut = d[3];

        /* (B) free recombination: each locus of a gamete comes from the
         * parent's haplotype 0 or 1 by one independent fair bit.  The bit for
         * locus l of parent pi (0 mother, 1 father) is bit l%32 of the draw
         * with stream index q = 2*(l/32) + pi. */
        const uint8_t *m0 = p->par + ((size_t)mother * 2 + 0) * L;
        const uint8_t *m1 = p->par + ((size_t)mother * 2 + 1) * L;
        const uint8_t *f0 = p->par + ((size_t)father * 2 + 0) * L;
        const uint8_t *f1 = p->par + ((size_t)father * 2 + 1) * L;
        if (p->continuous) {
            int16_t *v0 = p->vchi + ((size_t)j * 2 + 0) * L, *v1 = v0 + L;
            int32_t raw = continuous_offspring(p, j, g, mother, father, u_mut, v0, v1);
            uint32_t b = bin_of(p, raw);
            uint32_t thr = p->table[b];
            if (p->f != ORC_CERTAIN) thr = (uint32_t)(((uint64_t)thr * (uint64_t)p->f) >> 32);
            int alive = (thr == ORC_CERTAIN) || (u_surv < thr);
            if (alive) {
                p->surv_next[survivors++] = j;
                st->sum_raw_surv += raw;
                if (p->has_eco) st->consumption += p->attack[b];
            }
            st->sum_raw += raw;
            st->sum_raw2 += (uint64_t)((int64_t)raw * (int64_t)raw);
            if (raw < st->min_raw) st->min_raw = raw;
            if (raw > st->max_raw) st->max_raw = raw;
            for (uint32_t l = 0; l < L; ++l) {
                st->het += (uint64_t)(v0[l] != v1[l]);
                st->allele += (uint64_t)((int64_t)v0[l] * v0[l] + (int64_t)v1[l] * v1[l]);
            }
            continue;
        }
        if (p->linked) {
            linked_gamete(p, j, g, 0, m0, m1, c0); /* maternal gamete -> haplotype 0 */
            linked_gamete(p, j, g, 1, f0, f1, c1); /* paternal gamete -> haplotype 1 */
        }
        for (uint32_t w = 0; w < W && !p->linked; ++w) {
            uint32_t qm = 2 * w + 0, qf = 2 * w + 1, dm[4], df[4];
            draw4(p, j, g, ORC_RECOMB, qm / 4, dm);
            draw4(p, j, g, ORC_RECOMB, qf / 4, df);
            uint32_t mask_m = dm[qm % 4], mask_f = df[qf % 4];
            for (uint32_t bit = 0; bit < 32; ++bit) {
                uint32_t l = 32 * w + bit;
                c0[l] = ((mask_m >> bit) & 1u) ? m1[l] : m0[l]; /* maternal gamete -> haplotype 0 */
                c1[l] = ((mask_f >> bit) & 1u) ? f1[l] : f0[l]; /* paternal gamete -> haplotype 1 */
            }
        }

        /* (B) mutation: K ~ Binomial(2L, mu) allele copies, at K distinct
         * uniformly drawn positions p in [0, 2L) (p < L: haplotype 0 locus p,
         * else haplotype 1 locus p - L); each mutation flips the allele. */
        uint32_t k = 0;
        for (uint32_t i = 0; i < p->kmax; ++i)
            if (u_mut >= p->cdf[i]) k++;
        uint32_t chosen[ORC_MAX_KMAX];
        uint32_t n_chosen = 0;
        for (uint32_t a = 0; a < ORC_MUT_DRAWS && n_chosen < k; ++a) {
            uint32_t dp[4];
            draw4(p, j, g, ORC_MUTPOS, a / 4, dp);
            uint32_t pos = scaled_index(dp[a % 4], 2 * L);
            int dup = 0;
            for (uint32_t t = 0; t < n_chosen; ++t)
                if (chosen[t] == pos) dup = 1;
            if (!dup) chosen[n_chosen++] = pos;
        }
        for (uint32_t t = 0; t < n_chosen; ++t) {
            uint32_t pos = chosen[t];
            if (pos < L) c0[pos] ^= 1u;
            else c1[pos - L] ^= 1u;
        }

        /* (C) additive phenotype */
        int32_t raw = genetic_value(p, c0, c1);

        /* (D) survival against the selective environment */
        uint32_t b = bin_of(p, raw);
        p->bin_chi[j] = (uint16_t)b;
        uint32_t thr = p->table[b];
        if (p->f != ORC_CERTAIN) thr = (uint32_t)(((uint64_t)thr * (uint64_t)p->f) >> 32);
        int alive = (thr == ORC_CERTAIN) || (u_surv < thr);

        /* (E) survivors, kept in offspring order */
        if (alive) {
            p->surv_next[survivors++] = j;
            st->sum_raw_surv += raw;
            if (p->has_eco) st->consumption += p->attack[b];
        }

        /* statistics over all offspring */
        st->sum_raw += raw;
        st->sum_raw2 += (uint64_t)((int64_t)raw * (int64_t)raw);
        if (raw < st->min_raw) st->min_raw = raw;
        if (raw > st->max_raw) st->max_raw = raw;
        for (uint32_t l = 0; l < L; ++l) {
            st->het += (uint64_t)(c0[l] != c1[l]);
            st->allele += (uint64_t)c0[l] + (uint64_t)c1[l];
        }
    }
    st->s = survivors;

    /* (F) environment update from the survivors */
    if (p->has_eco) {
        if (p->eco_model == 1) p->R = resource_update_bh(p->R, growth_rate(p, g), p->K, st->consumption);
        else p->R = resource_update(p->R, p->r, p->K, st->consumption);
        p->f = factor_q32(p->R, p->R_half);
        st->R = p->R;
    } else {
        st->R = 0.0;
    }
    st->f = p->f;

    /* the offspring become the next generation's parents */
    uint8_t *t8 = p->par; p->par = p->chi; p->chi = t8;
    uint32_t *t32 = p->surv; p->surv = p->surv_next; p->surv_next = t32;
    uint16_t *t16 = p->bin_par; p->bin_par = p->bin_chi; p->bin_chi = t16;
    int16_t *tv = p->vpar; p->vpar = p->vchi; p->vchi = tv;
    p->S = survivors;
    p->gen = g;
    if (survivors == 0) p->status = ORC_EXTINCT;
    st->status = (uint32_t)p->status;
}

/* Advance n_gen generations (fewer if the population goes extinct); one
 * statistics record per generation is written to out (may be NULL).
 * Returns the number of generations run, or a negative error. */
int orc_step(orc_pop *p, uint32_t n_gen, orc_stats *out)
{
    if (!p) return ORC_ERR_INVALID;
    int done = 0;
    for (uint32_t t = 0; t < n_gen; ++t) {
        if (p->status == ORC_EXTINCT) break;
        orc_stats st;
        one_generation(p, &st);
        if (out) out[done] = st;
        done++;
    }
    return done;
}

/* Packed genotypes of the current generation (all N individuals). */
int orc_read_genotypes(const orc_pop *p, uint32_t *out)
{
    if (!p || !out) return ORC_ERR_INVALID;
    if (p->continuous) { /* records of 2L int16 values (L words) */
        memcpy(out, p->vpar, sizeof(int16_t) * (size_t)p->n * 2 * p->L);
        return ORC_OK;
    }
    uint32_t W = p->L / 32;
    memset(out, 0, sizeof(uint32_t) * (size_t)p->n * 2 * W);
    for (uint32_t i = 0; i < p->n; ++i)
        for (uint32_t h = 0; h < 2; ++h)
            for (uint32_t l = 0; l < p->L; ++l)
                if (p->par[((size_t)i * 2 + h) * p->L + l])
                    out[(size_t)i * 2 * W + h * W + l / 32] |= 1u << (l % 32);
    return ORC_OK;
}

/* Per-locus allele counts of the current generation (the offspring formed
 * last, all N of them): out[l] = the allele-1 copies at locus l over both
 * haplotypes of every individual, so that out[l] / 2N is the allele frequency
 * of locus l (S2 "Genetics": biallelic loci, diploid individuals).
 * Biallelic populations only. */
int orc_locus_counts(const orc_pop *p, uint32_t *out)
{
    if (!p || !out || p->continuous) return ORC_ERR_INVALID;
    for (uint32_t l = 0; l < p->L; ++l) out[l] = 0;
    for (uint32_t i = 0; i < p->n; ++i)
        for (uint32_t h = 0; h < 2; ++h)
            for (uint32_t l = 0; l < p->L; ++l)
                if (p->par[((size_t)i * 2 + h) * p->L + l]) out[l] += 1u;
    return ORC_OK;
}

int orc_read_survivors(const orc_pop *p, uint32_t *out, uint32_t *S)
{
    if (!p || !S) return ORC_ERR_INVALID;
    *S = p->S;
    if (out) memcpy(out, p->surv, sizeof(uint32_t) * p->S);
    return ORC_OK;
}

void orc_get_state(const orc_pop *p, uint32_t *gen, uint32_t *S, int32_t *status, double *R, uint32_t *f)
{
    *gen = p->gen; *S = p->S; *status = p->status; *R = p->R; *f = p->f;
}

uint32_t orc_stats_size(void) { return (uint32_t)sizeof(orc_stats); }

/* FP32 summaries of one statistics record, derived from its exact integer
 * sums: mean and variance of the trait z = raw/512 over offspring, survival
 * fraction, mean heterozygosity per locus, allele-1 frequency. */
void orc_summarize(const orc_stats *st, uint32_t L, float out[5])
{
    double n = (double)st->n;
    double mean_raw = (double)st->sum_raw / n;
    double var_raw = (double)st->sum_raw2 / n - mean_raw * mean_raw;
    out[0] = (float)(mean_raw / 512.0);
    out[1] = (float)(var_raw / (512.0 * 512.0));
    out[2] = (float)((double)st->s / n);
    out[3] = (float)((double)st->het / (n * (double)L));
    out[4] = (float)((double)st->allele / (2.0 * n * (double)L));
}
