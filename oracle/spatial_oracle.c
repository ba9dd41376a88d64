/*
 * CPU oracle for the spatial, age-structured multi-species community --
 * TEST INFRASTRUCTURE ONLY (loaded by the tests and the benchmark's CPU legs;
 * shares no code with the CUDA library).
 *
 * What it follows: Fig. 1 (parents, transmission, phenotype, survival against
 * the environment, removal of the dead, environment from the survivors), the
 * migration among patches and multi-species interactions of the Main text and
 * S3 (patches linked by migration to neighbouring patches; species interact
 * within a patch), age structure (overlapping generations), S2 "Genetics" for
 * transmission, and Fig. S5 B (every deme updated from its own index).
 *
 * Readings (the paper's S3 model is continuous and its parameters are not
 * available), all integer so both implementations agree exactly:
 *   - X x Y torus of patches; species s in each patch p form deme d = s*P + p,
 *     stored adults first: age 2, then age 1, then age 0;
 *   - at step t, with counts n_k (all ages) and m_s (age 2) at the start:
 *       survival factor  f = CERTAIN if sum_k A_sk n_k == 0,
 *                        else min(floor(2^32 D_s / (D_s + sum_k A_sk n_k)), 0xFFFFFFFE)
 *       recruitment      num = G_s + sum_k P_sk n_k, den = num + E_s + sum_k C_sk n_k,
 *                        g = den ? floor(2^32 num / den) : 0,
 *                        births B = min(bmax_s, floor(m_s * beta_s * g / 2^48))  (beta in Q16);
 *   - pre-existing individual of rank r (age a): survives iff its viability
 *     T_s[a][bin] (scaled by f) exceeds a Philox draw; survivors age to
 *     min(a+1, 2) and disperse with probability disp to one of the 4
 *     neighbours (N = y-1, S = y+1, E = x+1, W = x-1, wrapping);
 *   - newborn k of the deme: mother and father uniform over the deme's m_s
 *     adults, gametes by free recombination + mutation exactly as in the
 *     single-population update, age 0, no survival draw this step, disperses
 *     like a survivor;
 *   - new deme (s, q): for age class 2, 1, 0: the movers into q from source
 *     slots (q staying, from north, from south, from east, from west), each in
 *     source order (survivors by rank, then newborns by birth index).
 * Draws (Philox4x32-10, key = seed, counter (i, t, deme, purpose<<24 | sub)):
 *   founders 1 (i = rank, t = 0), newborn parents 2 (lanes: mother, father,
 *   move, mutation count), gametes 3, mutation positions 4, survivor 5 (lanes:
 *   survival, move, direction), newborn direction 6 (lane 0).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SP_BINS 4096
#define SP_MAX_SPECIES 4
#define SP_MAX_KMAX 32
#define SP_MUT_DRAWS 64
#define SP_CERTAIN 0xFFFFFFFFu
enum { SP_FOUNDER = 1, SP_MATE = 2, SP_RECOMB = 3, SP_MUTPOS = 4, SP_SURV = 5, SP_DISP = 6 };

/* species parameters (same layout as the library's spg_species) */
typedef struct {
    const int16_t *effects;     /* [L] */
    const uint32_t *tables;     /* [3][4096] viability by age */
    int32_t bin_bias;
    uint32_t bin_shift;
    double mu;
    uint32_t n0;                /* founders per patch */
    uint32_t p0_q32;
    uint32_t D, A[SP_MAX_SPECIES];
    uint32_t G, P[SP_MAX_SPECIES], E, C[SP_MAX_SPECIES];
    uint32_t beta_q16, bmax;
} orc_species_desc;

typedef struct {
    uint32_t t, species;
    uint32_t n_before, adults_before, births, survivors, movers, n_after, adults_after;
    uint32_t pad;
    int64_t sum_raw_surv;       /* raw phenotype summed over surviving pre-existing individuals */
    uint64_t het_newborn;       /* heterozygous loci summed over newborns */
    uint64_t allele_newborn;    /* allele-1 copies summed over newborns */
} orc_sp_stats;

typedef struct {
    uint32_t *rec;  /* [cap][2W] */
    uint8_t *age;
    uint32_t n, cap;
} orc_list;

typedef struct {
    uint32_t X, Y, P, ns, L, W;
    uint64_t seed;
    uint32_t disp_q32;
    int16_t effects[SP_MAX_SPECIES][256];
    uint32_t tables[SP_MAX_SPECIES][3][SP_BINS];
    orc_species_desc sp[SP_MAX_SPECIES];
    uint32_t cdf[SP_MAX_SPECIES][SP_MAX_KMAX], kmax[SP_MAX_SPECIES];
    uint32_t t;
    orc_list *deme; /* [ns * P] */
} orc_space;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint32_t orc_mutation_cdf(double mu, uint32_t n_copies, uint32_t *cdf_out);

static void sp_draw4(const orc_space *c, uint32_t i, uint32_t t, uint32_t deme, uint32_t purpose, uint32_t sub,
                     uint32_t out[4])
{
    uint32_t ctr[4] = { i, t, deme, (purpose << 24) | sub };
    uint32_t key[2] = { (uint32_t)(c->seed & 0xFFFFFFFFu), (uint32_t)(c->seed >> 32) };
    orc_philox4x32_10(ctr, key, out);
}

static uint32_t sp_index(uint32_t u, uint32_t n) { return (uint32_t)(((uint64_t)u * n) >> 32); }

static int list_push(orc_list *l, const uint32_t *rec, uint8_t age, uint32_t W)
{
    if (l->n == l->cap) {
        uint32_t cap = l->cap ? l->cap * 2 : 16;
        uint32_t *r = (uint32_t *)realloc(l->rec, sizeof(uint32_t) * 2 * W * cap);
        if (!r) return -1;
        l->rec = r;
        uint8_t *a = (uint8_t *)realloc(l->age, cap);
        if (!a) return -1;
        l->age = a;
        l->cap = cap;
    }
    memcpy(l->rec + (size_t)l->n * 2 * W, rec, sizeof(uint32_t) * 2 * W);
    l->age[l->n] = age;
    l->n++;
    return 0;
}

static uint32_t get_bit(const uint32_t *words, uint32_t pos) { return (words[pos / 32] >> (pos % 32)) & 1u; }

/* additive phenotype, per locus (eq. S2-phenval) */
static int32_t sp_phenotype(const int16_t *e, uint32_t L, uint32_t W, const uint32_t *rec)
{
    int32_t raw = 0;
    for (uint32_t l = 0; l < L; ++l)
        raw += (int32_t)e[l] * (int32_t)(get_bit(rec, l) + get_bit(rec + W, l));
    return raw;
}

static uint32_t sp_bin(const orc_species_desc *s, int32_t raw)
{
    int64_t v = (int64_t)raw + s->bin_bias;
    if (v < 0) return 0;
    int64_t b = v >> s->bin_shift;
    return b > SP_BINS - 1 ? SP_BINS - 1 : (uint32_t)b;
}

void orc_space_destroy(orc_space *c)
{
    if (!c) return;
    if (c->deme)
        for (uint32_t d = 0; d < c->ns * c->P; ++d) { free(c->deme[d].rec); free(c->deme[d].age); }
    free(c->deme);
    free(c);
}

orc_space *orc_space_create(uint32_t X, uint32_t Y, uint32_t n_species, uint32_t L, uint64_t seed,
                            uint32_t disp_q32, const orc_species_desc *species)
{
    if (!X || !Y || !n_species || n_species > SP_MAX_SPECIES || (L % 32) || !L || L > 256 || !species) return NULL;
    orc_space *c = (orc_space *)calloc(1, sizeof(orc_space));
    if (!c) return NULL;
    c->X = X; c->Y = Y; c->P = X * Y; c->ns = n_species; c->L = L; c->W = L / 32;
    c->seed = seed; c->disp_q32 = disp_q32; c->t = 0;
    c->deme = (orc_list *)calloc((size_t)n_species * c->P, sizeof(orc_list));
    if (!c->deme) { orc_space_destroy(c); return NULL; }
    for (uint32_t s = 0; s < n_species; ++s) {
        c->sp[s] = species[s];
        memcpy(c->effects[s], species[s].effects, sizeof(int16_t) * L);
        memcpy(c->tables[s], species[s].tables, sizeof(uint32_t) * 3 * SP_BINS);
        c->sp[s].effects = c->effects[s];
        c->sp[s].tables = &c->tables[s][0][0];
        c->kmax[s] = orc_mutation_cdf(species[s].mu, 2 * L, c->cdf[s]);
    }
    uint32_t rec[16];
    for (uint32_t s = 0; s < n_species; ++s) {
        for (uint32_t p = 0; p < c->P; ++p) {
            uint32_t d = s * c->P + p, n0 = species[s].n0;
            for (uint32_t r = 0; r < n0; ++r) {
                memset(rec, 0, sizeof rec);
                for (uint32_t h = 0; h < 2; ++h)
                    for (uint32_t l = 0; l < L; ++l) {
                        uint32_t q = h * L + l, u[4];
                        sp_draw4(c, r, 0, d, SP_FOUNDER, q / 4, u);
                        if (u[q % 4] < species[s].p0_q32) rec[h * c->W + l / 32] |= 1u << (l % 32);
                    }
                /* founders: first half adults, next quarter age 1, rest age 0 */
                uint8_t age = r < n0 / 2 ? 2 : (r < n0 / 2 + n0 / 4 ? 1 : 0);
                if (list_push(&c->deme[d], rec, age, c->W)) { orc_space_destroy(c); return NULL; }
            }
        }
    }
    return c;
}

/* destination patch of a move from patch p in direction dir (0 stay, 1 N, 2 S, 3 E, 4 W) */
static uint32_t sp_dest(const orc_space *c, uint32_t p, uint32_t dir)
{
    uint32_t x = p % c->X, y = p / c->X;
    if (dir == 1) y = (y + c->Y - 1) % c->Y;
    else if (dir == 2) y = (y + 1) % c->Y;
    else if (dir == 3) x = (x + 1) % c->X;
    else if (dir == 4) x = (x + c->X - 1) % c->X;
    return y * c->X + x;
}

/* slot of a move in the destination's source order (stay, from north, from
 * south, from east, from west): moving S comes from the north, etc. */
static uint32_t sp_slot(uint32_t dir)
{
    static const uint32_t slot[5] = { 0, 2, 1, 4, 3 };
    return slot[dir];
}

static void sp_plan(const orc_space *c, uint32_t s, uint32_t p, const uint32_t *n_of, uint32_t m,
                    uint32_t *f_out, uint32_t *b_out)
{
    const orc_species_desc *sp = &c->sp[s];
    uint64_t pressure = 0, benefit = sp->G, cost = sp->E;
    for (uint32_t k = 0; k < c->ns; ++k) {
        uint64_t nk = n_of[k * c->P + p];
        pressure += (uint64_t)sp->A[k] * nk;
        benefit += (uint64_t)sp->P[k] * nk;
        cost += (uint64_t)sp->C[k] * nk;
    }
    if (pressure == 0) {
        *f_out = SP_CERTAIN;
    } else {
        unsigned __int128 q = ((unsigned __int128)sp->D << 32) / ((uint64_t)sp->D + pressure);
        *f_out = q > 0xFFFFFFFEull ? 0xFFFFFFFEu : (uint32_t)q;
    }
    uint64_t den = benefit + cost;
    uint64_t g = 0;
    if (den) {
        unsigned __int128 q = ((unsigned __int128)benefit << 32) / den;
        g = (uint64_t)q; /* <= 2^32 */
    }
    unsigned __int128 prod = (unsigned __int128)((uint64_t)m * sp->beta_q16) * g;
    uint64_t births = (uint64_t)(prod >> 48);
    *b_out = births > sp->bmax ? sp->bmax : (uint32_t)births;
}

/* One step of the whole community; one statistics record per species. */
int orc_space_step(orc_space *c, orc_sp_stats *out)
{
    const uint32_t P = c->P, ns = c->ns, L = c->L, W = c->W, t = c->t + 1;
    const uint32_t nd = ns * P;
    uint32_t *n_of = (uint32_t *)calloc(nd, sizeof(uint32_t));
    uint32_t *m_of = (uint32_t *)calloc(nd, sizeof(uint32_t));
    orc_list *bucket = (orc_list *)calloc((size_t)nd * 15, sizeof(orc_list)); /* [dest][age class 2,1,0][slot] */
    if (!n_of || !m_of || !bucket) { free(n_of); free(m_of); free(bucket); return -1; }
    for (uint32_t d = 0; d < nd; ++d) {
        n_of[d] = c->deme[d].n;
        for (uint32_t r = 0; r < c->deme[d].n; ++r) m_of[d] += c->deme[d].age[r] == 2;
    }
    for (uint32_t s = 0; s < ns; ++s) {
        memset(&out[s], 0, sizeof out[s]);
        out[s].t = t;
        out[s].species = s;
    }
    uint32_t rec[16];
    int err = 0;
    for (uint32_t s = 0; s < ns && !err; ++s) {
        const orc_species_desc *sp = &c->sp[s];
        for (uint32_t p = 0; p < P && !err; ++p) {
            const uint32_t d = s * P + p;
            const orc_list *src = &c->deme[d];
            const uint32_t m = m_of[d];
            uint32_t f, B;
            sp_plan(c, s, p, n_of, m, &f, &B);
            out[s].n_before += src->n;
            out[s].adults_before += m;
            out[s].births += B;
            /* pre-existing individuals: survival, ageing, dispersal */
            for (uint32_t r = 0; r < src->n && !err; ++r) {
                const uint32_t *x = src->rec + (size_t)r * 2 * W;
                uint32_t a = src->age[r], u[4];
                sp_draw4(c, r, t, d, SP_SURV, 0, u);
                int32_t raw = sp_phenotype(sp->effects, L, W, x);
                uint32_t thr = sp->tables[a * SP_BINS + sp_bin(sp, raw)];
                if (f != SP_CERTAIN) thr = (uint32_t)(((uint64_t)thr * f) >> 32);
                if (!(thr == SP_CERTAIN || u[0] < thr)) continue;
                out[s].survivors++;
                out[s].sum_raw_surv += raw;
                uint32_t dir = u[1] < c->disp_q32 ? 1 + sp_index(u[2], 4) : 0;
                out[s].movers += dir != 0;
                uint32_t na = a + 1 > 2 ? 2 : a + 1;
                uint32_t dest = s * P + sp_dest(c, p, dir);
                err |= list_push(&bucket[(size_t)dest * 15 + (2 - na) * 5 + sp_slot(dir)], x, (uint8_t)na, W);
            }
            /* newborns */
            for (uint32_t k = 0; k < B && !err; ++k) {
                uint32_t u[4];
                sp_draw4(c, k, t, d, SP_MATE, 0, u);
                const uint32_t *mo = src->rec + (size_t)sp_index(u[0], m) * 2 * W;
                const uint32_t *fa = src->rec + (size_t)sp_index(u[1], m) * 2 * W;
                memset(rec, 0, sizeof rec);
                for (uint32_t w = 0; w < W; ++w) {
                    uint32_t qm = 2 * w, qf = 2 * w + 1, dm[4], df[4];
                    sp_draw4(c, k, t, d, SP_RECOMB, qm / 4, dm);
                    sp_draw4(c, k, t, d, SP_RECOMB, qf / 4, df);
                    for (uint32_t b = 0; b < 32; ++b) {
                        uint32_t l = 32 * w + b;
                        uint32_t am = (dm[qm % 4] >> b) & 1u ? get_bit(mo + W, l) : get_bit(mo, l);
                        uint32_t af = (df[qf % 4] >> b) & 1u ? get_bit(fa + W, l) : get_bit(fa, l);
                        rec[w] |= am << b;
                        rec[W + w] |= af << b;
                    }
                }
                uint32_t nmut = 0;
                for (uint32_t i = 0; i < c->kmax[s]; ++i) nmut += u[3] >= c->cdf[s][i];
                uint32_t chosen[SP_MAX_KMAX], nc = 0;
                for (uint32_t a2 = 0; a2 < SP_MUT_DRAWS && nc < nmut; ++a2) {
                    uint32_t dp[4];
                    sp_draw4(c, k, t, d, SP_MUTPOS, a2 / 4, dp);
                    uint32_t pos = sp_index(dp[a2 % 4], 2 * L), dup = 0;
                    for (uint32_t i = 0; i < nc; ++i) dup |= chosen[i] == pos;
                    if (!dup) chosen[nc++] = pos;
                }
                for (uint32_t i = 0; i < nc; ++i) {
                    uint32_t pos = chosen[i];
                    uint32_t word = pos < L ? pos / 32 : W + (pos - L) / 32;
                    rec[word] ^= 1u << (pos % 32);
                }
                for (uint32_t w = 0; w < W; ++w) {
                    out[s].het_newborn += (uint64_t)__builtin_popcount(rec[w] ^ rec[W + w]);
                    out[s].allele_newborn += (uint64_t)__builtin_popcount(rec[w]) + __builtin_popcount(rec[W + w]);
                }
                uint32_t dd[4];
                sp_draw4(c, k, t, d, SP_DISP, 0, dd);
                uint32_t dir = u[2] < c->disp_q32 ? 1 + sp_index(dd[0], 4) : 0;
                out[s].movers += dir != 0;
                uint32_t dest = s * P + sp_dest(c, p, dir);
                err |= list_push(&bucket[(size_t)dest * 15 + 2 * 5 + sp_slot(dir)], rec, 0, W);
            }
        }
    }
    if (!err) {
        for (uint32_t d = 0; d < nd; ++d) {
            orc_list *dl = &c->deme[d];
            dl->n = 0;
            for (uint32_t b = 0; b < 15 && !err; ++b) {
                orc_list *bl = &bucket[(size_t)d * 15 + b];
                for (uint32_t i = 0; i < bl->n && !err; ++i)
                    err |= list_push(dl, bl->rec + (size_t)i * 2 * W, bl->age[i], W);
            }
            const uint32_t s = d / P;
            out[s].n_after += dl->n;
            for (uint32_t i = 0; i < dl->n; ++i) out[s].adults_after += dl->age[i] == 2;
        }
    }
    for (size_t b = 0; b < (size_t)nd * 15; ++b) { free(bucket[b].rec); free(bucket[b].age); }
    free(bucket); free(n_of); free(m_of);
    if (err) return -1;
    c->t = t;
    return 0;
}

uint32_t orc_space_deme_size(const orc_space *c, uint32_t species, uint32_t patch)
{
    return c->deme[species * c->P + patch].n;
}

/* copy a deme's records ([n][2W]) and ages ([n]) */
int orc_space_read_deme(const orc_space *c, uint32_t species, uint32_t patch, uint32_t *rec, uint8_t *age)
{
    const orc_list *l = &c->deme[species * c->P + patch];
    if (rec) memcpy(rec, l->rec, sizeof(uint32_t) * 2 * c->W * l->n);
    if (age) memcpy(age, l->age, l->n);
    return (int)l->n;
}

uint32_t orc_sp_stats_size(void) { return (uint32_t)sizeof(orc_sp_stats); }
uint32_t orc_species_desc_size(void) { return (uint32_t)sizeof(orc_species_desc); }

/* Replace a deme's contents (records [n][2W], ages [n]); ages must be
 * non-increasing (adults first).  Used by the tests to build special states. */
int orc_space_set_deme(orc_space *c, uint32_t species, uint32_t patch, const uint32_t *rec, const uint8_t *age,
                       uint32_t n)
{
    if (species >= c->ns || patch >= c->P) return -1;
    for (uint32_t i = 1; i < n; ++i)
        if (age[i] > age[i - 1] || age[i] > 2) return -1;
    orc_list *l = &c->deme[species * c->P + patch];
    l->n = 0;
    for (uint32_t i = 0; i < n; ++i)
        if (list_push(l, rec + (size_t)i * 2 * c->W, age[i], c->W)) return -1;
    return 0;
}
