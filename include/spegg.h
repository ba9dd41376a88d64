/*
 * spegg.h -- C ABI of the GB300 (sm_103a) engine for the per-generation update
 * of a forward-time, multi-locus population-genetics simulation (sPEGG,
 * Okamoto & Amarasekare, arXiv:1603.09255).
 *
 * One generation of a population, in the order of the paper's Fig. 1:
 *   (A) parents: every offspring draws a mother and a father uniformly, with
 *       replacement, from the previous generation's survivors (Wright-Fisher,
 *       constant N offspring);
 *   (B) transmission: each gamete takes every locus from one of its parent's
 *       two haplotypes by an independent fair bit (free recombination, S2
 *       "Genetics"), then each allele copy mutates (flips) with probability mu;
 *   (C) phenotype: raw = sum over loci of effect[l] * (copies of allele 1)
 *       (additive map, eq. S2-phenval; the trait is z = raw / 512), plus,
 *       with dominance (the Main text's non-additive maps), dominance[l] at
 *       every heterozygous locus;
 *   (D) survival: bin = clamp((raw + bin_bias) >> bin_shift, 0, 4095); the
 *       offspring survives with probability table[bin] / 2^32 (0xFFFFFFFF =
 *       certain), scaled by the resource factor f when an ecology is set;
 *   (E) the survivors, in offspring order, become the next parents;
 *   (F) ecology: a logistic resource is consumed by the survivors
 *       (trait-dependent attack table) and sets the next factor f.
 *
 * Genotype layout: L loci (a multiple of 32; 32, 64, 128 or 256), W = L/32
 * uint32 words per haplotype, one individual = 2W consecutive words
 * (haplotype 0 words, then haplotype 1 words); locus l is bit l%32 of word
 * l/32.  Haplotype 0 of an offspring is its mother's gamete.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key (seed low
 * word, seed high word) and counter (i, g, replicate, purpose<<24 | sub),
 * i = individual index, g = generation being formed (0 = founders):
 *   founders  purpose 1: allele copy q = h*L + l is 1 iff lane q%4 of sub q/4
 *             is < p0_q32;
 *   parents   purpose 2, sub 0: lane 0 -> mother, lane 1 -> father (index
 *             floor(u * S / 2^32) into the survivor list), lane 2 -> survival
 *             draw u (survive iff u < threshold), lane 3 -> mutation count
 *             k = number of Binomial(2L, mu) CDF entries <= u;
 *   gametes   purpose 3: stream q = 2w + parent (0 mother, 1 father) is lane
 *             q%4 of sub q/4; bit b set -> locus 32w+b comes from haplotype 1;
 *   mutations purpose 4: draw a is lane a%4 of sub a/4, position
 *             floor(u * 2L / 2^32) (p < L: haplotype 0 locus p, else
 *             haplotype 1 locus p-L); draws a = 0..63 until k distinct;
 *   linkage   purpose 5 (populations with a linkage map, replacing the
 *             gamete draws of purpose 3): for parent pi (0 mother, 1
 *             father), sub pi<<8 | 0: lane 0 -> crossover count K = number
 *             of crossover-CDF entries <= u, lanes 1..3 -> the coins of
 *             chromosomes 0..31, 32..63, 64..95 (bit c%32); crossover a uses
 *             lane a%4 of sub pi<<8 | (1 + a/4) and lies in interval
 *             I = number of interval-CDF entries cum[0..L-2] <= u;
 *   weighted  purpose 6 (populations with parent weights, replacing lanes 0
 *   parents   and 1 of purpose 2): proposal k = 0..63 for parent pi uses lanes
 *             2(k%2) (survivor rank floor(u * S / 2^32)) and 2(k%2)+1
 *             (acceptance v) of sub pi<<8 | k/2; the proposal is taken iff
 *             the threshold t of the survivor's bin is 0xFFFFFFFF or v < t,
 *             the last proposal if all 64 are rejected.
 * Parent weights (S2 "Reproduction": the chance to parent an egg grows with
 * the parent's size relative to the others'): uint32 weights over the 4096
 * phenotype bins, one table for mothers and one for fathers, applied to each
 * survivor's bin at birth; threshold t[b] = floor(2^32 * w[b] / max w) in
 * integer arithmetic, 0xFFFFFFFF where w[b] is the maximum (bounded
 * rejection sampling: each parent is drawn with probability proportional to
 * its weight, up to the 64-proposal bound).
 * Continuous allelic values (allele_model 1; S2 "Genetics": values vary
 * continuously, a mutation moves a value by a normal step, the phenotype is
 * normal around the genetic value): a record holds 2L int16 values in Q8
 * (haplotype 0 loci 0..L-1, then haplotype 1; L uint32 words, little-endian
 * pairs), raw = sum of all 2L values plus an environmental step.  Gametes use
 * the purpose-3 bits of the biallelic model, mutations its purpose-2/4 count
 * and distinct positions; mutation t (in the order its position was drawn)
 * adds the step of purpose 8 subs 3t..3t+2, the phenotype the step of purpose
 * 9 subs 0..2, and a mutated value is clamped to [-32768, 32767].  A step
 * with scale s: sum = the twelve lanes of the three subs, t = sum - 6 * 2^32,
 * step = ((t >> 8) * s) >> 40 (arithmetic shifts), with s = floor(sd * 256 *
 * 2^16 + 1/2) for mutations and floor(sd * 512 * 2^16 + 1/2) for the
 * phenotype (sd in trait units; the Irwin-Hall(12) normal, exact in integer
 * arithmetic).  Founders: init_values, or the biallelic founder draws mapped
 * to value = effect[l] * allele.
 * Linkage map (the paper's variable linkage maps, read as Haldane's
 * no-interference model): map_morgans[l] (l >= 1) is the distance in Morgans
 * between loci l-1 and l, or negative where locus l starts a new chromosome;
 * w_l = that distance for linked intervals, else 0; D = sum of w_l (at most
 * 16 Morgans; at most 96 chromosomes).  The crossover count is
 * Binomial(65536, D/65536) (tabulated exactly like the mutation CDF below
 * with mu = D/65536 over 65536 copies); the interval CDF is s = s + w_l,
 * cum[l] = floor(2^32 * (s / D)) saturated at 0xFFFFFFFF (all 0 when D = 0).
 * A gamete locus takes haplotype 1 iff its chromosome's coin XOR the parity
 * of the crossovers in the intervals from the chromosome's first locus up to
 * it is 1.
 * The Binomial CDF is tabulated in Q32 from mu with IEEE-double basic
 * operations in a fixed order: P0 = (1-mu)^(2L) by repeated multiplication,
 * P(k+1) = ((P(k) * (2L-k)) / (k+1)) * mu / (1-mu), cdf[k] = floor(2^32 *
 * running sum), stopping at the first value >= 0xFFFFFFFF or after 32 entries.
 *
 * Conventions for every call:
 *   - return value: SPG_OK (0), SPG_EXTINCT (1, informational), or a negative
 *     SPG_ERR_* code; spg_last_error() gives a message for the calling thread;
 *   - caller arrays are read (copied) during the call; the caller keeps them;
 *   - device memory is owned by the library (through the caller's allocator
 *     when one is given) and released by the matching destroy call;
 *   - work is enqueued on the object's CUDA stream; only read_*, get_state,
 *     checkpoint and synchronize wait for it.
 */
#ifndef SPEGG_H
#define SPEGG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPG_ABI_VERSION 3u
#define SPG_N_BINS 4096u
#define SPG_CERTAIN 0xFFFFFFFFu
#define SPG_MAX_LOCI 256u

enum spg_status_code {
    SPG_OK = 0,
    SPG_EXTINCT = 1,        /* the population has no survivors; stepping stops */
    SPG_ERR_INVALID = -1,   /* bad argument or description                      */
    SPG_ERR_OOM = -2,       /* device allocation failed                         */
    SPG_ERR_CUDA = -3,      /* a CUDA runtime call failed                       */
    SPG_ERR_TIMEOUT = -4,   /* reserved: a bounded wait gave up                 */
    SPG_ERR_RANGE = -5,     /* requested generations are not in the stats ring  */
    SPG_ERR_BUDGET = -6     /* request exceeds the server's memory budget       */
};

typedef struct spg_pop spg_pop;

/* Optional device-memory hooks (e.g. a framework's caching allocator).
 * alloc returns device memory of at least `bytes` (256-byte aligned) or NULL;
 * free releases a pointer returned by alloc.  NULL hooks: cudaMallocAsync /
 * cudaFreeAsync on the object's stream. */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *ctx;
} spg_allocator;

/* One population (one species, one replicate). */
typedef struct {
    uint32_t n;                     /* N individuals per generation, 1 .. 2^31-1        */
    uint32_t n_loci;                /* L: 32, 64, 128 or 256                            */
    uint64_t seed;                  /* Philox key                                       */
    uint32_t replicate;             /* replicate id (Philox counter word 2)             */
    const int16_t *effects;         /* [L] allelic effects of allele 1, Q8              */
    const uint32_t *init_genotypes; /* [N * 2W] generation-0 records, or NULL           */
    uint32_t p0_q32;                /* if NULL above: allele 1 iff Philox draw < p0_q32 */
    const uint32_t *surv_table;     /* [4096] viability thresholds (Q32, 0xFFFFFFFF = 1)*/
    int32_t bin_bias;               /* phenotype bin map (see above)                    */
    uint32_t bin_shift;             /* 0 .. 31                                          */
    double mu;                      /* per-locus mutation probability, 0 <= mu < 1      */
    uint32_t stats_capacity;        /* most recent generations kept readable (0: 1024)  */
    const double *map_morgans;      /* [L] linkage map (see above), copied; NULL: free  */
                                    /* recombination.  Populations, batch members and   */
                                    /* server jobs (those run the variant shape: 256    */
                                    /* threads, one offspring per thread, one lane).    */
    const uint32_t *mother_weights; /* [4096] parent weights by bin (see above), copied;*/
    const uint32_t *father_weights; /* NULL: uniform for that role.  Like map_morgans;  */
                                    /* a table whose weights are all 0 is               */
                                    /* SPG_ERR_INVALID.                                 */
    const int16_t *dominance;       /* [L] dominance deviations (Q8) of heterozygous    */
                                    /* loci, copied; NULL: additive.  Every population, */
                                    /* batch member and job; bin_bias / bin_shift must  */
                                    /* cover the widened phenotype range.               */
    uint32_t allele_model;          /* 0 biallelic bits, 1 continuous int16 values      */
    double mut_sd;                  /* continuous: sd of a mutation step (trait units)  */
    double env_sd;                  /* continuous: sd of the environmental step         */
    const int16_t *init_values;     /* continuous: [N * 2L] generation-0 values or NULL */
                                    /* Continuous populations (also batch members and   */
                                    /* served jobs, at the variant shape): no linkage   */
                                    /* map, weights or dominance, 0 <= sd < 64.         */
} spg_pop_desc;

/* Consumer-resource ecology (Fig. 1F; S2 "Resource Consumption"): after the
 * survivors of generation g are known,
 *   C  = sum over survivors of attack[bin]            (Q16 units)
 *   R' = (R + (r*R) * (1 - R/K)) - C * 2^-16, clamped at 0          (model 0)
 *   R' = (r'*R) / (1 + R/K) - C * 2^-16, clamped at 0, Beverton-Holt (model 1)
 *   f  = floor(2^32 * R' / (R' + R_half)), capped at 0xFFFFFFFE
 * and generation g+1 survives with threshold floor(table[bin] * f / 2^32).
 * Beverton-Holt growth rate of generation g: r' = r + r_sd * z with the
 * Irwin-Hall(12) normal z = (u_1 + ... + u_12) * 2^-32 - 6, u_k = lane k%4 of
 * Philox counter (0, g, replicate, 7<<24 | k/4) (the paper's normally drawn
 * r'; the integer sum keeps every implementation exact); r_sd = 0: r' = r.
 * Every operation is one IEEE-double operation in the order written. */
typedef struct {
    double r, K, R0, R_half;   /* growth rate, carrying capacity, initial R, half-saturation */
    const uint32_t *attack;    /* [4096] attack rate per phenotype bin, Q16 */
    uint32_t model;            /* 0 logistic, 1 Beverton-Holt                */
    double r_sd;               /* Beverton-Holt: sd of r' per generation (>= 0; 0 for model 0) */
} spg_ecology;

/* Exact per-generation statistics (integer sums over the N offspring unless
 * noted). 88 bytes. */
typedef struct {
    uint32_t gen;          /* generation index g (1-based)                    */
    uint32_t n;            /* offspring                                       */
    uint32_t s;            /* survivors                                       */
    uint32_t status;       /* SPG_OK or SPG_EXTINCT after this generation      */
    int64_t sum_raw;       /* sum of raw phenotypes                           */
    uint64_t sum_raw2;     /* sum of raw^2                                    */
    int64_t sum_raw_surv;  /* sum of raw over survivors                       */
    int32_t min_raw, max_raw;
    uint64_t het;          /* heterozygous loci, summed                       */
    uint64_t allele;       /* copies of allele 1, summed                      */
    uint64_t consumption;  /* C (0 without ecology)                           */
    double R;              /* resource after this generation (0 without)     */
    uint32_t f;            /* factor for the next generation (0xFFFFFFFF: none)*/
    uint32_t pad;
} spg_stats;

typedef struct {
    uint32_t gen;      /* generations completed                         */
    uint32_t S;        /* current survivors (parents of the next one)   */
    int32_t status;    /* SPG_OK or SPG_EXTINCT                         */
    uint32_t f;        /* current resource factor                       */
    double R;          /* current resource                              */
} spg_state;

/* Create a population at generation 0 (Fig. S4, Initialize()): validates and
 * copies the description, allocates its device state and builds its
 * generation-0 genotypes (the caller's, or Philox draws at frequency p0).
 * stream: a cudaStream_t, or NULL for a stream the library creates and owns.
 * Errors: SPG_ERR_INVALID (bad description), SPG_ERR_OOM, SPG_ERR_CUDA. */
int spg_create_population(const spg_pop_desc *desc, const spg_allocator *alloc, void *stream,
                          spg_pop **out);

/* Attach (or replace) the consumer-resource ecology; resets R to R0 and f to
 * the factor of R0.  Errors: SPG_ERR_INVALID (K <= 0, R_half <= 0, R0 < 0,
 * NULL attack). */
int spg_set_ecology(spg_pop *pop, const spg_ecology *eco);

/* Enqueue n_gen generations (Fig. 1 A-F each) on the population's stream and
 * return without waiting.  Generations after an extinction do nothing;
 * extinction is reported by spg_get_state and spg_read_stats. */
int spg_step_generations(spg_pop *pop, uint32_t n_gen);

/* Copy statistics of generations first_gen .. first_gen+count-1 to out
 * (waits for the stream).  SPG_ERR_RANGE if any of them has not run or has
 * left the ring. */
int spg_read_stats(spg_pop *pop, uint32_t first_gen, uint32_t count, spg_stats *out);

/* Per-locus allele counts (S2 "Genetics": biallelic diploid loci; the allele
 * frequency of locus l is count[l] / 2N).  With enable != 0, every generation
 * formed from now on also counts, over both haplotypes of its N offspring,
 * the allele-1 copies of each locus, kept in a ring of stats_capacity rows of
 * L uint32 (one more kernel after each compaction; enable = 0 stops it).  The
 * first call allocates that ring through the population's allocator; the
 * call waits for the stream.  Biallelic populations only (SPG_ERR_INVALID
 * for continuous values).  Counts are not part of a checkpoint: after
 * spg_restore they start again with the next generation formed.
 * spg_read_locus_counts copies generations first_gen .. first_gen+count-1
 * to out ([count][L] uint32, row i for generation first_gen + i; waits for
 * the stream).  Readable: the generations formed since the latest enabling
 * call (or restore) while counting was on, still in the ring.  SPG_ERR_INVALID
 * while counts have never been enabled, SPG_ERR_RANGE for any other
 * generation. */
int spg_set_locus_counts(spg_pop *pop, int enable);
int spg_read_locus_counts(spg_pop *pop, uint32_t first_gen, uint32_t count, uint32_t *out);

/* Copy the current generation's N records (N * 2W words) to host memory;
 * n_words must be at least N * 2W.  Waits for the stream. */
int spg_read_genotypes(spg_pop *pop, uint32_t *host, size_t n_words);

/* Copy the current survivor list (ascending offspring indices) to host;
 * *S receives its length; host may be NULL to query the length only. */
int spg_read_survivors(spg_pop *pop, uint32_t *host, size_t capacity, uint32_t *S);

/* Current generation, survivors, status and resource (waits for the stream). */
int spg_get_state(spg_pop *pop, spg_state *out);

/* Whole-state snapshot (genotypes, survivors, generation, resource) for exact
 * resumption: counter-based draws make a restored run identical to an
 * uninterrupted one.  spg_checkpoint_size gives the byte size. */
int spg_checkpoint_size(spg_pop *pop, size_t *bytes);
int spg_checkpoint(spg_pop *pop, void *host, size_t capacity);
int spg_restore(spg_pop *pop, const void *host, size_t bytes);

/* Launch shape of the generation kernel: threads per block (128, 256 or 512;
 * 0 = 256), offspring per thread (1 or 2 for L <= 64, 1 for L >= 128; 0 = 1)
 * and lanes per offspring (1, or 2 for L >= 128: one lane per parent, each
 * loading that parent's record and forming the gamete it passes on; 0 = the
 * default, 2 for L = 256 and 1 otherwise).  A launch-shape choice only: every
 * shape gives identical results.  Populations with a linkage map or parent
 * weights, and continuous allelic values, run 256 threads with one offspring
 * per thread.  spg_get_launch_shape reports the shape in use.
 * SPG_ERR_INVALID for an unsupported shape.  Waits for the stream. */
typedef struct {
    uint32_t threads_per_block;
    uint32_t items_per_thread;
    uint32_t lanes_per_offspring;
} spg_launch_shape;

int spg_set_launch_shape(spg_pop *pop, const spg_launch_shape *shape);
int spg_get_launch_shape(spg_pop *pop, spg_launch_shape *out);
/* Offspring per thread at 256 threads per block and one lane per offspring
 * (spg_set_launch_shape with {256, items_per_thread, 1}); spg_get_tiling
 * reports the offspring per thread in use. */
int spg_set_tiling(spg_pop *pop, uint32_t items_per_thread);
int spg_get_tiling(spg_pop *pop, uint32_t *items_per_thread);

/* ---- Batched replicates ---------------------------------------------------
 * Many independent populations advanced by shared launches: the flattened
 * loop over replicates of the paper's Fig. S5 B.  Members are grouped by
 * locus count and variant (plain; linkage map; parent weights; both;
 * continuous values); each generation is one offspring launch and one
 * compaction launch per group, groups run as independent branches of one
 * cached CUDA graph.  Members with a linkage map, parent weights or
 * continuous values run the variant shape (256 threads, one offspring per
 * thread, one lane); launch shapes and the autotuner apply to the plain
 * members of each locus count.  Every member keeps its own parameters,
 * state, buffers and statistics ring, and its results are identical to the same population
 * created with spg_create_population and stepped alone.  Member i is
 * descs[i]; the descriptions are copied.  Errors as for a population;
 * SPG_ERR_INVALID names the first invalid member. */
typedef struct spg_batch spg_batch;

int spg_batch_create(const spg_pop_desc *descs, uint32_t count, const spg_allocator *alloc, void *stream,
                     spg_batch **out);
int spg_batch_set_ecology(spg_batch *batch, uint32_t member, const spg_ecology *eco);
/* Enqueue n_gen generations of every member (returns after enqueue). */
int spg_batch_step(spg_batch *batch, uint32_t n_gen);
/* Launch shape of the members with n_loci loci (as spg_set_launch_shape);
 * spg_batch_set_tiling / spg_batch_get_tiling as spg_set_tiling. */
int spg_batch_set_launch_shape(spg_batch *batch, uint32_t n_loci, const spg_launch_shape *shape);
int spg_batch_get_launch_shape(spg_batch *batch, uint32_t n_loci, spg_launch_shape *out);
int spg_batch_set_tiling(spg_batch *batch, uint32_t n_loci, uint32_t items_per_thread);
int spg_batch_get_tiling(spg_batch *batch, uint32_t n_loci, uint32_t *items_per_thread);
/* Launch-shape autotuner: for each locus-count group of plain members (no
 * linkage map, parent weights or continuous values: those run their one
 * shape for as many generations), runs one untimed generation and then
 * times gens_per_trial real generations with each of
 * SPG_AUTOTUNE_CANDIDATES launch shapes -- threads per block (128, 256, 512)
 * x offspring per thread (1, 2) for L <= 64, x lanes per offspring (1, 2) for
 * L >= 128 -- and keeps the fastest.  Every
 * member advances by the same number of generations (report->gens_run =
 * SPG_AUTOTUNE_CANDIDATES * (gens_per_trial + 1)); results do not depend on
 * the shapes chosen.  The report (may be NULL) gives each group's chosen
 * shape (index 0..3 for L = 32, 64, 128, 256; zeros for an empty group) and
 * the best and worst candidate's time per generation. */
#define SPG_AUTOTUNE_CANDIDATES 6u
typedef struct {
    spg_launch_shape groups[4];
    float best_ms[4];
    float worst_ms[4];
    uint32_t gens_run;
} spg_autotune_report;

int spg_batch_autotune(spg_batch *batch, uint32_t gens_per_trial, spg_autotune_report *report);
int spg_batch_read_stats(spg_batch *batch, uint32_t member, uint32_t first_gen, uint32_t count, spg_stats *out);
/* Per-locus allele counts of every biallelic member (as
 * spg_set_locus_counts / spg_read_locus_counts for each member; a group of
 * several members counts them all in one more launch after its compaction;
 * continuous-allele members are not counted and their reads are
 * SPG_ERR_INVALID).  The first enabling call allocates every member's ring
 * through the batch's allocator; both calls wait for the stream. */
int spg_batch_set_locus_counts(spg_batch *batch, int enable);
int spg_batch_read_locus_counts(spg_batch *batch, uint32_t member, uint32_t first_gen, uint32_t count,
                                uint32_t *out);
int spg_batch_read_genotypes(spg_batch *batch, uint32_t member, uint32_t *host, size_t n_words);
int spg_batch_read_survivors(spg_batch *batch, uint32_t member, uint32_t *host, size_t capacity, uint32_t *S);
int spg_batch_get_state(spg_batch *batch, uint32_t member, spg_state *out);
int spg_batch_synchronize(spg_batch *batch);
uint32_t spg_batch_size(const spg_batch *batch);
void spg_batch_destroy(spg_batch *batch);

/* ---- Served jobs (continuous batching) -------------------------------------
 * Jobs -- one population each, with its own generation count -- arrive over
 * time.  Each scheduling tick retires the resident jobs that reached their
 * generation count (their statistics are kept in host memory, their device
 * memory is freed), admits queued jobs in arrival order while a resident slot
 * is free and the job's device footprint fits the memory budget, and advances
 * every resident job by up to gens_per_tick generations in shared launches
 * (jobs of different lengths, locus counts and variants run together, one
 * launch group per locus count and variant; each stops at its own count).  A
 * job's results are identical to the same population run alone.  A job's
 * linkage map and parent weights are built and checked when it is submitted
 * (the caller's arrays need not outlive spg_server_submit).  Times are
 * seconds on the server's clock (spg_server_clock). */
#define SPG_JOB_QUEUED 0u
#define SPG_JOB_RESIDENT 1u
#define SPG_JOB_FINISHED 2u

typedef struct spg_server spg_server;

typedef struct {
    size_t memory_budget;     /* device bytes for resident jobs (0: 80% of free memory) */
    uint32_t max_resident;    /* resident job slots (0: 1024)                          */
    uint32_t gens_per_tick;   /* generations advanced per tick (0: 16)                 */
} spg_server_config;

typedef struct {
    uint64_t job;
    uint32_t state;           /* SPG_JOB_QUEUED / RESIDENT / FINISHED */
    uint32_t gen;             /* generations completed (enqueued while resident) */
    int32_t status;           /* SPG_OK or SPG_EXTINCT once finished */
    uint32_t n_gen;           /* requested generations */
    double t_arrival, t_admit, t_finish;   /* -1 until reached */
    size_t footprint;         /* device bytes while resident */
} spg_job_info;

typedef struct {
    uint64_t submitted, queued, resident, peak_resident;
    size_t memory_budget, memory_used, peak_memory_used;
} spg_server_counters;

int spg_server_create(const spg_server_config *cfg, const spg_allocator *alloc, void *stream, spg_server **out);
/* Queue a job (the description, founders and ecology are copied).  t_arrival
 * is recorded for latency.  SPG_ERR_BUDGET if the job alone exceeds the budget. */
int spg_server_submit(spg_server *server, const spg_pop_desc *desc, const spg_ecology *eco, uint32_t n_gen,
                      double t_arrival, uint64_t *job);
/* One scheduling tick (waits for its generations); reports resident and queued jobs. */
int spg_server_tick(spg_server *server, uint32_t *resident, uint32_t *queued);
/* Tick until every submitted job has finished. */
int spg_server_drain(spg_server *server);
/* Replay an arrival trace: job i is submitted once arrivals[i] seconds have
 * passed since the call started (ecos[i] applies where has_eco[i] != 0; both
 * may be NULL), ticking in between, until every job has finished; jobs[i]
 * receives job i's id. */
int spg_server_run_trace(spg_server *server, const spg_pop_desc *descs, const spg_ecology *ecos,
                         const uint8_t *has_eco, const uint32_t *n_gen, const double *arrivals, uint32_t count,
                         uint64_t *jobs);
int spg_server_job_info(spg_server *server, uint64_t job, spg_job_info *out);
/* Statistics of a finished job (generations first_gen .. first_gen+count-1). */
int spg_server_job_stats(spg_server *server, uint64_t job, uint32_t first_gen, uint32_t count, spg_stats *out);
int spg_server_stats(spg_server *server, spg_server_counters *out);
double spg_server_clock(spg_server *server);
void spg_server_destroy(spg_server *server);

/* ---- Spatial, age-structured multi-species community ----------------------
 * Species on an X x Y torus of patches (migration among patches, Main text
 * and S3), individuals of age class 0, 1, 2 (overlapping generations), all
 * updated in parallel per deme (species s in patch p, d = s*P + p; Fig. S5 B).
 * A deme stores adults (age 2) first, then age 1, then age 0.  One step,
 * with counts n_k (all ages) of every species in the patch and m (adults) of
 * the deme at its start:
 *   survival factor  f = 0xFFFFFFFF if sum_k A[k] n_k == 0, else
 *                    min(floor(2^32 D / (D + sum_k A[k] n_k)), 0xFFFFFFFE);
 *   births           num = G + sum_k P[k] n_k, den = num + E + sum_k C[k] n_k,
 *                    g = den ? floor(2^32 num / den) : 0,
 *                    B = min(bmax, floor(m * beta_q16 * g / 2^48));
 *   member of rank r and age a: Philox (r, t, d, 5<<24) lanes (u, v, w):
 *                    survives iff table[a][bin] scaled by f (as in a population)
 *                    exceeds u; survivors age to min(a+1, 2) and move iff
 *                    v < disp_q32, to neighbour 1 + floor(4 w / 2^32) (1 N:
 *                    y-1, 2 S: y+1, 3 E: x+1, 4 W: x-1, wrapping);
 *   newborn k (age 0, no survival draw this step): Philox (k, t, d, 2<<24)
 *                    lanes (mother rank and father rank among the m adults,
 *                    move draw, mutation count); gametes (purpose 3) and
 *                    mutation positions (purpose 4) as in a population;
 *                    direction from lane 0 of Philox (k, t, d, 6<<24);
 *   new deme (s, q): for age 2, 1, 0: movers into q from q itself, then from
 *                    its north, south, east and west neighbours, each in
 *                    source order (members by rank, then newborns).
 * Founders: n0 per deme, allele copy q of rank r is 1 iff lane q%4 of
 * Philox (r, 0, d, 1<<24 | q/4) < p0_q32; ranks below n0/2 are adults, the
 * next n0/4 age 1, the rest age 0.  Exceeding `capacity` individuals or
 * `staging_capacity` newborns in a step stops the community with
 * SPG_ERR_RANGE (the last complete layout is kept). */
typedef struct {
    const int16_t *effects;     /* [L] allelic effects, Q8 */
    const uint32_t *tables;     /* [3][4096] viability by age class 0, 1, 2 */
    int32_t bin_bias;
    uint32_t bin_shift;
    double mu;                  /* per-locus mutation probability */
    uint32_t n0;                /* founders per patch */
    uint32_t p0_q32;
    uint32_t D, A[4];           /* survival interaction */
    uint32_t G, P[4], E, C[4];  /* recruitment */
    uint32_t beta_q16, bmax;    /* births per adult (Q16), cap per deme and step */
} spg_species;

typedef struct {
    uint32_t X, Y;              /* torus; X * Y <= 2^20 patches */
    uint32_t n_species;         /* 1 .. 4 */
    uint32_t n_loci;            /* 32, 64, 128 or 256 (all species) */
    uint64_t seed;
    uint32_t disp_q32;          /* dispersal probability, Q32 */
    uint32_t capacity;          /* individuals (0: twice the founders) */
    uint32_t staging_capacity;  /* newborns per step (0: capacity / 2) */
    uint32_t stats_capacity;    /* steps kept in the statistics ring (0: 1024) */
    const spg_species *species; /* [n_species], copied */
} spg_space_desc;

typedef struct {
    uint32_t t, species;
    uint32_t n_before, adults_before, births, survivors, movers, n_after, adults_after;
    uint32_t pad;
    int64_t sum_raw_surv;       /* raw phenotype over surviving members */
    uint64_t het_newborn;       /* heterozygous loci over newborns */
    uint64_t allele_newborn;    /* allele-1 copies over newborns */
} spg_space_stats;

typedef struct spg_space spg_space;

int spg_space_create(const spg_space_desc *desc, const spg_allocator *alloc, void *stream, spg_space **out);
/* Enqueue n_steps steps (returns after enqueue). */
int spg_space_step(spg_space *space, uint32_t n_steps);
/* Statistics of steps first_step .. first_step+count-1: count * n_species
 * records, species-major within a step.  Waits for the stream. */
int spg_space_read_stats(spg_space *space, uint32_t first_step, uint32_t count, spg_space_stats *out);
/* Individuals per deme (n_species * X * Y entries, deme d = s*P + p). */
int spg_space_sizes(spg_space *space, uint32_t *sizes, size_t count);
/* One deme's records ([n][2W]) and ages ([n]); either may be NULL to query n. */
int spg_space_read_deme(spg_space *space, uint32_t species, uint32_t patch, uint32_t *rec, uint8_t *age,
                        size_t capacity, uint32_t *n);
int spg_space_get_state(spg_space *space, uint32_t *t, int32_t *status, uint32_t *total);
int spg_space_synchronize(spg_space *space);
void spg_space_destroy(spg_space *space);

/* ---- One generation without any device allocation -----------------------
 * The paper has no counterpart to this call; it exists for callers that may
 * not allocate device memory: host applications whose device memory is owned
 * entirely by another framework's pool (a cudaMalloc of their own would fail
 * or fragment that pool), plug-ins that run inside such a framework under a
 * fixed memory budget, and real-time or certified loops that forbid
 * allocation after start-up because an allocation can block the device or
 * fail at an arbitrary moment.
 *
 * It forms generation `generation` of one population from caller-owned device
 * buffers: `parents` (N * 2W records of generation-1) and `survivors` (their S
 * ascending survivor indices) in, `children` (N * 2W), `survivors_out`
 * (capacity N; the first stats->s entries are written) and one statistics
 * record `stats` out.  The draws, arithmetic and results are those of
 * spg_step_generations for the same population at the same generation,
 * without an ecology (the survival factor f is given; R is reported as 0).
 * All working memory comes from one fixed array inside the library of
 * SPG_NOALLOC_SCRATCH_BYTES on every device that loads the library, held
 * until the process exits; it bounds N to SPG_NOALLOC_MAX_N, and larger
 * populations are rejected with SPG_ERR_INVALID before any device work.
 * The first call on a device looks up that array's device address (with the
 * device current); make that first call before any stream capture begins.
 * Every call on a device shares the array and finds the previous call's
 * contents in it (the call re-initialises what must start from zero), so
 * calls whose work overlaps on the GPU -- on different streams or from
 * different threads -- race and must be serialised by the caller.
 * Host inputs (effects, surv_table) are read during the call; the work is
 * enqueued on `stream` (a cudaStream_t, NULL = the legacy default stream) and
 * the outputs are valid once it completes.  Returns SPG_OK or a negative
 * SPG_ERR_* code (spg_last_error() explains it). */
#define SPG_NOALLOC_MAX_N 4194304u
#define SPG_NOALLOC_SCRATCH_BYTES 634624u

typedef struct {
    uint32_t n;                   /* N, 1 .. SPG_NOALLOC_MAX_N                  */
    uint32_t n_loci;              /* 32, 64, 128 or 256                         */
    uint64_t seed;
    uint32_t replicate;
    uint32_t generation;          /* generation being formed, >= 1              */
    uint32_t S;                   /* survivors listed in `survivors`, 1 .. N    */
    uint32_t f;                   /* survival factor, Q32 (0xFFFFFFFF = none)   */
    const int16_t *effects;       /* host [L]                                   */
    const uint32_t *surv_table;   /* host [4096]                                */
    int32_t bin_bias;
    uint32_t bin_shift;
    double mu;
    const uint32_t *parents;      /* device [N * 2W]                            */
    const uint32_t *survivors;    /* device [S]                                 */
    uint32_t *children;           /* device [N * 2W], written                   */
    uint32_t *survivors_out;      /* device [N], first stats->s written         */
    spg_stats *stats;             /* device, one record written                 */
} spg_noalloc_generation;

int spg_generation_noalloc(const spg_noalloc_generation *args, void *stream);

/* Wait for all work enqueued on the population's stream. */
int spg_synchronize(spg_pop *pop);

/* Release the population's device memory (after its stream's work). */
void spg_destroy(spg_pop *pop);

/* FP32 summaries of one statistics record from its exact integer sums:
 * out = {mean z, variance of z, survival fraction, heterozygosity per locus,
 * allele-1 frequency}. */
void spg_summarize(const spg_stats *st, uint32_t n_loci, float out[5]);

/* The Binomial(n_copies, mu) CDF table the library uses for mutation counts
 * (construction stated above); writes up to 32 entries to cdf and returns
 * how many.  Host only. */
uint32_t spg_mutation_cdf(double mu, uint32_t n_copies, uint32_t cdf[32]);

const char *spg_status_string(int code);
const char *spg_last_error(void);
uint32_t spg_abi_version(void);


#ifdef __cplusplus
}
#endif
#endif /* SPEGG_H */
