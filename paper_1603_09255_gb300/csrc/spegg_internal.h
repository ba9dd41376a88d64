// Internal types shared by the host engine and the kernels of libspegg_gb300.
// Not part of the C ABI (include/spegg.h is).
#pragma once

#include <cstddef>
#include <cstdint>

#include "spegg.h"

namespace spg {

constexpr int kBins = 4096;
constexpr int kMaxKmax = 32;      // entries of the Binomial(2L, mu) CDF table
constexpr int kMutDraws = 64;     // position draws tried per offspring
constexpr int kMaxPlanes = 16;    // bit planes of the offset-binary effects
constexpr int kMaxWords = 8;      // W = L/32 <= 8
constexpr int kBlock = 256;       // threads per block of the continuous-allele kernel
constexpr int kLutWords = 256;    // entries of one byte table (one per byte value)
constexpr uint32_t kBucket = 4096;                 // offspring per compaction bucket
constexpr uint32_t kBucketWords = kBucket / 32;    // bitmap words per bucket = compaction threads
constexpr uint32_t kCompactCopyThreads = 256;  // threads that write a bucket's survivors (8 warps)
constexpr uint32_t kCompactThreads = kCompactCopyThreads + 32;  // + one warp that closes the generation
constexpr uint32_t kCertain = 0xFFFFFFFFu;
// Single-lane offspring kernels for L <= 128 without linkage copy their parent
// records into a shared-memory ring of kParentStages tiles with cp.async
// (each thread its own records, kParentStages - 1 tiles ahead).
constexpr bool kStagedParents = true;
constexpr uint32_t kParentStages = 3;
constexpr int kAccCopies = 16;    // copies of the statistics accumulators (spread atomics)

constexpr int kMaxLoci = 256;
constexpr int kMaxLutBytes = kMaxLoci / 8;  // byte positions of a haplotype (L / 8)
constexpr int kMaxChrom = 96;            // chromosomes of a linkage map
constexpr uint32_t kLinkSites = 65536;   // crossover opportunities per gamete
constexpr double kMaxMapMorgans = 16.0;  // total length of a linkage map
constexpr int kLinkGuideBits = 12;       // the crossover uniform's top bits that index the guide table
constexpr int kLinkGuide = 1 << kLinkGuideBits;

// Philox counter word 3 = purpose << 24 | sub
enum Purpose : uint32_t {
    kFounder = 1, kMate = 2, kRecomb = 3, kMutPos = 4, kLink = 5, kMateW = 6, kGrowth = 7, kMutSize = 8, kEnv = 9
};
constexpr uint32_t kMateAttempts = 64;   // proposals per weighted parent

// Acceptance thresholds of weighted parents (device global memory): acc[0]
// mothers, acc[1] fathers, by phenotype bin (Q32, 0xFFFFFFFF = always).
struct alignas(16) WeightParams {
    uint32_t acc[2][kBins];
};

// Tables of a linkage map (device global memory, one per linked population).
struct alignas(16) LinkParams {
    uint32_t cdf[kMaxKmax];      // crossover count per gamete, Binomial(kLinkSites, D / kLinkSites) CDF, Q32
    uint32_t cum[kMaxLoci];      // interval CDF, Q32: crossover interval = #{l <= L-2 : cum[l] <= u}
    // bucket h of crossover uniforms (u >> 20 == h): interval I0 of u = h << 20
    // (bits 0-7), chrom[I0] (bits 8-14), chrom[I0 + 1] (bits 15-21), and how
    // many cum[l] (l <= L-2) lie inside the bucket (bits 26-27: 0, 1, or 2 =
    // two or more)
    uint32_t guide[kLinkGuide];
    uint8_t chrom[kMaxLoci];     // chromosome holding each locus
    uint16_t first[kMaxChrom];   // first locus of each chromosome
    uint16_t clast[kMaxChrom];   // last locus of each chromosome
    uint32_t kmax;               // entries of cdf
    uint32_t nchrom;
};

// Read-only parameters of one population (device global memory).
struct alignas(16) PopParams {
    uint32_t table[kBins];                  // viability thresholds per bin
    uint32_t attack[kBins];                 // Q16 attack rate per bin (ecology)
    uint32_t planes[kMaxPlanes * kMaxWords];// plane b, word w at [b * W + w]
    uint32_t dplanes[kMaxPlanes * kMaxWords];// dominance deviations, offset binary like planes
    int32_t d_min;                          // dominance = d_min + sum_b 2^b * dplane_b
    uint32_t ndplanes;                      // 0: additive genetic value
    uint32_t has_dom;                       // some locus has a non-zero dominance deviation
    // byte tables of the genetic value: lut[k * 256 + v] is the sum of the
    // effects of loci 8k .. 8k+7 whose bit is set in v (L / 8 tables), dlut
    // the same for the dominance deviations (applied to h0 ^ h1)
    alignas(16) int32_t lut[kMaxLutBytes * kLutWords];
    alignas(16) int32_t dlut[kMaxLutBytes * kLutWords];
    uint32_t cdf[kMaxKmax];                 // Binomial(2L, mu) CDF, Q32
    int32_t e_min;                          // effects = e_min + sum_b 2^b * plane_b
    uint32_t nplanes;
    int32_t bias;
    uint32_t shift;
    uint32_t kmax;
    uint32_t n;
    uint32_t n_loci;
    uint32_t words;
    uint32_t key0, key1, rep;
    uint32_t has_eco;
    double r, K, R_half;
    double r_sd;                 // Beverton-Holt: sd of the growth rate
    uint32_t eco_model;          // 0 logistic, 1 Beverton-Holt
    uint32_t continuous;         // allelic values are int16 Q8 (records of L words)
    long long s_mut, s_env;      // continuous: Irwin-Hall step scales, Q16
    uint32_t ntiles;
    uint32_t stats_cap;
    const LinkParams *link;      // linkage map tables, or null (free recombination)
    uint32_t linked;
    uint32_t weighted;           // parents drawn by weight (weights != null)
    const WeightParams *weights;
};

// the offspring kernel copies these tables with 16-byte cp.async
static_assert(offsetof(PopParams, table) % 16 == 0 && offsetof(PopParams, attack) % 16 == 0 &&
                  offsetof(PopParams, lut) % 16 == 0 && offsetof(PopParams, dlut) % 16 == 0,
              "tables copied in 16-byte chunks");

// Mutable per-population state (device global memory).
struct alignas(16) DevState {
    uint32_t gen;     // generations completed
    uint32_t S;       // survivors of generation `gen` (parents of the next)
    uint32_t f;       // resource factor applied to the next generation
    int32_t status;   // SPG_OK or SPG_EXTINCT
    double R;         // resource density
    uint32_t done;    // compaction buckets of the running generation that have finished
    uint32_t target;  // generations stop once gen reaches target (0xFFFFFFFF: never)
    // the generation being closed: computed while its survivors are being
    // compacted, committed by the block that finishes the last bucket
    uint32_t next_S, next_f;
    int32_t next_status;
    uint32_t pad;
    double next_R;
};

// Statistics of the generation being formed, accumulated by atomics; each
// population has kAccCopies copies on separate cache lines.
struct alignas(128) StatAcc {
    unsigned long long s;
    long long sum_raw, sum_raw_s;
    unsigned long long sum_raw2, cons, het, allele;
    int mn, mx;
};

// One population as seen by a generation launch.
struct alignas(16) Segment {
    const PopParams *prm;
    uint32_t *geno[2];                // ping-pong genotype buffers [N * 2W]
    uint32_t *dense;                  // the survivors' records in rank order [N * 2W] (parents of the next
                                      // generation), or null: parents through the survivor list
    uint32_t *surv[2];                // ping-pong survivor lists [N]
    uint32_t *alive;                  // alive bitmap of the generation being formed [nbuckets * kBucketWords]
    uint32_t *bucket_sum;             // survivors per bucket, by generation parity [2][nbuckets]
    uint16_t *obin;                   // weighted parents: phenotype bin of each offspring [N]
    unsigned long long *survw;        // weighted parents: [2][N], role pi and rank r -> survivor index | its
                                      // acceptance threshold for role pi << 32
    DevState *state;
    StatAcc *acc;                     // [kAccCopies]
    spg_stats *ring;                  // [stats_cap]
    uint32_t n;                       // offspring per generation
    uint32_t tile_begin;              // first launch-wide tile of this population
    uint32_t ntiles;
    uint32_t bucket_begin;            // first launch-wide bucket of this population
    uint32_t nbuckets;
    uint32_t pad;
};

// One run of an offspring block: tiles tile0 .. tile0 + count - 1 of segment
// seg.  The population's tiles are split into `shares` runs (this is run
// `share`); each run prefetches the same share of the population's parent
// records into L2.
struct alignas(16) Run {
    uint32_t seg, tile0, count, share, shares, pad[3];
};

struct GenArgs {
    const Segment *segs;         // device array of nsegs segments (used when nsegs > 1)
    const Run *runs;             // runs of all offspring blocks, block by block (nsegs > 1)
    const uint32_t *block_runs;  // runs of block b: runs[block_runs[b] .. block_runs[b + 1]) (nsegs > 1)
    const uint32_t *bucket_seg;  // segment of each launch-wide bucket (nsegs > 1)
    const uint32_t *tile_seg;    // segment of each launch-wide tile (continuous-allele groups, nsegs > 1)
    uint32_t nsegs;
    uint32_t total_tiles;        // tiles of the single segment (nsegs == 1: contiguous shares per block)
    uint32_t total_buckets;
    // dynamic shared memory of the offspring kernel: the byte tables at 0,
    // the survival thresholds after them, attack rates after those when
    // eco_table, the dominance byte tables at smem_dlut (0: none)
    uint32_t eco_table;
    uint32_t smem_dlut;
    uint32_t smem_parents;  // the ring of staged parent records (single-lane kernels without linkage or weights)
    Segment one;           // the segment itself when nsegs == 1 (read from kernel parameters)
};

using GenKernel = void (*)(GenArgs);

// Launch shape of the offspring kernel: threads per block, offspring per
// thread (per lane pair when lanes = 2) and lanes per offspring (1, or 2 for
// L >= 128: one lane per parent and gamete).  Results never depend on it.
struct Shape {
    uint32_t block = 256, items = 1, lanes = 1;
};

// The offspring kernel of one launch: entry, shape, dynamic shared-memory
// layout and size, and the number of blocks resident on the device (its
// persistent grid).  persistent = false: the continuous-allele kernel, one
// block per 256 offspring and no dynamic shared memory.
struct OffspringKernel {
    GenKernel fn = nullptr;
    uint32_t words = 0, block = 256, items = 1, lanes = 1;
    uint32_t eco_table = 0, smem_dlut = 0, smem_parents = 0;
    uint32_t smem = 0;
    uint32_t resident = 0;
    bool persistent = true;
};

// Offspring kernels (offspring_w*.cu) and the other kernels (kernels.cu).
bool supported_shape(uint32_t words, const Shape &shape);
// The offspring kernel of a shape; eco: some population of the launch has an
// ecology (the survival table carries attack rates), dom: some has dominance.
// staged: stage the parents through shared memory where the kernel supports
// it (for parents resident in HBM rather than L2).
OffspringKernel offspring_kernel(uint32_t words, const Shape &shape, bool linked, bool weighted, bool eco, bool dom,
                                 bool staged);
// Parent records above this many bytes (N x 8W) are staged in a single
// population's launch; launch groups and weighted populations always stage.
constexpr size_t kStageParentBytes = (size_t)48 << 20;
int prepare_offspring(OffspringKernel &k);  // sets the shared-memory limit, fills `resident`
GenKernel compact_kernel(uint32_t words);  // the compaction kernel for records of 2W words
uint32_t compact_smem();                   // its dynamic shared memory (the ring of child records)

// Per-locus allele counts of a population (optional, biallelic records):
// the counts of the generations kept in a ring [cap][L] (generation g in slot
// (g - 1) % cap), the count kernel's accumulator row [L] (zero between
// launches), the counter of its blocks that are done and the last generation
// it counted (0: none).
// A launch group counts every member at once: `member` holds each member's
// own arguments (its blocks are first .. first + blocks - 1 of the launch)
// and `block_member` the member of each block of the launch.
struct LocusArgs {
    uint32_t *ring, *acc, *done, *last;
    uint32_t cap, blocks, first;
    const LocusArgs *member;        // launch groups: [members] (null: one population, the fields above)
    const uint32_t *block_member;   // launch groups: [blocks]
};
constexpr uint32_t kLocusBlock = 256;     // threads per block of the per-locus count kernel
constexpr uint32_t kLocusMaxGrid = 608;   // its blocks, at most (four per SM)
constexpr uint32_t kLocusGroupsPerWarp = 16;  // groups of 32 records a warp counts, at least (grid size)
constexpr int kLocusPlanes = 5;           // bit-sliced counter planes per lane (31 records between flushes)
constexpr uint32_t kLocusBatch = 4;       // groups a warp loads before adding them (loads in flight)
using LocusKernel = void (*)(GenArgs, LocusArgs);
LocusKernel locus_kernel(uint32_t words, bool group = false);  // the count kernel for records of 2W words
uint32_t tile_size(const Shape &shape);  // offspring per tile: block * items / lanes
// Copy the offspring kernel's shape and shared-memory layout into a launch.
void apply_kernel(const OffspringKernel &k, GenArgs &a);
// Enqueue founders: generation-0 records by Philox draws, survivors = 0..n-1.
int launch_founders(uint32_t words, uint32_t *geno, uint32_t *surv, uint32_t n, uint32_t key0, uint32_t key1,
                    uint32_t rep, uint32_t p0_q32, void *stream);
// Enqueue survivors = 0..n-1 only (caller-supplied founders).
int launch_iota(uint32_t *surv, uint32_t n, void *stream);
// Enqueue dense[r] = geno[surv[r]] for the S current survivors (records of
// 2W words): the dense parent buffer after founders or a restore.
int launch_dense_gather(uint32_t words, const uint32_t *geno, const uint32_t *surv, uint32_t S, uint32_t *dense,
                        void *stream);
// The generation kernel of a continuous-allele population (one warp per
// offspring at a time, 256 offspring per block, no persistent grid).
OffspringKernel continuous_kernel(uint32_t n_loci, bool group = false);  // group: several populations (tile map)
// Enqueue continuous founders: value = effect[l] * allele of the biallelic
// founder draws (records of 2L int16), survivors = 0..n-1.
int launch_founders_cont(const PopParams *prm, uint32_t n_loci, uint32_t *geno, uint32_t *surv, uint32_t n,
                         uint32_t p0_q32, void *stream);
// Enqueue the weighted-parent words of the S current survivors (surv
// NULL: survivor r is record r), the bin computed from the record; the
// father words start n words after the mother words.
int launch_survivor_bins(const PopParams *prm, uint32_t words, const uint32_t *geno, const uint32_t *surv,
                         uint32_t S, uint32_t n, unsigned long long *survw, void *stream);
// Enqueue a state reset: state fields and cleared statistics accumulators.
int launch_set_state(DevState *st, StatAcc *acc, uint32_t gen, uint32_t S, uint32_t f, double R, int32_t status,
                     uint32_t target, void *stream);

}  // namespace spg
