// Host-side helpers shared by the population, batch and server engines.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "spegg.h"
#include "spegg_internal.h"

namespace spg {

constexpr uint32_t kGraphChunk = 32;          // generations per cached graph
constexpr uint32_t kPieceOffspring = 8192;     // least offspring of a launch group's piece of work (but one round)
constexpr uint32_t kMaxGridBlocks = 8192;     // offspring blocks of a launch group, at most
constexpr uint32_t kCheckpointMagic = 0x43475053u;  // "SPGC"

struct CheckpointHeader {
    uint32_t magic, version, n, n_loci, gen, S;
    int32_t status;
    uint32_t f;
    double R;
    uint64_t seed;
    uint32_t replicate, pad;
};

struct Allocator {
    spg_allocator hooks{nullptr, nullptr, nullptr};
    void *alloc(size_t bytes, cudaStream_t s) const;
    void release(void *p, cudaStream_t s) const;
};

// Byte offsets of one population's buffers inside its arena.
struct PopLayout {
    size_t params, state, acc, geno0, geno1, dense, surv0, surv1, alive, buckets, ring, segment, link;
    size_t weights, obin, survw;  // weighted parents only (0 otherwise)
    bool weighted;
    size_t total;
};

// One population's device memory: its arena, layout and sizes.
struct PopView {
    char *base = nullptr;
    PopLayout L{};
    uint32_t n = 0, words = 0, cap = 0, nbuckets = 0;
    cudaStream_t stream = nullptr;
};

// The two launches of one generation for a launch group.
struct GenLaunch {
    OffspringKernel offspring;
    GenKernel compact = nullptr;
    GenArgs args{};
    uint32_t blocks = 0;   // offspring grid: min(tiles, resident blocks)
    uint32_t buckets = 0;  // compaction grid
    LocusKernel locus = nullptr;  // per-locus allele counts after the compaction (single populations; null: off)
    LocusArgs la{};
};

// A cached CUDA graph of `length` generations (2 dependent launches each, 3
// with per-locus counts).
struct GraphChain {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t length = 0;
    ~GraphChain();
    void reset();
    int build(const GenLaunch &gl, uint32_t len);
};

int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
uint32_t mutation_cdf(double mu, uint32_t n_copies, uint32_t *cdf);
void effect_planes(const int16_t *effects, uint32_t n_loci, PopParams &prm);
uint32_t factor_q32_host(double R, double R_half);
size_t align_up(size_t x, size_t a);
int validate_desc(const spg_pop_desc *d);
int build_params(const spg_pop_desc *d, PopParams &prm);
// Linkage-map tables from map_morgans[L] (validated; see spegg.h).
int build_link(const double *map_morgans, uint32_t n_loci, LinkParams &lp);
// Acceptance thresholds from the mother and father weight tables (NULL: uniform).
int build_weights(const uint32_t *mother_w, const uint32_t *father_w, WeightParams &wp);
// dense: the population has a dense parent buffer (biallelic records; not
// the continuous-allele model, whose generation kernel reads parents by index).
PopLayout layout_for(uint32_t n, uint32_t words, uint32_t nbuckets, uint32_t cap, bool weighted = false,
                     bool dense = true);
Segment segment_at(char *base, const PopLayout &L, uint32_t n, uint32_t ntiles, uint32_t tile_begin,
                   uint32_t nbuckets, uint32_t bucket_begin);
uint32_t bucket_count(uint32_t n);
Shape default_shape(uint32_t words);
constexpr uint32_t kAutotuneCandidates = SPG_AUTOTUNE_CANDIDATES;  // launch shapes timed per group
Shape autotune_candidate(uint32_t words, uint32_t c);
int shape_from_abi(uint32_t words, const spg_launch_shape *in, Shape &out);
// One generation's launches (each kernel may start while its predecessor in
// the stream finishes; see griddep_wait in the kernels).
int launch_generation(const GenLaunch &gl, cudaStream_t stream);
// Append a chain of `len` generations of one launch group to a graph
// (kernel nodes joined by programmatic edges); params: the GenArgs pointer.
int add_generation_nodes(cudaGraph_t graph, const GenLaunch &gl, void **params, uint32_t len);
size_t group_table_bytes(uint32_t members, uint64_t offspring, uint32_t buckets);
int read_locus_rows(const LocusArgs &la, uint32_t n_loci, uint32_t from, uint32_t until, const DevState &st,
                    uint32_t first_gen, uint32_t count, uint32_t *out);
// Blocks of the per-locus count kernel for a population of n (16 groups of
// 32 records per warp at least, at most kLocusMaxGrid).
uint32_t locus_blocks(uint32_t n);
uint32_t tiles_for(uint32_t n, const Shape &shape);
void schedule_runs(const std::vector<uint32_t> &tiles, uint32_t G, uint32_t min_piece, std::vector<Run> &runs,
                   std::vector<uint32_t> &block_runs);
// Segment table, runs and bucket map of one launch group, uploaded into
// `table` (device memory; synchronous), and the group's launch description.
// eco / dom: some member has an ecology / dominance deviations.
// linked / weighted / continuous: the members' variant (all alike; such
// groups take the variant shape only: kBlock threads, one offspring per
// thread, one lane; continuous: words = L / 2, the int16 records' words).
int build_group_launch(const std::vector<const PopView *> &members, uint32_t words, const Shape &shape, bool eco,
                       bool dom, char *table, size_t table_capacity, GenLaunch &gl, bool linked = false,
                       bool weighted = false, bool continuous = false);
int view_sync(const PopView &v);
int view_state(const PopView &v, DevState &st);
int view_set_state(const PopView &v, uint32_t gen, uint32_t S, uint32_t f, double R, int32_t status,
                   uint32_t target);
int view_init(const PopView &v, const PopParams &prm, const uint32_t *init_genotypes, uint32_t p0_q32);
int check_ecology(const spg_ecology *eco);
int view_set_ecology(const PopView &v, PopParams &prm, const spg_ecology *eco);
int view_read_stats(const PopView &v, uint32_t first_gen, uint32_t count, spg_stats *out);
int view_read_genotypes(const PopView &v, uint32_t *host, size_t n_words);
int view_read_survivors(const PopView &v, uint32_t *host, size_t capacity, uint32_t *S);
int view_get_state(const PopView &v, spg_state *out);
int enqueue_generations(const GenLaunch &gl, uint32_t n_gen, GraphChain &chain, cudaStream_t stream);

}  // namespace spg
