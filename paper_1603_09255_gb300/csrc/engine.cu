// Host engine and C ABI of libspegg_gb300 (see include/spegg.h).
//
// A population owns one device arena holding its parameters, two genotype
// buffers and two survivor lists (ping-pong by generation parity, chosen on
// the device so every generation launch has identical arguments), its
// look-back status words, its state and its statistics ring.  Generations are
// enqueued as a cached CUDA graph of kGraphChunk back-to-back launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <queue>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "spegg.h"
#include "spegg_engine.h"
#include "spegg_internal.h"

namespace spg {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(SPG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------ host tables
// Binomial(n_copies, mu) CDF in Q32 with IEEE-double basic operations in the
// fixed order stated in spegg.h (each product/quotient rounded separately).
uint32_t mutation_cdf(double mu, uint32_t n_copies, uint32_t *cdf) {
    const double q = 1.0 - mu;
    double p_k = 1.0;
    for (uint32_t i = 0; i < n_copies; ++i) p_k = p_k * q;
    double running = 0.0;
    uint32_t entries = 0;
    for (uint32_t k = 0; k <= n_copies && entries < (uint32_t)kMaxKmax; ++k) {
        running = running + p_k;
        const double q32 = running * 4294967296.0;
        if (q32 >= 4294967295.0) break;
        cdf[entries++] = (uint32_t)q32;
        const double t1 = p_k * (double)(n_copies - k);
        const double t2 = t1 / (double)(k + 1);
        const double t3 = t2 * mu;
        p_k = t3 / q;
    }
    return entries;
}

// Per-locus values in offset binary: v_l - v_min split into bit planes, plane
// b word w holding bit b of the offsets of loci 32w .. 32w+31.
static void offset_planes(const int16_t *v, uint32_t n_loci, uint32_t *planes, int32_t &v_min, uint32_t &nplanes) {
    const uint32_t W = n_loci / 32;
    int32_t lo = v[0], hi = v[0];
    for (uint32_t l = 1; l < n_loci; ++l) {
        lo = std::min<int32_t>(lo, v[l]);
        hi = std::max<int32_t>(hi, v[l]);
    }
    const uint32_t span = (uint32_t)(hi - lo);
    uint32_t np = 0;
    while (np < 32 && (span >> np) != 0u) ++np;
    std::memset(planes, 0, sizeof(uint32_t) * kMaxPlanes * kMaxWords);
    for (uint32_t l = 0; l < n_loci; ++l) {
        const uint32_t off = (uint32_t)((int32_t)v[l] - lo);
        for (uint32_t b = 0; b < np && b < (uint32_t)kMaxPlanes; ++b)
            if ((off >> b) & 1u) planes[b * W + l / 32] |= 1u << (l % 32);
    }
    v_min = lo;
    nplanes = np;
}

// Effects in offset binary (the additive genetic value's bit planes).
void effect_planes(const int16_t *effects, uint32_t n_loci, PopParams &prm) {
    offset_planes(effects, n_loci, prm.planes, prm.e_min, prm.nplanes);
}

// Byte tables of per-locus values v (effects, or dominance deviations): table
// k, entry b is the sum of v[8k + i] over the bits i set in b -- the value of
// the eight loci 8k .. 8k+7 held in byte k of a haplotype (locus l is bit l % 32
// of word l / 32).  Exact in int32 (at most 8 * 32768 in magnitude).
static void byte_tables(const int16_t *v, uint32_t n_loci, int32_t *lut) {
    std::memset(lut, 0, sizeof(int32_t) * kMaxLutBytes * kLutWords);
    for (uint32_t k = 0; k < n_loci / 8; ++k)
        for (uint32_t b = 0; b < (uint32_t)kLutWords; ++b) {
            int32_t sum = 0;
            for (uint32_t i = 0; i < 8; ++i)
                if ((b >> i) & 1u) sum += v[8 * k + i];
            lut[k * kLutWords + b] = sum;
        }
}

// Resource factor of the ecology, same arithmetic as the device finalizer.
uint32_t factor_q32_host(double R, double R_half) {
    const double den = R + R_half;
    const double q = R / den;
    const double scaled = q * 4294967296.0;
    if (scaled >= 4294967294.0) return 0xFFFFFFFEu;
    if (!(scaled > 0.0)) return 0u;
    return (uint32_t)scaled;
}

// ----------------------------------------------------------- device memory
void *Allocator::alloc(size_t bytes, cudaStream_t s) const {
    if (hooks.alloc) return hooks.alloc(bytes, hooks.ctx);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void Allocator::release(void *p, cudaStream_t s) const {
    if (!p) return;
    if (hooks.free) hooks.free(p, hooks.ctx);
    else cudaFreeAsync(p, s);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ----------------------------------------------------------- validation
int validate_desc(const spg_pop_desc *d) {
    if (!d) return fail(SPG_ERR_INVALID, "population description is NULL");
    if (d->n == 0 || d->n > 0x7FFFFFFFu) return fail(SPG_ERR_INVALID, "n must be in [1, 2^31-1] (got %u)", d->n);
    if (!(d->n_loci == 32 || d->n_loci == 64 || d->n_loci == 128 || d->n_loci == 256))
        return fail(SPG_ERR_INVALID, "n_loci must be 32, 64, 128 or 256 (got %u)", d->n_loci);
    if (!d->effects) return fail(SPG_ERR_INVALID, "effects is NULL");
    if (!d->surv_table) return fail(SPG_ERR_INVALID, "surv_table is NULL");
    if (d->bin_shift > 31) return fail(SPG_ERR_INVALID, "bin_shift must be <= 31");
    if (!(d->mu >= 0.0 && d->mu < 1.0)) return fail(SPG_ERR_INVALID, "mu must be in [0, 1)");
    if (d->stats_capacity > (1u << 24)) return fail(SPG_ERR_INVALID, "stats_capacity must be <= 2^24");
    if (d->allele_model > 1u) return fail(SPG_ERR_INVALID, "allele_model must be 0 (biallelic) or 1 (continuous)");
    if (d->allele_model == 1u) {
        if (d->map_morgans || d->mother_weights || d->father_weights || d->dominance || d->init_genotypes)
            return fail(SPG_ERR_INVALID, "continuous allelic values take no linkage map, weights, dominance or "
                                         "init_genotypes (use init_values)");
        if (!(d->mut_sd >= 0.0 && d->mut_sd < 64.0) || !(d->env_sd >= 0.0 && d->env_sd < 64.0))
            return fail(SPG_ERR_INVALID, "mut_sd and env_sd must be in [0, 64)");
    }
    return SPG_OK;
}

int build_params(const spg_pop_desc *d, PopParams &prm) {
    std::memset(&prm, 0, sizeof prm);
    std::memcpy(prm.table, d->surv_table, sizeof prm.table);
    effect_planes(d->effects, d->n_loci, prm);
    if (prm.nplanes > (uint32_t)kMaxPlanes) return fail(SPG_ERR_INVALID, "effects span more than 16 bits");
    byte_tables(d->effects, d->n_loci, prm.lut);
    if (d->dominance) {
        offset_planes(d->dominance, d->n_loci, prm.dplanes, prm.d_min, prm.ndplanes);
        if (prm.ndplanes > (uint32_t)kMaxPlanes)
            return fail(SPG_ERR_INVALID, "dominance deviations span more than 16 bits");
        for (uint32_t l = 0; l < d->n_loci; ++l) prm.has_dom |= d->dominance[l] != 0 ? 1u : 0u;
        byte_tables(d->dominance, d->n_loci, prm.dlut);
    }
    prm.kmax = mutation_cdf(d->mu, 2 * d->n_loci, prm.cdf);
    prm.bias = d->bin_bias;
    prm.shift = d->bin_shift;
    prm.n = d->n;
    prm.n_loci = d->n_loci;
    prm.words = d->n_loci / 32;
    prm.key0 = (uint32_t)(d->seed & 0xFFFFFFFFull);
    prm.key1 = (uint32_t)(d->seed >> 32);
    prm.rep = d->replicate;
    prm.has_eco = 0;
    prm.stats_cap = d->stats_capacity ? d->stats_capacity : 1024u;
    prm.linked = d->map_morgans ? 1u : 0u;
    prm.link = nullptr;  // set once the population's memory exists
    prm.weighted = (d->mother_weights || d->father_weights) ? 1u : 0u;
    prm.weights = nullptr;
    prm.continuous = d->allele_model == 1u ? 1u : 0u;
    prm.s_mut = prm.continuous ? (long long)std::floor(d->mut_sd * 256.0 * 65536.0 + 0.5) : 0;
    prm.s_env = prm.continuous ? (long long)std::floor(d->env_sd * 512.0 * 65536.0 + 0.5) : 0;
    return SPG_OK;
}

// Linkage map (Haldane, no interference): w_l = map distance of the linked
// interval between loci l-1 and l (0 where locus l starts a chromosome),
// D = sum w_l; crossover count CDF = Binomial(kLinkSites, D / kLinkSites);
// interval CDF cum[l] = floor(2^32 * (s / D)) with s the running sum of w.
int build_link(const double *map, uint32_t n_loci, LinkParams &lp) {
    std::memset(&lp, 0, sizeof lp);
    double w[kMaxLoci];
    double D = 0.0;
    uint32_t chrom = 0;
    lp.first[0] = 0;
    w[0] = 0.0;
    for (uint32_t l = 1; l < n_loci; ++l) {
        const double m = map[l];
        if (!(m == m) || std::isinf(m)) return fail(SPG_ERR_INVALID, "map_morgans[%u] is not finite", l);
        if (m < 0.0) {
            lp.clast[chrom] = (uint16_t)(l - 1);
            if (++chrom >= (uint32_t)kMaxChrom)
                return fail(SPG_ERR_INVALID, "a linkage map holds at most %d chromosomes", kMaxChrom);
            lp.first[chrom] = (uint16_t)l;
            w[l] = 0.0;
        } else {
            w[l] = m;
        }
        D = D + w[l];
    }
    lp.clast[chrom] = (uint16_t)(n_loci - 1);
    lp.nchrom = chrom + 1;
    if (!(D <= kMaxMapMorgans)) return fail(SPG_ERR_INVALID, "the linkage map is longer than 16 Morgans");
    for (uint32_t c = 0; c < lp.nchrom; ++c)
        for (uint32_t l = lp.first[c]; l <= lp.clast[c]; ++l) lp.chrom[l] = (uint8_t)c;
    lp.kmax = mutation_cdf(D / (double)kLinkSites, kLinkSites, lp.cdf);
    double run = 0.0;
    for (uint32_t l = 0; l < n_loci; ++l) {
        if (D > 0.0) {
            run = run + w[l];
            const double x = (run / D) * 4294967296.0;
            lp.cum[l] = x >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)x;
        } else {
            lp.cum[l] = 0;
        }
    }
    // guide[h]: the interval of the bucket's first uniform, the chromosomes of
    // it and of the next interval, and the interval boundaries inside the
    // bucket (none for most buckets: the guide entry is the answer)
    constexpr uint32_t shift = 32u - (uint32_t)kLinkGuideBits;
    auto interval = [&](uint32_t u) {
        uint32_t I = 0;
        while (I + 1 < n_loci && lp.cum[I] <= u) ++I;
        return I;
    };
    for (uint32_t h = 0; h < (uint32_t)kLinkGuide; ++h) {
        const uint32_t lo = h << shift, hi = lo | ((1u << shift) - 1u);
        const uint32_t I0 = interval(lo), nb = std::min<uint32_t>(interval(hi) - I0, 2u);
        const uint32_t c0 = lp.chrom[I0], c1 = nb != 0u ? lp.chrom[I0 + 1u] : 0u;
        lp.guide[h] = I0 | (c0 << 8) | (c1 << 15) | (nb << 26);
    }
    return SPG_OK;
}

// Weighted parents: t[b] = floor(2^32 * w[b] / max w) (integer arithmetic),
// 0xFFFFFFFF where w[b] is the maximum; a NULL table is uniform.
static int weight_thresholds(const uint32_t *w, uint32_t *acc, const char *role) {
    if (!w) {
        for (int b = 0; b < kBins; ++b) acc[b] = kCertain;
        return SPG_OK;
    }
    uint32_t mx = 0;
    for (int b = 0; b < kBins; ++b) mx = std::max(mx, w[b]);
    if (mx == 0) return fail(SPG_ERR_INVALID, "%s weights are all zero", role);
    for (int b = 0; b < kBins; ++b)
        acc[b] = w[b] == mx ? kCertain : (uint32_t)(((uint64_t)w[b] << 32) / mx);
    return SPG_OK;
}

int build_weights(const uint32_t *mother_w, const uint32_t *father_w, WeightParams &wp) {
    int rc = weight_thresholds(mother_w, wp.acc[0], "mother");
    if (rc == SPG_OK) rc = weight_thresholds(father_w, wp.acc[1], "father");
    return rc;
}

// ------------------------------------------------------------ population
uint32_t bucket_count(uint32_t n) { return (n + kBucket - 1) / kBucket; }

PopLayout layout_for(uint32_t n, uint32_t words, uint32_t nbuckets, uint32_t cap, bool weighted, bool dense) {
    PopLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    L.params = take(sizeof(PopParams));
    L.state = take(sizeof(DevState));
    L.acc = take(sizeof(StatAcc) * kAccCopies);
    L.geno0 = take((size_t)n * 2 * words * 4);
    L.geno1 = take((size_t)n * 2 * words * 4);
    L.dense = dense ? take((size_t)n * 2 * words * 4) : 0;
    L.surv0 = take((size_t)n * 4);
    L.surv1 = take((size_t)n * 4);
    L.alive = take((size_t)nbuckets * kBucketWords * 4);
    L.buckets = take((size_t)2 * nbuckets * 4);
    L.ring = take((size_t)cap * sizeof(spg_stats));
    L.segment = take(sizeof(Segment));
    L.link = take(sizeof(LinkParams));
    L.weighted = weighted;
    if (weighted) {
        L.weights = take(sizeof(WeightParams));
        L.obin = take((size_t)n * 2);
        L.survw = take((size_t)n * 16);
    }
    L.total = off;
    return L;
}

Segment segment_at(char *base, const PopLayout &L, uint32_t n, uint32_t ntiles, uint32_t tile_begin,
                   uint32_t nbuckets, uint32_t bucket_begin) {
    Segment s{};
    s.n = n;
    s.acc = reinterpret_cast<StatAcc *>(base + L.acc);
    s.prm = reinterpret_cast<const PopParams *>(base + L.params);
    s.geno[0] = reinterpret_cast<uint32_t *>(base + L.geno0);
    s.geno[1] = reinterpret_cast<uint32_t *>(base + L.geno1);
    s.dense = L.dense ? reinterpret_cast<uint32_t *>(base + L.dense) : nullptr;
    s.surv[0] = reinterpret_cast<uint32_t *>(base + L.surv0);
    s.surv[1] = reinterpret_cast<uint32_t *>(base + L.surv1);
    s.alive = reinterpret_cast<uint32_t *>(base + L.alive);
    s.bucket_sum = reinterpret_cast<uint32_t *>(base + L.buckets);
    s.state = reinterpret_cast<DevState *>(base + L.state);
    if (L.weighted) {
        s.obin = reinterpret_cast<uint16_t *>(base + L.obin);
        s.survw = reinterpret_cast<unsigned long long *>(base + L.survw);
    }
    s.ring = reinterpret_cast<spg_stats *>(base + L.ring);
    s.tile_begin = tile_begin;
    s.ntiles = ntiles;
    s.bucket_begin = bucket_begin;
    s.nbuckets = nbuckets;
    return s;
}

// Launch shapes the batch autotuner times, per locus count: threads per
// block x offspring per thread for L <= 64, threads per block x lanes per
// offspring for L >= 128.
Shape autotune_candidate(uint32_t words, uint32_t c) {
    static const uint32_t narrow[kAutotuneCandidates][3] = {{128, 1, 1}, {128, 2, 1}, {256, 1, 1},
                                                             {256, 2, 1}, {512, 1, 1}, {512, 2, 1}};
    static const uint32_t wide[kAutotuneCandidates][3] = {{128, 1, 1}, {256, 1, 1}, {512, 1, 1},
                                                           {128, 1, 2}, {256, 1, 2}, {512, 1, 2}};
    const uint32_t(&e)[3] = words >= 4 ? wide[c % kAutotuneCandidates] : narrow[c % kAutotuneCandidates];
    Shape s;
    s.block = e[0];
    s.items = e[1];
    s.lanes = e[2];
    return s;
}

// A caller's launch shape: 0 fields take the defaults of the locus count.
// words 0: the continuous-allele kernel (256 threads, one offspring each).
int shape_from_abi(uint32_t words, const spg_launch_shape *in, Shape &out) {
    if (words == 0) {
        out = Shape{(uint32_t)kBlock, 1u, 1u};
        if ((in->threads_per_block && in->threads_per_block != (uint32_t)kBlock) ||
            (in->items_per_thread && in->items_per_thread != 1u) ||
            (in->lanes_per_offspring && in->lanes_per_offspring != 1u))
            return fail(SPG_ERR_INVALID, "continuous allelic values run 256 threads, one offspring each");
        return SPG_OK;
    }
    out = default_shape(words);
    if (in->threads_per_block) out.block = in->threads_per_block;
    if (in->lanes_per_offspring) out.lanes = in->lanes_per_offspring;
    out.items = in->items_per_thread ? in->items_per_thread : 1u;
    if (!supported_shape(words, out))
        return fail(SPG_ERR_INVALID,
                    "unsupported launch shape (%u threads, %u offspring per thread, %u lanes per offspring) for %u "
                    "loci: threads 128, 256 or 512; L <= 64: 1 lane, 1 or 2 offspring per thread; L >= 128: 1 or 2 "
                    "lanes, 1 offspring",
                    out.block, out.items, out.lanes, 32u * words);
    return SPG_OK;
}

Shape default_shape(uint32_t words) {
    Shape s;
    s.block = 256;
    s.items = 1;
    s.lanes = words == 8 ? 2u : 1u;  // L = 256: a lane per parent record (two records do not fit a thread)
    return s;
}

GraphChain::~GraphChain() { reset(); }

void GraphChain::reset() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    length = 0;
}

// The launches of a generation kernel: grid, block, shared memory, and
// whether it may start while its predecessor finishes (programmatic
// dependent launch: the kernel waits with griddepcontrol.wait before reading
// the predecessor's results).  The continuous-allele kernel does not.
namespace {
struct KernelLaunch {
    void *fn;
    dim3 grid, block;
    unsigned smem;
    bool programmatic;
};
KernelLaunch offspring_launch(const GenLaunch &gl) {
    return {reinterpret_cast<void *>(gl.offspring.fn), dim3(gl.blocks), dim3(gl.offspring.block), gl.offspring.smem,
            gl.offspring.persistent};
}
KernelLaunch compact_launch(const GenLaunch &gl) {
    return {reinterpret_cast<void *>(gl.compact), dim3(gl.buckets), dim3(kCompactThreads), compact_smem(), true};
}
// after the compaction has finished (it reads the committed state)
KernelLaunch locus_launch(const GenLaunch &gl) {
    return {reinterpret_cast<void *>(gl.locus), dim3(gl.la.blocks), dim3(kLocusBlock), 0u, false};
}
}  // namespace

int add_generation_nodes(cudaGraph_t graph, const GenLaunch &gl, void **params, uint32_t len) {
    cudaGraphNode_t prev = nullptr;
    LocusArgs la = gl.la;
    void *locus_params[] = {params[0], &la};  // argument values are copied into the nodes
    const uint32_t per_gen = gl.locus ? 3u : 2u;
    for (uint32_t i = 0; i < per_gen * len; ++i) {
        const uint32_t step = i % per_gen;
        const KernelLaunch k = step == 0 ? offspring_launch(gl) : step == 1 ? compact_launch(gl) : locus_launch(gl);
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeKernel;
        np.kernel.func = k.fn;
        np.kernel.gridDim = k.grid;
        np.kernel.blockDim = k.block;
        np.kernel.sharedMemBytes = k.smem;
        np.kernel.kernelParams = step == 2 ? locus_params : params;
        cudaGraphEdgeData edge{};
        if (k.programmatic) {
            edge.from_port = cudaGraphKernelNodePortProgrammatic;
            edge.type = cudaGraphDependencyTypeProgrammatic;
        }
        cudaGraphNode_t node;
        const cudaError_t e = cudaGraphAddNode(&node, graph, prev ? &prev : nullptr, prev ? &edge : nullptr,
                                               prev ? 1 : 0, &np);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphAddNode");
        prev = node;
    }
    return SPG_OK;
}

// A graph of `len` generations: offspring -> compaction -> offspring -> ...
int GraphChain::build(const GenLaunch &gl, uint32_t len) {
    reset();
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
    GenArgs a = gl.args;
    void *params[] = {&a};
    const int rc = add_generation_nodes(graph, gl, params, len);
    if (rc != SPG_OK) {
        reset();
        return rc;
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        reset();
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    length = len;
    return SPG_OK;
}

int launch_generation(const GenLaunch &gl, cudaStream_t stream) {
    GenArgs a = gl.args;
    void *params[] = {&a};
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    LocusArgs la = gl.la;
    void *locus_params[] = {&a, &la};
    cudaError_t e = cudaSuccess;
    for (uint32_t step = 0; step < (gl.locus ? 3u : 2u); ++step) {
        const KernelLaunch k = step == 0 ? offspring_launch(gl) : step == 1 ? compact_launch(gl) : locus_launch(gl);
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = k.grid;
        cfg.blockDim = k.block;
        cfg.dynamicSmemBytes = k.smem;
        cfg.stream = stream;
        cfg.attrs = &attr;
        cfg.numAttrs = k.programmatic ? 1u : 0u;
        e = cudaLaunchKernelExC(&cfg, k.fn, step == 2 ? locus_params : params);
        if (e != cudaSuccess) break;
    }
    return e == cudaSuccess ? SPG_OK : cuda_fail(e, "generation launch");
}

int enqueue_generations(const GenLaunch &gl, uint32_t n_gen, GraphChain &chain, cudaStream_t stream) {
    if (n_gen == 0 || gl.blocks == 0) return SPG_OK;
    if (n_gen >= kGraphChunk) {
        if (!chain.exec) {
            const int rc = chain.build(gl, kGraphChunk);
            if (rc != SPG_OK) return rc;
        }
        for (uint32_t i = 0; i + kGraphChunk <= n_gen; i += kGraphChunk) {
            const cudaError_t e = cudaGraphLaunch(chain.exec, stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        }
    }
    for (uint32_t i = 0; i < n_gen % kGraphChunk; ++i) {
        const int rc = launch_generation(gl, stream);
        if (rc != SPG_OK) return rc;
    }
    return SPG_OK;
}

// ------------------------------------------------- launch groups
// Bytes of a launch group's table: segments, runs (at most one per member plus
// one per piece: one round of blocks, or pieces of kPieceOffspring offspring
// or more), the blocks' run offsets, the bucket map and the tile map.
size_t group_table_bytes(uint32_t members, uint64_t offspring, uint32_t buckets) {
    const uint64_t runs = 2ull * members + offspring / kPieceOffspring + kMaxGridBlocks + 1ull;
    return align_up((size_t)members * sizeof(Segment), 256) + align_up((size_t)runs * sizeof(Run), 256) +
           align_up((size_t)(kMaxGridBlocks + 1) * 4, 256) + align_up((size_t)buckets * 4, 256) +
           align_up((size_t)(offspring / kBlock + members + 1) * 4, 256);  // tile map (continuous groups)
}

uint32_t tiles_for(uint32_t n, const Shape &shape) {
    const uint32_t t = tile_size(shape);
    return (n + t - 1) / t;
}

// Runs of a launch group (see GenArgs): the members' tiles, in member order,
// with one unit of set-up (tables, pipeline start) before each member, cut
// into P pieces of equal work dealt round-robin to the G blocks (block b
// forms pieces b, b + G, ...: rounds of G pieces of at least min_piece tiles,
// each round a contiguous window of the member list, so the populations being
// formed at any moment are few and their parent records stay in L2 -- the
// flattened replicate loop of Fig. S5 B, scheduled for locality).  A piece is
// one run per member it touches, so every block's work is within a set-up or
// two of the others'.
void schedule_runs(const std::vector<uint32_t> &tiles, uint32_t G, uint32_t min_piece, std::vector<Run> &runs,
                   std::vector<uint32_t> &block_runs) {
    const uint32_t M = (uint32_t)tiles.size();
    std::vector<uint64_t> ustart(M + 1, 0ull), tstart(M + 1, 0ull);  // prefix units, prefix tiles
    for (uint32_t m = 0; m < M; ++m) {
        ustart[m + 1] = ustart[m] + (tiles[m] ? tiles[m] + 1ull : 0ull);
        tstart[m + 1] = tstart[m] + tiles[m];
    }
    const uint64_t U = ustart[M], T = tstart[M];
    // rounds of G pieces of min_piece tiles or more (one round at least)
    const uint64_t P = (uint64_t)G * std::max<uint64_t>(1ull, T / ((uint64_t)G * std::max(1u, min_piece)));
    std::vector<uint64_t> cut(P + 1);  // cut p (0..P) as a flattened tile coordinate
    uint32_t m = 0;
    for (uint64_t p = 0; p < P; ++p) {
        const uint64_t x = U * p / P;
        while (m < M && x >= ustart[m + 1]) ++m;
        const uint64_t off = m < M && x > ustart[m] ? x - ustart[m] - 1ull : 0ull;  // tiles of m before the cut
        cut[p] = m < M ? tstart[m] + std::min<uint64_t>(off, tiles[m]) : T;
    }
    cut[P] = T;
    std::vector<std::vector<Run>> piece_runs(P);
    std::vector<uint32_t> nruns(M, 0u);
    m = 0;
    for (uint64_t p = 0; p < P; ++p) {
        for (uint64_t g = cut[p]; g < cut[p + 1];) {
            while (g >= tstart[m + 1]) ++m;
            const uint64_t e = std::min(cut[p + 1], tstart[m + 1]);
            piece_runs[p].push_back(Run{m, (uint32_t)(g - tstart[m]), (uint32_t)(e - g), nruns[m]++, 0u, {0u, 0u, 0u}});
            g = e;
        }
    }
    runs.clear();
    block_runs.assign(G + 1, 0u);
    for (uint32_t b = 0; b < G; ++b) {
        block_runs[b] = (uint32_t)runs.size();
        for (uint64_t p = b; p < P; p += G)
            for (Run r : piece_runs[p]) {
                r.shares = nruns[r.seg];  // the member's parents prefetched in shares, one per run
                runs.push_back(r);
            }
    }
    block_runs[G] = (uint32_t)runs.size();
}

int build_group_launch(const std::vector<const PopView *> &members, uint32_t words, const Shape &shape, bool eco,
                       bool dom, char *table, size_t table_capacity, GenLaunch &gl, bool linked, bool weighted,
                       bool continuous) {
    if (members.empty()) {
        gl = GenLaunch{};
        return SPG_OK;
    }
    const bool one_shape = linked || weighted || continuous;
    if ((!continuous && !supported_shape(words, shape)) ||
        (one_shape && (shape.block != (uint32_t)kBlock || shape.items != 1u || shape.lanes != 1u)))
        return fail(SPG_ERR_INVALID,
                    "unsupported launch shape (%u threads, %u offspring per thread, %u lanes per offspring) for %u loci",
                    shape.block, shape.items, shape.lanes, continuous ? 2u * words : 32u * words);
    // members in HBM: staged parents (where an instance has them); continuous
    // values (records of 2L int16, words = L / 2): one block per 256 offspring
    OffspringKernel k = continuous ? continuous_kernel(2u * words, members.size() > 1)
                                   : offspring_kernel(words, shape, linked, weighted, eco, dom, true);
    int rc = prepare_offspring(k);
    if (rc != SPG_OK) return fail(rc, "offspring kernel setup failed");
    std::vector<Segment> segs;
    std::vector<uint32_t> tiles, bucket_map, tile_map;
    segs.reserve(members.size());
    uint32_t total_tiles = 0, buckets = 0;
    uint64_t offspring = 0;
    for (uint32_t si = 0; si < members.size(); ++si) {
        const PopView &v = *members[si];
        const uint32_t nt = continuous ? (v.n + kBlock - 1) / kBlock : tiles_for(v.n, shape);
        segs.push_back(segment_at(v.base, v.L, v.n, nt, total_tiles, v.nbuckets, buckets));
        tiles.push_back(nt);
        if (continuous) tile_map.insert(tile_map.end(), nt, si);
        bucket_map.insert(bucket_map.end(), v.nbuckets, si);
        total_tiles += nt;
        buckets += v.nbuckets;
        offspring += v.n;
    }
    const uint32_t G = std::max(1u, std::min(k.resident, kMaxGridBlocks));
    const uint32_t min_piece = std::max(1u, kPieceOffspring / tile_size(shape));
    std::vector<Run> runs;
    std::vector<uint32_t> block_runs;
    if (!continuous) schedule_runs(tiles, G, min_piece, runs, block_runs);
    if (group_table_bytes((uint32_t)segs.size(), offspring, buckets) > table_capacity)
        return fail(SPG_ERR_INVALID, "launch table does not fit its buffer");
    const size_t off_runs = align_up(segs.size() * sizeof(Segment), 256);
    const size_t off_block = off_runs + align_up(runs.size() * sizeof(Run), 256);
    const size_t off_buckets = off_block + align_up((size_t)(kMaxGridBlocks + 1) * 4, 256);
    const size_t off_tiles = off_buckets + align_up((size_t)buckets * 4, 256);
    cudaError_t e = cudaMemcpy(table, segs.data(), segs.size() * sizeof(Segment), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(table + off_runs, runs.data(), runs.size() * sizeof(Run), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(table + off_block, block_runs.data(), block_runs.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(table + off_buckets, bucket_map.data(), bucket_map.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !tile_map.empty())
        e = cudaMemcpy(table + off_tiles, tile_map.data(), tile_map.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload launch table");
    gl = GenLaunch{};
    gl.offspring = k;
    gl.compact = compact_kernel(words);
    gl.args.segs = reinterpret_cast<const Segment *>(table);
    gl.args.runs = reinterpret_cast<const Run *>(table + off_runs);
    gl.args.block_runs = reinterpret_cast<const uint32_t *>(table + off_block);
    gl.args.bucket_seg = reinterpret_cast<const uint32_t *>(table + off_buckets);
    gl.args.tile_seg = reinterpret_cast<const uint32_t *>(table + off_tiles);
    gl.args.nsegs = (uint32_t)segs.size();
    if (segs.size() == 1) {
        // one member: contiguous shares of its tiles per block (no run table)
        gl.args.one = segs[0];
        gl.args.nsegs = 1;
    }
    gl.args.total_tiles = total_tiles;
    gl.args.total_buckets = buckets;
    if (continuous) {
        gl.blocks = total_tiles;  // not persistent
    } else {
        apply_kernel(k, gl.args);
        gl.blocks = segs.size() == 1 ? std::min(total_tiles, G) : G;
    }
    gl.buckets = buckets;
    return SPG_OK;
}

// ------------------------------------------------- one population's memory
int view_sync(const PopView &v) {
    const cudaError_t e = cudaStreamSynchronize(v.stream);
    return e == cudaSuccess ? SPG_OK : cuda_fail(e, "cudaStreamSynchronize");
}

int view_state(const PopView &v, DevState &st) {
    int rc = view_sync(v);
    if (rc != SPG_OK) return rc;
    const cudaError_t e = cudaMemcpy(&st, v.base + v.L.state, sizeof st, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SPG_OK : cuda_fail(e, "read state");
}

int view_set_state(const PopView &v, uint32_t gen, uint32_t S, uint32_t f, double R, int32_t status,
                   uint32_t target) {
    return launch_set_state(reinterpret_cast<DevState *>(v.base + v.L.state),
                            reinterpret_cast<StatAcc *>(v.base + v.L.acc), gen, S, f, R, status, target, v.stream);
}

// Enqueue the generation-0 set-up of one population: parameters, counters,
// founders and state.  `prm` and `init_genotypes` must stay valid until the
// stream has run the copies (callers synchronise before returning).
int view_init(const PopView &v, const PopParams &prm, const uint32_t *init_genotypes, uint32_t p0_q32) {
    cudaError_t e = cudaMemsetAsync(v.base + v.L.buckets, 0, (size_t)2 * v.nbuckets * 4, v.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.base + v.L.ring, 0, (size_t)v.cap * sizeof(spg_stats), v.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(v.base + v.L.params, &prm, sizeof(PopParams), cudaMemcpyHostToDevice, v.stream);
    if (e != cudaSuccess) return cuda_fail(e, "initialise device memory");
    uint32_t *geno0 = reinterpret_cast<uint32_t *>(v.base + v.L.geno0);
    uint32_t *surv0 = reinterpret_cast<uint32_t *>(v.base + v.L.surv0);
    int rc;
    if (init_genotypes) {
        e = cudaMemcpyAsync(geno0, init_genotypes, (size_t)v.n * 2 * v.words * 4, cudaMemcpyHostToDevice, v.stream);
        if (e != cudaSuccess) return cuda_fail(e, "upload founders");
        rc = launch_iota(surv0, v.n, v.stream);
    } else if (prm.continuous) {
        rc = launch_founders_cont(reinterpret_cast<const PopParams *>(v.base + v.L.params), prm.n_loci, geno0, surv0,
                                  v.n, p0_q32, v.stream);
    } else {
        rc = launch_founders(v.words, geno0, surv0, v.n, prm.key0, prm.key1, prm.rep, p0_q32, v.stream);
    }
    if (rc != SPG_OK) return fail(rc, "founder launch failed");
    if (v.L.dense) {  // every founder survives: the dense parents are the founders in index order
        rc = launch_dense_gather(v.words, geno0, nullptr, v.n, reinterpret_cast<uint32_t *>(v.base + v.L.dense),
                                 v.stream);
        if (rc != SPG_OK) return fail(rc, "dense-parent launch failed");
    }
    if (v.L.weighted) {  // every founder is a potential parent, in index order
        rc = launch_survivor_bins(reinterpret_cast<const PopParams *>(v.base + v.L.params), v.words, geno0, nullptr,
                                  v.n, v.n, reinterpret_cast<unsigned long long *>(v.base + v.L.survw), v.stream);
        if (rc != SPG_OK) return fail(rc, "survivor-bin launch failed");
    }
    rc = view_set_state(v, 0, v.n, kCertain, 0.0, SPG_OK, 0xFFFFFFFFu);
    return rc == SPG_OK ? SPG_OK : fail(rc, "state launch failed");
}

int check_ecology(const spg_ecology *eco) {
    if (!eco) return fail(SPG_ERR_INVALID, "ecology is NULL");
    if (!eco->attack) return fail(SPG_ERR_INVALID, "attack table is NULL");
    if (!(eco->K > 0.0) || !(eco->R_half > 0.0) || !(eco->R0 >= 0.0) || !std::isfinite(eco->r) ||
        !std::isfinite(eco->K) || !std::isfinite(eco->R0))
        return fail(SPG_ERR_INVALID, "ecology needs K > 0, R_half > 0, R0 >= 0, finite r");
    if (eco->model > 1u) return fail(SPG_ERR_INVALID, "ecology model must be 0 (logistic) or 1 (Beverton-Holt)");
    if (!(eco->r_sd >= 0.0) || !std::isfinite(eco->r_sd) || (eco->model == 0u && eco->r_sd != 0.0))
        return fail(SPG_ERR_INVALID, "r_sd must be finite, >= 0, and 0 for the logistic resource");
    return SPG_OK;
}

// Attach an ecology: parameters (host copy updated and uploaded, then the
// stream synchronised) and the state's R and f.
int view_set_ecology(const PopView &v, PopParams &prm, const spg_ecology *eco) {
    int rc = check_ecology(eco);
    if (rc != SPG_OK) return rc;
    DevState st;
    rc = view_state(v, st);
    if (rc != SPG_OK) return rc;
    std::memcpy(prm.attack, eco->attack, sizeof prm.attack);
    prm.has_eco = 1;
    prm.eco_model = eco->model;
    prm.r_sd = eco->r_sd;
    prm.r = eco->r;
    prm.K = eco->K;
    prm.R_half = eco->R_half;
    const cudaError_t e =
        cudaMemcpyAsync(v.base + v.L.params, &prm, sizeof(PopParams), cudaMemcpyHostToDevice, v.stream);
    if (e != cudaSuccess) return cuda_fail(e, "upload parameters");
    rc = view_set_state(v, st.gen, st.S, factor_q32_host(eco->R0, eco->R_half), eco->R0, st.status, st.target);
    if (rc != SPG_OK) return rc;
    return view_sync(v);
}

int view_read_stats(const PopView &v, uint32_t first_gen, uint32_t count, spg_stats *out) {
    if (!out && count) return fail(SPG_ERR_INVALID, "NULL argument");
    DevState st;
    int rc = view_state(v, st);
    if (rc != SPG_OK) return rc;
    if (count == 0) return SPG_OK;
    const uint64_t last = (uint64_t)first_gen + count - 1;
    if (first_gen == 0 || last > st.gen || (uint64_t)st.gen - first_gen >= v.cap)
        return fail(SPG_ERR_RANGE, "generations %u..%llu not in the ring (completed %u, capacity %u)", first_gen,
                    (unsigned long long)last, st.gen, v.cap);
    const spg_stats *ring = reinterpret_cast<const spg_stats *>(v.base + v.L.ring);
    for (uint32_t i = 0; i < count;) {
        const uint32_t slot = (first_gen - 1 + i) % v.cap;
        const uint32_t run = std::min(count - i, v.cap - slot);
        const cudaError_t e = cudaMemcpy(out + i, ring + slot, run * sizeof(spg_stats), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "read stats");
        i += run;
    }
    return st.status < 0 ? fail(st.status, "device status %d", st.status) : SPG_OK;
}

uint32_t locus_blocks(uint32_t n) {
    const uint32_t groups = (n + 31u) / 32u, per_block = kLocusGroupsPerWarp * (kLocusBlock / 32u);
    return std::max(1u, std::min(kLocusMaxGrid, (groups + per_block - 1u) / per_block));
}

// Rows of per-locus counts of generations first_gen .. first_gen+count-1
// from a population's ring: counted generations are from .. min(until, the
// current one) and the ring keeps the last la.cap of them.
int read_locus_rows(const LocusArgs &la, uint32_t n_loci, uint32_t from, uint32_t until, const DevState &st,
                    uint32_t first_gen, uint32_t count, uint32_t *out) {
    if (count == 0) return SPG_OK;
    const uint64_t last = (uint64_t)first_gen + count - 1;
    until = std::min(until, st.gen);
    if (first_gen == 0 || first_gen < from || last > until || (uint64_t)st.gen - first_gen >= la.cap)
        return fail(SPG_ERR_RANGE, "per-locus counts of generations %u..%llu not kept (counted %u..%u, capacity %u)",
                    first_gen, (unsigned long long)last, from, until, la.cap);
    const size_t row = n_loci;
    for (uint32_t i = 0; i < count;) {
        const uint32_t slot = (first_gen - 1 + i) % la.cap;
        const uint32_t run = std::min(count - i, la.cap - slot);
        const cudaError_t e = cudaMemcpy(out + (size_t)i * row, la.ring + (size_t)slot * row, run * row * 4u,
                                         cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "read per-locus counts");
        i += run;
    }
    return st.status < 0 ? fail(st.status, "device status %d", st.status) : SPG_OK;
}

int view_read_genotypes(const PopView &v, uint32_t *host, size_t n_words) {
    if (!host) return fail(SPG_ERR_INVALID, "NULL argument");
    const size_t need = (size_t)v.n * 2 * v.words;
    if (n_words < need) return fail(SPG_ERR_INVALID, "buffer holds %zu words, need %zu", n_words, need);
    DevState st;
    int rc = view_state(v, st);
    if (rc != SPG_OK) return rc;
    const char *src = v.base + ((st.gen & 1u) ? v.L.geno1 : v.L.geno0);
    const cudaError_t e = cudaMemcpy(host, src, need * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SPG_OK : cuda_fail(e, "read genotypes");
}

int view_read_survivors(const PopView &v, uint32_t *host, size_t capacity, uint32_t *S) {
    if (!S) return fail(SPG_ERR_INVALID, "NULL argument");
    DevState st;
    int rc = view_state(v, st);
    if (rc != SPG_OK) return rc;
    *S = st.S;
    if (!host) return SPG_OK;
    if (capacity < st.S) return fail(SPG_ERR_INVALID, "buffer holds %zu, need %u", capacity, st.S);
    const char *src = v.base + ((st.gen & 1u) ? v.L.surv1 : v.L.surv0);
    const cudaError_t e = cudaMemcpy(host, src, (size_t)st.S * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SPG_OK : cuda_fail(e, "read survivors");
}

int view_get_state(const PopView &v, spg_state *out) {
    if (!out) return fail(SPG_ERR_INVALID, "NULL argument");
    DevState st;
    const int rc = view_state(v, st);
    if (rc != SPG_OK) return rc;
    out->gen = st.gen;
    out->S = st.S;
    out->status = st.status;
    out->f = st.f;
    out->R = st.R;
    return SPG_OK;
}

}  // namespace spg


using namespace spg;

extern "C" {
uint32_t spg_abi_version(void) { return SPG_ABI_VERSION; }

uint32_t spg_mutation_cdf(double mu, uint32_t n_copies, uint32_t cdf[32]) {
    if (!cdf || !(mu >= 0.0 && mu < 1.0)) return 0;
    return mutation_cdf(mu, n_copies, cdf);
}

const char *spg_last_error(void) { return g_last_error.c_str(); }

const char *spg_status_string(int code) {
    switch (code) {
        case SPG_OK: return "ok";
        case SPG_EXTINCT: return "extinct: no survivors";
        case SPG_ERR_INVALID: return "invalid argument";
        case SPG_ERR_OOM: return "device allocation failed";
        case SPG_ERR_CUDA: return "CUDA runtime error";
        case SPG_ERR_TIMEOUT: return "bounded device wait timed out";
        case SPG_ERR_RANGE: return "generations not available";
        case SPG_ERR_BUDGET: return "memory budget exceeded";
        default: return "unknown status";
    }
}

void spg_summarize(const spg_stats *st, uint32_t n_loci, float out[5]) {
    const double n = (double)st->n;
    const double mean_raw = (double)st->sum_raw / n;
    const double second = (double)st->sum_raw2 / n;
    const double sq = mean_raw * mean_raw;
    const double var_raw = second - sq;
    out[0] = (float)(mean_raw / 512.0);
    out[1] = (float)(var_raw / (512.0 * 512.0));
    out[2] = (float)((double)st->s / n);
    out[3] = (float)((double)st->het / (n * (double)n_loci));
    out[4] = (float)((double)st->allele / (2.0 * n * (double)n_loci));
}

}  // extern "C"
