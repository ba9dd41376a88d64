// C ABI of one population (spg_pop): create, ecology, stepping, reads,
// checkpoint/restore, tiling (see include/spegg.h).
//
// A population owns one device arena (parameters, state, accumulators, two
// genotype buffers, two survivor lists, bitmap, bucket counts, statistics
// ring).  Generations are enqueued as a cached CUDA graph of kGraphChunk
// generations (two launches each); every launch has identical arguments
// because buffers are chosen on the device by generation parity.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "spegg.h"
#include "spegg_engine.h"
#include "spegg_internal.h"

using namespace spg;

struct spg_pop {
    uint32_t n = 0, n_loci = 0, words = 0, ntiles = 0, nbuckets = 0, cap = 0;
    Shape shape;
    uint64_t seed = 0;
    uint32_t rep = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Allocator alloc;
    char *arena = nullptr;
    PopLayout L{};
    PopParams *host_prm = nullptr;  // host copy of the parameters
    LinkParams link{};              // linkage-map tables (when host_prm->linked)
    WeightParams *weights = nullptr;  // parent acceptance thresholds (when host_prm->weighted)
    GenLaunch gl;
    GraphChain chain;
    // per-locus allele counts (off until spg_set_locus_counts): ring, partial
    // rows and counter in one allocation; readable from generation locus_from
    char *locus_mem = nullptr;
    LocusArgs locus{};
    bool locus_on = false;
    uint32_t locus_from = 0, locus_until = 0;  // counted generations: locus_from .. (on ? now : locus_until)

    PopView view() const {
        PopView v;
        v.base = arena;
        v.L = L;
        v.n = n;
        v.words = words;
        v.cap = cap;
        v.nbuckets = nbuckets;
        v.stream = stream;
        return v;
    }
};

namespace {

// The per-locus count kernel after each compaction, or none.
void attach_locus(spg_pop *p) {
    p->gl.locus = p->locus_on ? locus_kernel(p->words) : nullptr;
    p->gl.la = p->locus;
    p->chain.reset();
}

// Point the launch at the population's single segment with a launch shape
// (uploads the device copy of the segment; synchronous).
int configure_launch(spg_pop *p, const Shape &shape) {
    const PopParams &prm = *p->host_prm;
    const bool continuous = prm.continuous != 0u;
    OffspringKernel k;
    if (continuous) {
        if (shape.block != (uint32_t)kBlock || shape.items != 1u)
            return fail(SPG_ERR_INVALID, "continuous allelic values run 256 threads, one offspring each");
        k = continuous_kernel(p->n_loci);
    } else {
        if (!supported_shape(p->words, shape))
            return fail(SPG_ERR_INVALID,
                        "unsupported launch shape (%u threads, %u offspring per thread, %u lanes per offspring) for %u loci",
                        shape.block, shape.items, shape.lanes, p->n_loci);
        if ((prm.linked || prm.weighted) && (shape.block != 256u || shape.items != 1u || shape.lanes != 1u))
            return fail(SPG_ERR_INVALID,
                        "a population with a linkage map or parent weights runs 256 threads, one offspring each");
        k = offspring_kernel(p->words, shape, prm.linked != 0u, prm.weighted != 0u, prm.has_eco != 0u,
                             prm.has_dom != 0u, prm.weighted != 0u || (size_t)p->n * 8u * p->words > kStageParentBytes);
    }
    int rc = prepare_offspring(k);
    if (rc != SPG_OK) return fail(rc, "offspring kernel setup failed");
    p->shape = shape;
    p->ntiles = continuous ? (p->n + kBlock - 1) / kBlock : tiles_for(p->n, shape);
    const Segment seg = segment_at(p->arena, p->L, p->n, p->ntiles, 0, p->nbuckets, 0);
    cudaError_t e = cudaMemcpyAsync(p->arena + p->L.segment, &seg, sizeof seg, cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "upload segment");
    rc = view_sync(p->view());
    if (rc != SPG_OK) return rc;
    p->gl = GenLaunch{};
    p->gl.offspring = k;
    p->gl.compact = compact_kernel(p->words);
    p->gl.args.segs = reinterpret_cast<const Segment *>(p->arena + p->L.segment);
    p->gl.args.one = seg;
    p->gl.args.nsegs = 1;
    p->gl.args.total_tiles = p->ntiles;
    p->gl.args.total_buckets = p->nbuckets;
    if (!continuous) apply_kernel(k, p->gl.args);
    p->gl.blocks = continuous ? p->ntiles : std::min(p->ntiles, k.resident);  // continuous: not persistent
    p->gl.buckets = p->nbuckets;
    attach_locus(p);  // also drops the cached graph
    return SPG_OK;
}

}  // namespace

extern "C" {

int spg_create_population(const spg_pop_desc *desc, const spg_allocator *alloc, void *stream, spg_pop **out) {
    if (!out) return fail(SPG_ERR_INVALID, "out is NULL");
    *out = nullptr;
    int rc = validate_desc(desc);
    if (rc != SPG_OK) return rc;
    spg_pop *p = new (std::nothrow) spg_pop();
    if (!p) return fail(SPG_ERR_OOM, "host allocation failed");
    p->n = desc->n;
    p->n_loci = desc->n_loci;
    // record = 2 * words uint32: bit-packed haplotypes, or 2L int16 values
    p->words = desc->allele_model == 1u ? desc->n_loci / 2 : desc->n_loci / 32;
    p->seed = desc->seed;
    p->rep = desc->replicate;
    p->host_prm = new (std::nothrow) PopParams();
    if (!p->host_prm) {
        delete p;
        return fail(SPG_ERR_OOM, "host allocation failed");
    }
    const bool variant = desc->map_morgans || desc->mother_weights || desc->father_weights;
    const Shape shape =
        (desc->allele_model == 1u || variant) ? Shape{(uint32_t)kBlock, 1u, 1u} : default_shape(p->words);
    rc = build_params(desc, *p->host_prm);
    if (rc != SPG_OK) {
        delete p->host_prm;
        delete p;
        return rc;
    }
    if (desc->map_morgans) rc = build_link(desc->map_morgans, p->n_loci, p->link);
    if (rc == SPG_OK && p->host_prm->weighted) {
        p->weights = new (std::nothrow) WeightParams();
        rc = p->weights ? build_weights(desc->mother_weights, desc->father_weights, *p->weights)
                        : fail(SPG_ERR_OOM, "host allocation failed");
    }
    if (rc != SPG_OK) {
        delete p->weights;
        delete p->host_prm;
        delete p;
        return rc;
    }
    p->cap = p->host_prm->stats_cap;
    p->nbuckets = bucket_count(p->n);
    if (alloc) p->alloc.hooks = *alloc;
    if (stream) {
        p->stream = (cudaStream_t)stream;
    } else {
        const cudaError_t e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete p->host_prm;
            delete p;
            return cuda_fail(e, "cudaStreamCreate");
        }
        p->own_stream = true;
    }
    p->L = layout_for(p->n, p->words, p->nbuckets, p->cap, p->host_prm->weighted != 0u,
                      p->host_prm->continuous == 0u);
    p->arena = static_cast<char *>(p->alloc.alloc(p->L.total, p->stream));
    if (!p->arena) {
        spg_destroy(p);
        return fail(SPG_ERR_OOM, "device allocation of %zu bytes failed", p->L.total);
    }
    if (p->host_prm->linked) {
        p->host_prm->link = reinterpret_cast<const LinkParams *>(p->arena + p->L.link);
        const cudaError_t e =
            cudaMemcpyAsync(p->arena + p->L.link, &p->link, sizeof(LinkParams), cudaMemcpyHostToDevice, p->stream);
        if (e != cudaSuccess) {
            spg_destroy(p);
            return cuda_fail(e, "upload linkage map");
        }
    }
    if (p->host_prm->weighted) {
        p->host_prm->weights = reinterpret_cast<const WeightParams *>(p->arena + p->L.weights);
        const cudaError_t e = cudaMemcpyAsync(p->arena + p->L.weights, p->weights, sizeof(WeightParams),
                                              cudaMemcpyHostToDevice, p->stream);
        if (e != cudaSuccess) {
            spg_destroy(p);
            return cuda_fail(e, "upload parent weights");
        }
    }
    rc = view_init(p->view(), *p->host_prm,
                   desc->allele_model == 1u ? reinterpret_cast<const uint32_t *>(desc->init_values)
                                            : desc->init_genotypes,
                   desc->p0_q32);
    if (rc == SPG_OK) rc = view_sync(p->view());  // the caller's arrays are read before returning
    if (rc == SPG_OK) rc = configure_launch(p, shape);
    if (rc != SPG_OK) {
        spg_destroy(p);
        return rc;
    }
    *out = p;
    return SPG_OK;
}

int spg_set_ecology(spg_pop *p, const spg_ecology *eco) {
    if (!p) return fail(SPG_ERR_INVALID, "population is NULL");
    const int rc = view_set_ecology(p->view(), *p->host_prm, eco);
    if (rc != SPG_OK) return rc;
    // the survival table of the offspring kernel now carries attack rates
    if (!p->host_prm->continuous && !p->gl.offspring.eco_table) return configure_launch(p, p->shape);
    return SPG_OK;
}

int spg_step_generations(spg_pop *p, uint32_t n_gen) {
    if (!p) return fail(SPG_ERR_INVALID, "population is NULL");
    return enqueue_generations(p->gl, n_gen, p->chain, p->stream);
}

int spg_read_stats(spg_pop *p, uint32_t first_gen, uint32_t count, spg_stats *out) {
    if (!p) return fail(SPG_ERR_INVALID, "population is NULL");
    return view_read_stats(p->view(), first_gen, count, out);
}

int spg_set_locus_counts(spg_pop *p, int enable) {
    if (!p) return fail(SPG_ERR_INVALID, "population is NULL");
    if (p->host_prm->continuous) return fail(SPG_ERR_INVALID, "per-locus allele counts are for biallelic populations");
    DevState st;
    int rc = view_state(p->view(), st);  // synchronises: no generation in flight
    if (rc != SPG_OK) return rc;
    if (enable && !p->locus_mem) {
        const uint32_t L = p->n_loci, blocks = locus_blocks(p->n);
        const size_t ring = align_up((size_t)p->cap * L * 4u, 256), row = align_up((size_t)L * 4u, 256);
        p->locus_mem = static_cast<char *>(p->alloc.alloc(ring + row + 256u, p->stream));
        if (!p->locus_mem) return fail(SPG_ERR_OOM, "device allocation of %zu bytes failed", ring + row + 256u);
        p->locus.ring = reinterpret_cast<uint32_t *>(p->locus_mem);
        p->locus.acc = reinterpret_cast<uint32_t *>(p->locus_mem + ring);
        p->locus.done = reinterpret_cast<uint32_t *>(p->locus_mem + ring + row);
        p->locus.last = p->locus.done + 1;
        p->locus.cap = p->cap;
        p->locus.blocks = blocks;
        const cudaError_t e = cudaMemsetAsync(p->locus.acc, 0, row + 8u, p->stream);  // row, counter, last
        if (e != cudaSuccess) return cuda_fail(e, "clear per-locus counts");
    }
    if (enable && !p->locus_on && p->locus_mem) {  // the next generation is counted whatever was counted before
        const cudaError_t e = cudaMemsetAsync(p->locus.last, 0, 4, p->stream);
        if (e != cudaSuccess) return cuda_fail(e, "clear per-locus counts");
    }
    if (enable) {
        if (!p->locus_on) p->locus_from = st.gen + 1u;  // the first generation formed from now on
    } else if (p->locus_on) {
        p->locus_until = st.gen;  // the last generation counted
    }
    p->locus_on = enable != 0;
    attach_locus(p);
    return view_sync(p->view());
}

int spg_read_locus_counts(spg_pop *p, uint32_t first_gen, uint32_t count, uint32_t *out) {
    if (!p) return fail(SPG_ERR_INVALID, "population is NULL");
    if (!out && count) return fail(SPG_ERR_INVALID, "NULL argument");
    if (!p->locus_mem) return fail(SPG_ERR_INVALID, "per-locus allele counts are off");
    DevState st;
    const int rc = view_state(p->view(), st);
    if (rc != SPG_OK) return rc;
    if (count == 0) return SPG_OK;
    return read_locus_rows(p->locus, p->n_loci, p->locus_from, p->locus_on ? st.gen : p->locus_until, st, first_gen,
                           count, out);
}

int spg_read_genotypes(spg_pop *p, uint32_t *host, size_t n_words) {
    if (!p) return fail(SPG_ERR_INVALID, "population is NULL");
    return view_read_genotypes(p->view(), host, n_words);
}

int spg_read_survivors(spg_pop *p, uint32_t *host, size_t capacity, uint32_t *S) {
    if (!p) return fail(SPG_ERR_INVALID, "population is NULL");
    return view_read_survivors(p->view(), host, capacity, S);
}

int spg_get_state(spg_pop *p, spg_state *out) {
    if (!p) return fail(SPG_ERR_INVALID, "population is NULL");
    return view_get_state(p->view(), out);
}

int spg_checkpoint_size(spg_pop *p, size_t *bytes) {
    if (!p || !bytes) return fail(SPG_ERR_INVALID, "NULL argument");
    *bytes = sizeof(CheckpointHeader) + (size_t)p->n * 2 * p->words * 4 + (size_t)p->n * 4;
    return SPG_OK;
}

int spg_checkpoint(spg_pop *p, void *host, size_t capacity) {
    size_t need = 0;
    int rc = spg_checkpoint_size(p, &need);
    if (rc != SPG_OK) return rc;
    if (!host || capacity < need) return fail(SPG_ERR_INVALID, "checkpoint buffer too small (need %zu)", need);
    DevState st;
    rc = view_state(p->view(), st);
    if (rc != SPG_OK) return rc;
    CheckpointHeader h{};
    h.magic = kCheckpointMagic;
    h.version = SPG_ABI_VERSION;
    h.n = p->n;
    h.n_loci = p->n_loci;
    h.gen = st.gen;
    h.S = st.S;
    h.status = st.status;
    h.f = st.f;
    h.R = st.R;
    h.seed = p->seed;
    h.replicate = p->rep;
    char *dst = static_cast<char *>(host);
    std::memcpy(dst, &h, sizeof h);
    const size_t gbytes = (size_t)p->n * 2 * p->words * 4;
    cudaError_t e = cudaMemcpy(dst + sizeof h, p->arena + ((st.gen & 1u) ? p->L.geno1 : p->L.geno0), gbytes,
                               cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(dst + sizeof h + gbytes, p->arena + ((st.gen & 1u) ? p->L.surv1 : p->L.surv0),
                       (size_t)st.S * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SPG_OK : cuda_fail(e, "checkpoint copy");
}

int spg_restore(spg_pop *p, const void *host, size_t bytes) {
    size_t need = 0;
    int rc = spg_checkpoint_size(p, &need);
    if (rc != SPG_OK) return rc;
    if (!host || bytes < sizeof(CheckpointHeader)) return fail(SPG_ERR_INVALID, "checkpoint too small");
    CheckpointHeader h;
    std::memcpy(&h, host, sizeof h);
    if (h.magic != kCheckpointMagic || h.n != p->n || h.n_loci != p->n_loci || h.S > p->n || bytes < need)
        return fail(SPG_ERR_INVALID, "checkpoint does not match this population");
    if ((h.S == 0) != (h.status == SPG_EXTINCT) || h.status < 0)
        return fail(SPG_ERR_INVALID, "checkpoint state is inconsistent");
    const char *src = static_cast<const char *>(host);
    const size_t gbytes = (size_t)p->n * 2 * p->words * 4;
    {
        // survivors index parent records: strictly increasing and < n
        const uint32_t *sv = reinterpret_cast<const uint32_t *>(src + sizeof h + gbytes);
        uint32_t prev = 0;
        for (uint32_t i = 0; i < h.S; ++i) {
            uint32_t v;
            std::memcpy(&v, sv + i, 4);
            if (v >= p->n || (i > 0 && v <= prev)) return fail(SPG_ERR_INVALID, "checkpoint survivor list is invalid");
            prev = v;
        }
    }
    rc = view_sync(p->view());
    if (rc != SPG_OK) return rc;
    cudaError_t e = cudaMemcpy(p->arena + ((h.gen & 1u) ? p->L.geno1 : p->L.geno0), src + sizeof h, gbytes,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->arena + ((h.gen & 1u) ? p->L.surv1 : p->L.surv0), src + sizeof h + gbytes,
                       (size_t)h.S * 4, cudaMemcpyHostToDevice);
    // per-bucket survivor counts of the replaced run must not leak into the
    // generations about to be replayed
    if (e == cudaSuccess) e = cudaMemset(p->arena + p->L.buckets, 0, (size_t)2 * p->nbuckets * 4);
    if (e != cudaSuccess) return cuda_fail(e, "restore copy");
    if (p->L.dense) {  // the restored survivors' records in rank order: the next generation's parents
        const uint32_t par = h.gen & 1u;
        rc = launch_dense_gather(p->words, reinterpret_cast<const uint32_t *>(p->arena + (par ? p->L.geno1 : p->L.geno0)),
                                 reinterpret_cast<const uint32_t *>(p->arena + (par ? p->L.surv1 : p->L.surv0)), h.S,
                                 reinterpret_cast<uint32_t *>(p->arena + p->L.dense), p->stream);
        if (rc != SPG_OK) return fail(rc, "dense-parent launch failed");
    }
    if (p->host_prm->weighted) {  // the restored survivors' bins, from their records
        const uint32_t par = h.gen & 1u;
        rc = launch_survivor_bins(reinterpret_cast<const PopParams *>(p->arena + p->L.params), p->words,
                                  reinterpret_cast<const uint32_t *>(p->arena + (par ? p->L.geno1 : p->L.geno0)),
                                  reinterpret_cast<const uint32_t *>(p->arena + (par ? p->L.surv1 : p->L.surv0)), h.S,
                                  p->n, reinterpret_cast<unsigned long long *>(p->arena + p->L.survw), p->stream);
        if (rc != SPG_OK) return fail(rc, "survivor-bin launch failed");
    }
    rc = view_set_state(p->view(), h.gen, h.S, h.f, h.R, h.status, 0xFFFFFFFFu);
    if (rc != SPG_OK) return rc;
    p->locus_from = h.gen + 1u;  // counts of the restored run start with its next generation
    p->locus_until = h.gen;
    if (p->locus_mem) {  // that generation is counted even if a generation of that number was before
        const cudaError_t e = cudaMemsetAsync(p->locus.last, 0, 4, p->stream);
        if (e != cudaSuccess) return cuda_fail(e, "clear per-locus counts");
    }
    return view_sync(p->view());
}

int spg_set_tiling(spg_pop *p, uint32_t items) {
    spg_launch_shape sh{256u, items, 1u};
    return spg_set_launch_shape(p, &sh);
}

int spg_get_tiling(spg_pop *p, uint32_t *items) {
    if (!p || !items) return fail(SPG_ERR_INVALID, "NULL argument");
    *items = p->shape.items;
    return SPG_OK;
}

int spg_set_launch_shape(spg_pop *p, const spg_launch_shape *shape) {
    if (!p || !shape) return fail(SPG_ERR_INVALID, "NULL argument");
    Shape sh;
    int rc = shape_from_abi(p->host_prm->continuous ? 0u : p->words, shape, sh);
    if (rc != SPG_OK) return rc;
    rc = view_sync(p->view());
    if (rc != SPG_OK) return rc;
    return configure_launch(p, sh);
}

int spg_get_launch_shape(spg_pop *p, spg_launch_shape *out) {
    if (!p || !out) return fail(SPG_ERR_INVALID, "NULL argument");
    out->threads_per_block = p->gl.offspring.block;
    out->items_per_thread = p->gl.offspring.items;
    out->lanes_per_offspring = p->gl.offspring.lanes;
    return SPG_OK;
}

int spg_synchronize(spg_pop *p) {
    if (!p) return fail(SPG_ERR_INVALID, "population is NULL");
    return view_sync(p->view());
}

void spg_destroy(spg_pop *p) {
    if (!p) return;
    if (p->stream) cudaStreamSynchronize(p->stream);
    p->chain.reset();
    if (p->locus_mem) p->alloc.release(p->locus_mem, p->stream);
    if (p->arena) p->alloc.release(p->arena, p->stream);
    if (p->stream) cudaStreamSynchronize(p->stream);
    if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
    delete p->weights;
    delete p->host_prm;
    delete p;
}

}  // extern "C"
