// Batched replicates (spg_batch): many independent populations advanced by
// shared launches -- the flattened replicate loop of the paper's Fig. S5 B.
//
// Members are grouped by locus count and variant (the offspring kernel is
// specialised on W, linkage map and parent weights, and continuous values
// have a kernel of their own; members with a linkage map, parent weights or
// continuous values run at the variant shape, the others' shape is tuned per
// locus count).  A group's members are the segments of one launch: every
// generation is one offspring launch and one compaction launch per group,
// the groups' chains are independent branches of one CUDA graph (so groups
// overlap on the GPU), and the graph of kGraphChunk generations is replayed.
// Each member keeps its own parameters, state, buffers and statistics ring,
// and its Philox counters carry its own replicate id, so a member's results
// are identical to the same population stepped alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <memory>
#include <new>
#include <vector>

#include "spegg.h"
#include "spegg_engine.h"
#include "spegg_internal.h"

using namespace spg;

namespace {

struct Member {
    PopView v;
    std::unique_ptr<PopParams> prm;
    std::unique_ptr<LinkParams> link;       // linkage-map tables (host copy, until uploaded)
    std::unique_ptr<WeightParams> weights;  // parent acceptance thresholds (host copy, until uploaded)
    uint32_t group = 0;
    LocusArgs locus{};                      // per-locus counts (when the batch counts them)
    uint32_t locus_from = 0, locus_until = 0;  // generations counted: from .. (on ? now : until)
};

struct Group {
    uint32_t words = 0;
    bool linked = false, weighted = false, continuous = false;  // the members' variant
    Shape shape;
    std::vector<uint32_t> members;
    size_t table_off = 0, table_bytes = 0;  // launch table in the batch arena (sized for every shape)
    GenLaunch gl;
    LocusArgs locus{};  // the group's per-locus count launch (several members: member table and block map)
};

// A graph of `len` generations for every group: one dependent chain of
// (offspring, compaction) launches per group, chains independent.
struct MultiChain {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~MultiChain() { reset(); }
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
    int build(const std::vector<Group> &groups, uint32_t len) {
        reset();
        cudaError_t e = cudaGraphCreate(&graph, 0);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
        for (const Group &g : groups) {
            if (g.members.empty() || g.gl.blocks == 0) continue;
            GenArgs a = g.gl.args;  // copied into the node parameters
            void *params[] = {&a};
            const int rc = add_generation_nodes(graph, g.gl, params, len);
            if (rc != SPG_OK) {
                reset();
                return rc;
            }
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) {
            reset();
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        return SPG_OK;
    }
};

uint32_t group_of_words(uint32_t words) { return words == 1 ? 0u : words == 2 ? 1u : words == 4 ? 2u : 3u; }

// Groups 0-3: plain members by locus count (L = 32, 64, 128, 256);
// 4 + 4v + that index: variant v (0: linkage map, 1: parent weights, 2: both);
// 16 + that index: continuous values.
constexpr uint32_t kBatchGroups = 20;
uint32_t group_index(uint32_t n_loci, bool linked, bool weighted, bool continuous) {
    const uint32_t l = group_of_words(n_loci / 32);
    return continuous ? 16u + l : l + 4u * ((linked ? 1u : 0u) + (weighted ? 2u : 0u));
}
Shape group_shape(const Group &g) {
    return (g.linked || g.weighted || g.continuous) ? Shape{(uint32_t)kBlock, 1u, 1u} : default_shape(g.words);
}

}  // namespace

struct spg_batch {
    std::vector<Member> members;
    std::vector<Group> groups;  // indexed by group_index
    Allocator alloc;
    char *arena = nullptr;
    size_t arena_bytes = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::map<uint32_t, std::unique_ptr<MultiChain>> chains;  // by length
    char *locus_mem = nullptr;  // per-locus counts: every member's ring, row and counters, the groups' tables
    bool locus_on = false;
};

namespace {

// (Re)build a group's launch table for a launch shape (synchronous upload).
// The per-locus count launch after each of the group's compactions, or none
// (counts off, continuous values).  One member: its own arguments (the
// launch's segment is the member); several: the group's member table.
void attach_group_locus(spg_batch *b, Group &g) {
    g.gl.locus = nullptr;
    g.gl.la = LocusArgs{};
    if (!b->locus_on || g.continuous || g.members.empty()) return;
    const bool several = g.members.size() > 1;
    g.gl.locus = locus_kernel(g.words, several);
    g.gl.la = several ? g.locus : b->members[g.members[0]].locus;
    if (!several) g.gl.la.first = 0u;
}

int configure_group(spg_batch *b, Group &g, const Shape &shape) {
    if (g.members.empty()) return SPG_OK;
    std::vector<const PopView *> views;
    views.reserve(g.members.size());
    bool eco = false, dom = false;
    for (uint32_t mi : g.members) {
        views.push_back(&b->members[mi].v);
        eco |= b->members[mi].prm->has_eco != 0u;
        dom |= b->members[mi].prm->has_dom != 0u;
    }
    const int rc = build_group_launch(views, g.words, shape, eco, dom, b->arena + g.table_off, g.table_bytes, g.gl,
                                      g.linked, g.weighted, g.continuous);
    if (rc != SPG_OK) return rc;
    g.shape = shape;
    attach_group_locus(b, g);
    b->chains.clear();
    return SPG_OK;
}

int member_view(spg_batch *b, uint32_t member, PopView &v) {
    if (!b) return fail(SPG_ERR_INVALID, "batch is NULL");
    if (member >= b->members.size()) return fail(SPG_ERR_INVALID, "member %u out of range", member);
    v = b->members[member].v;
    return SPG_OK;
}

int run_chunk(spg_batch *b, uint32_t len) {
    auto it = b->chains.find(len);
    if (it == b->chains.end()) {
        std::unique_ptr<MultiChain> c(new (std::nothrow) MultiChain());
        if (!c) return fail(SPG_ERR_OOM, "host allocation failed");
        const int rc = c->build(b->groups, len);
        if (rc != SPG_OK) return rc;
        it = b->chains.emplace(len, std::move(c)).first;
    }
    const cudaError_t e = cudaGraphLaunch(it->second->exec, b->stream);
    return e == cudaSuccess ? SPG_OK : cuda_fail(e, "cudaGraphLaunch");
}

}  // namespace

extern "C" {

int spg_batch_create(const spg_pop_desc *descs, uint32_t count, const spg_allocator *alloc, void *stream,
                     spg_batch **out) {
    if (!out) return fail(SPG_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!descs || count == 0) return fail(SPG_ERR_INVALID, "a batch needs at least one population");
    for (uint32_t i = 0; i < count; ++i) {
        const int rc = validate_desc(descs + i);
        if (rc != SPG_OK) return fail(rc, "member %u: %s", i, spg_last_error());
    }
    std::unique_ptr<spg_batch> b(new (std::nothrow) spg_batch());
    if (!b) return fail(SPG_ERR_OOM, "host allocation failed");
    b->members.resize(count);
    b->groups.resize(kBatchGroups);
    for (uint32_t gi = 0; gi < kBatchGroups; ++gi) {
        Group &g = b->groups[gi];
        g.continuous = gi >= 16u;
        g.words = g.continuous ? (32u << (gi % 4u)) / 2u : 1u << (gi % 4u);
        g.linked = !g.continuous && ((gi / 4u) & 1u) != 0u;
        g.weighted = !g.continuous && ((gi / 4u) & 2u) != 0u;
    }
    size_t off = 0;
    for (uint32_t i = 0; i < count; ++i) {
        Member &m = b->members[i];
        const spg_pop_desc &d = descs[i];
        m.prm.reset(new (std::nothrow) PopParams());
        if (!m.prm) return fail(SPG_ERR_OOM, "host allocation failed");
        const bool continuous = d.allele_model == 1u;
        const uint32_t words = continuous ? d.n_loci / 2 : d.n_loci / 32;  // record words per haplotype
        int rc = build_params(&d, *m.prm);
        const bool linked = m.prm->linked != 0u, weighted = m.prm->weighted != 0u;
        if (rc == SPG_OK && linked) {
            m.link.reset(new (std::nothrow) LinkParams());
            rc = m.link ? build_link(d.map_morgans, d.n_loci, *m.link) : fail(SPG_ERR_OOM, "host allocation failed");
        }
        if (rc == SPG_OK && weighted) {
            m.weights.reset(new (std::nothrow) WeightParams());
            rc = m.weights ? build_weights(d.mother_weights, d.father_weights, *m.weights)
                           : fail(SPG_ERR_OOM, "host allocation failed");
        }
        if (rc != SPG_OK) return fail(rc, "member %u: %s", i, spg_last_error());
        m.v.n = d.n;
        m.v.words = words;
        m.v.cap = m.prm->stats_cap;
        m.v.nbuckets = bucket_count(d.n);
        m.v.L = layout_for(d.n, words, m.v.nbuckets, m.v.cap, weighted, !continuous);
        m.group = group_index(d.n_loci, linked, weighted, continuous);
        b->groups[m.group].members.push_back(i);
        m.v.base = reinterpret_cast<char *>(off);  // offset until the arena exists
        off = align_up(off + m.v.L.total, 256);
    }
    for (Group &g : b->groups) {
        if (g.members.empty()) continue;
        uint64_t offspring = 0;
        uint32_t buckets = 0;
        for (uint32_t mi : g.members) {
            offspring += b->members[mi].v.n;
            buckets += b->members[mi].v.nbuckets;
        }
        g.table_off = off;
        g.table_bytes = group_table_bytes((uint32_t)g.members.size(), offspring, buckets);
        off = align_up(off + g.table_bytes, 256);
    }
    b->arena_bytes = off;
    if (alloc) b->alloc.hooks = *alloc;
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        const cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        b->own_stream = true;
    }
    b->arena = static_cast<char *>(b->alloc.alloc(b->arena_bytes, b->stream));
    if (!b->arena) {
        spg_batch_destroy(b.release());
        return fail(SPG_ERR_OOM, "device allocation of %zu bytes failed", b->arena_bytes);
    }
    for (uint32_t i = 0; i < count; ++i) {
        Member &m = b->members[i];
        m.v.base = b->arena + reinterpret_cast<size_t>(m.v.base);
        m.v.stream = b->stream;
        cudaError_t e = cudaSuccess;
        if (m.link) {  // the variant tables in the member's memory (read by its parameters)
            m.prm->link = reinterpret_cast<const LinkParams *>(m.v.base + m.v.L.link);
            e = cudaMemcpyAsync(m.v.base + m.v.L.link, m.link.get(), sizeof(LinkParams), cudaMemcpyHostToDevice,
                                b->stream);
        }
        if (e == cudaSuccess && m.weights) {
            m.prm->weights = reinterpret_cast<const WeightParams *>(m.v.base + m.v.L.weights);
            e = cudaMemcpyAsync(m.v.base + m.v.L.weights, m.weights.get(), sizeof(WeightParams),
                                cudaMemcpyHostToDevice, b->stream);
        }
        if (e != cudaSuccess) {
            spg_batch_destroy(b.release());
            return cuda_fail(e, "upload a member's variant tables");
        }
        const int rc = view_init(m.v, *m.prm,
                                 descs[i].allele_model == 1u ? reinterpret_cast<const uint32_t *>(descs[i].init_values)
                                                             : descs[i].init_genotypes,
                                 descs[i].p0_q32);
        if (rc != SPG_OK) {
            spg_batch *raw = b.release();
            spg_batch_destroy(raw);
            return rc;
        }
    }
    int rc = view_sync(b->members[0].v);  // caller arrays and host parameters have been read
    for (Group &g : b->groups)
        if (rc == SPG_OK) rc = configure_group(b.get(), g, group_shape(g));
    if (rc != SPG_OK) {
        spg_batch_destroy(b.release());
        return rc;
    }
    *out = b.release();
    return SPG_OK;
}

int spg_batch_set_ecology(spg_batch *b, uint32_t member, const spg_ecology *eco) {
    PopView v;
    int rc = member_view(b, member, v);
    if (rc != SPG_OK) return rc;
    rc = view_set_ecology(v, *b->members[member].prm, eco);
    if (rc != SPG_OK) return rc;
    // the group's survival tables now carry attack rates
    Group &g = b->groups[b->members[member].group];
    if (!g.gl.offspring.eco_table) rc = configure_group(b, g, g.shape);
    return rc;
}

int spg_batch_step(spg_batch *b, uint32_t n_gen) {
    if (!b) return fail(SPG_ERR_INVALID, "batch is NULL");
    for (uint32_t i = 0; i + kGraphChunk <= n_gen; i += kGraphChunk) {
        const int rc = run_chunk(b, kGraphChunk);
        if (rc != SPG_OK) return rc;
    }
    if (n_gen % kGraphChunk) return run_chunk(b, n_gen % kGraphChunk);
    return SPG_OK;
}

int spg_batch_set_tiling(spg_batch *b, uint32_t n_loci, uint32_t items) {
    spg_launch_shape sh{256u, items, 1u};
    return spg_batch_set_launch_shape(b, n_loci, &sh);
}

int spg_batch_get_tiling(spg_batch *b, uint32_t n_loci, uint32_t *items) {
    if (!items) return fail(SPG_ERR_INVALID, "NULL argument");
    spg_launch_shape sh{};
    const int rc = spg_batch_get_launch_shape(b, n_loci, &sh);
    if (rc == SPG_OK) *items = sh.items_per_thread;
    return rc;
}

int spg_batch_set_launch_shape(spg_batch *b, uint32_t n_loci, const spg_launch_shape *shape) {
    if (!b || !shape) return fail(SPG_ERR_INVALID, "NULL argument");
    if (!(n_loci == 32 || n_loci == 64 || n_loci == 128 || n_loci == 256))
        return fail(SPG_ERR_INVALID, "n_loci must be 32, 64, 128 or 256");
    const uint32_t words = n_loci / 32;
    Shape sh;
    int rc = shape_from_abi(words, shape, sh);
    if (rc != SPG_OK) return rc;
    rc = view_sync(b->members[0].v);
    if (rc != SPG_OK) return rc;
    return configure_group(b, b->groups[group_of_words(words)], sh);
}

int spg_batch_get_launch_shape(spg_batch *b, uint32_t n_loci, spg_launch_shape *out) {
    if (!b || !out) return fail(SPG_ERR_INVALID, "NULL argument");
    if (!(n_loci == 32 || n_loci == 64 || n_loci == 128 || n_loci == 256))
        return fail(SPG_ERR_INVALID, "n_loci must be 32, 64, 128 or 256");
    const Group &g = b->groups[group_of_words(n_loci / 32)];
    out->threads_per_block = g.members.empty() ? g.shape.block : g.gl.offspring.block;
    out->items_per_thread = g.members.empty() ? g.shape.items : g.gl.offspring.items;
    out->lanes_per_offspring = g.members.empty() ? g.shape.lanes : g.gl.offspring.lanes;
    return SPG_OK;
}

int spg_batch_autotune(spg_batch *b, uint32_t gens_per_trial, spg_autotune_report *report) {
    if (!b || gens_per_trial == 0) return fail(SPG_ERR_INVALID, "batch is NULL or no trial generations");
    cudaEvent_t t0, t1;
    if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess)
        return fail(SPG_ERR_CUDA, "cudaEventCreate");
    int rc = SPG_OK;
    spg_autotune_report rep{};
    // every group runs the same number of trials (kAutotuneCandidates), each
    // one untimed generation (the new shape's first launches) then
    // gens_per_trial timed ones, so all members advance equally
    for (uint32_t gi = 0; gi < 4u && rc == SPG_OK; ++gi) {  // the plain groups (variants: one shape)
        Group &g = b->groups[gi];
        if (g.members.empty()) continue;
        float best_ms = 0.f, worst_ms = 0.f;
        Shape best = g.shape;
        for (uint32_t c = 0; c < kAutotuneCandidates && rc == SPG_OK; ++c) {
            const Shape cand = autotune_candidate(g.words, c);
            rc = configure_group(b, g, cand);
            if (rc == SPG_OK) rc = launch_generation(g.gl, b->stream);
            if (rc != SPG_OK) break;
            cudaEventRecord(t0, b->stream);
            for (uint32_t i = 0; i < gens_per_trial && rc == SPG_OK; ++i) rc = launch_generation(g.gl, b->stream);
            cudaEventRecord(t1, b->stream);
            if (cudaEventSynchronize(t1) != cudaSuccess) rc = fail(SPG_ERR_CUDA, "trial timing");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, t0, t1);
            if (c == 0 || ms < best_ms) {
                best_ms = ms;
                best = cand;
            }
            worst_ms = std::max(worst_ms, ms);
        }
        if (rc == SPG_OK) rc = configure_group(b, g, best);
        if (rc == SPG_OK) {
            rep.groups[gi].threads_per_block = g.gl.offspring.block;
            rep.groups[gi].items_per_thread = g.gl.offspring.items;
            rep.groups[gi].lanes_per_offspring = g.gl.offspring.lanes;
            rep.best_ms[gi] = best_ms / (float)gens_per_trial;
            rep.worst_ms[gi] = worst_ms / (float)gens_per_trial;
        }
    }
    // members with a linkage map, parent weights or continuous values keep the
    // variant shape and advance by as many generations as the tuned ones
    for (uint32_t gi = 4; gi < (uint32_t)b->groups.size() && rc == SPG_OK; ++gi) {
        const Group &g = b->groups[gi];
        if (g.members.empty()) continue;
        for (uint32_t i = 0; i < kAutotuneCandidates * (gens_per_trial + 1u) && rc == SPG_OK; ++i)
            rc = launch_generation(g.gl, b->stream);
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    rep.gens_run = kAutotuneCandidates * (gens_per_trial + 1);
    if (rc == SPG_OK && report) *report = rep;
    return rc;
}

int spg_batch_read_stats(spg_batch *b, uint32_t member, uint32_t first_gen, uint32_t count, spg_stats *out) {
    PopView v;
    const int rc = member_view(b, member, v);
    return rc != SPG_OK ? rc : view_read_stats(v, first_gen, count, out);
}

int spg_batch_set_locus_counts(spg_batch *b, int enable) {
    if (!b) return fail(SPG_ERR_INVALID, "batch is NULL");
    cudaError_t e = cudaStreamSynchronize(b->stream);  // no generation in flight
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    const uint32_t M = (uint32_t)b->members.size();
    if (enable && !b->locus_mem) {
        // layout: every biallelic member's ring and row, the members' counter
        // pairs (blocks done, last generation counted), each group's tables
        size_t off = 0;
        std::vector<size_t> ring_off(M, 0), row_off(M, 0);
        for (uint32_t m = 0; m < M; ++m) {
            const Member &mb = b->members[m];
            if (mb.prm->continuous) continue;
            ring_off[m] = off;
            off = align_up(off + (size_t)mb.v.cap * 32u * mb.v.words * 4u, 256);
            row_off[m] = off;
            off = align_up(off + (size_t)32u * mb.v.words * 4u, 256);
        }
        const size_t counters = off;
        off = align_up(off + (size_t)M * 8u, 256);
        std::vector<size_t> args_off(b->groups.size(), 0), map_off(b->groups.size(), 0);
        std::vector<uint32_t> group_blocks(b->groups.size(), 0);
        for (uint32_t gi = 0; gi < (uint32_t)b->groups.size(); ++gi) {
            const Group &g = b->groups[gi];
            if (g.continuous || g.members.size() < 2) continue;
            for (uint32_t mi : g.members) group_blocks[gi] += locus_blocks(b->members[mi].v.n);
            args_off[gi] = off;
            off = align_up(off + g.members.size() * sizeof(LocusArgs), 256);
            map_off[gi] = off;
            off = align_up(off + (size_t)group_blocks[gi] * 4u, 256);
        }
        b->locus_mem = static_cast<char *>(b->alloc.alloc(off, b->stream));
        if (!b->locus_mem) return fail(SPG_ERR_OOM, "device allocation of %zu bytes failed", off);
        e = cudaMemsetAsync(b->locus_mem, 0, off, b->stream);  // rows and counters start at zero
        for (uint32_t m = 0; m < M && e == cudaSuccess; ++m) {
            Member &mb = b->members[m];
            if (mb.prm->continuous) continue;
            LocusArgs &la = mb.locus;
            la.ring = reinterpret_cast<uint32_t *>(b->locus_mem + ring_off[m]);
            la.acc = reinterpret_cast<uint32_t *>(b->locus_mem + row_off[m]);
            la.done = reinterpret_cast<uint32_t *>(b->locus_mem + counters) + 2u * m;
            la.last = la.done + 1;
            la.cap = mb.v.cap;
            la.blocks = locus_blocks(mb.v.n);
        }
        for (uint32_t gi = 0; gi < (uint32_t)b->groups.size() && e == cudaSuccess; ++gi) {
            Group &g = b->groups[gi];
            if (g.continuous || g.members.size() < 2) continue;
            std::vector<LocusArgs> args;
            std::vector<uint32_t> map;
            for (uint32_t k = 0; k < (uint32_t)g.members.size(); ++k) {
                LocusArgs la = b->members[g.members[k]].locus;
                la.first = (uint32_t)map.size();
                map.insert(map.end(), la.blocks, k);  // k: the member's segment in the group's launch
                args.push_back(la);
            }
            e = cudaMemcpy(b->locus_mem + args_off[gi], args.data(), args.size() * sizeof(LocusArgs),
                           cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(b->locus_mem + map_off[gi], map.data(), map.size() * 4u, cudaMemcpyHostToDevice);
            g.locus = LocusArgs{};
            g.locus.blocks = (uint32_t)map.size();
            g.locus.member = reinterpret_cast<const LocusArgs *>(b->locus_mem + args_off[gi]);
            g.locus.block_member = reinterpret_cast<const uint32_t *>(b->locus_mem + map_off[gi]);
        }
        if (e != cudaSuccess) return cuda_fail(e, "set up per-locus counts");
    }
    for (uint32_t m = 0; m < M; ++m) {
        Member &mb = b->members[m];
        if (mb.prm->continuous || !b->locus_mem) continue;
        DevState st;
        const int rc = view_state(mb.v, st);
        if (rc != SPG_OK) return rc;
        if (enable && !b->locus_on) {
            mb.locus_from = st.gen + 1u;  // the first generation formed from now on
            e = cudaMemsetAsync(mb.locus.last, 0, 4, b->stream);
            if (e != cudaSuccess) return cuda_fail(e, "clear per-locus counts");
        } else if (!enable && b->locus_on) {
            mb.locus_until = st.gen;  // the last generation counted
        }
    }
    b->locus_on = enable != 0;
    for (Group &g : b->groups) attach_group_locus(b, g);
    b->chains.clear();
    e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? SPG_OK : cuda_fail(e, "cudaStreamSynchronize");
}

int spg_batch_read_locus_counts(spg_batch *b, uint32_t member, uint32_t first_gen, uint32_t count, uint32_t *out) {
    PopView v;
    int rc = member_view(b, member, v);
    if (rc != SPG_OK) return rc;
    if (!out && count) return fail(SPG_ERR_INVALID, "NULL argument");
    const Member &mb = b->members[member];
    if (mb.prm->continuous) return fail(SPG_ERR_INVALID, "per-locus allele counts are for biallelic members");
    if (!b->locus_mem) return fail(SPG_ERR_INVALID, "per-locus allele counts are off");
    DevState st;
    rc = view_state(v, st);
    if (rc != SPG_OK) return rc;
    return read_locus_rows(mb.locus, 32u * v.words, mb.locus_from, b->locus_on ? st.gen : mb.locus_until, st,
                           first_gen, count, out);
}

int spg_batch_read_genotypes(spg_batch *b, uint32_t member, uint32_t *host, size_t n_words) {
    PopView v;
    const int rc = member_view(b, member, v);
    return rc != SPG_OK ? rc : view_read_genotypes(v, host, n_words);
}

int spg_batch_read_survivors(spg_batch *b, uint32_t member, uint32_t *host, size_t capacity, uint32_t *S) {
    PopView v;
    const int rc = member_view(b, member, v);
    return rc != SPG_OK ? rc : view_read_survivors(v, host, capacity, S);
}

int spg_batch_get_state(spg_batch *b, uint32_t member, spg_state *out) {
    PopView v;
    const int rc = member_view(b, member, v);
    return rc != SPG_OK ? rc : view_get_state(v, out);
}

int spg_batch_synchronize(spg_batch *b) {
    if (!b) return fail(SPG_ERR_INVALID, "batch is NULL");
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? SPG_OK : cuda_fail(e, "cudaStreamSynchronize");
}

uint32_t spg_batch_size(const spg_batch *b) { return b ? (uint32_t)b->members.size() : 0u; }

void spg_batch_destroy(spg_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    b->chains.clear();
    if (b->locus_mem) b->alloc.release(b->locus_mem, b->stream);
    if (b->arena) b->alloc.release(b->arena, b->stream);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
