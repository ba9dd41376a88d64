// Served jobs (spg_server): continuous batching of independent populations.
//
// Jobs (one population each, with its own generation count) arrive over
// time.  A scheduling tick
//   1. retires resident jobs that reached their generation count (their
//      statistics are copied to host memory and their device memory freed),
//   2. admits queued jobs in arrival order while a resident slot is free and
//      the job's device footprint fits the memory budget,
//   3. rebuilds the launch tables when the resident set changed, and
//   4. advances every resident job by up to gens_per_tick generations in
//      shared launches (one offspring + one compaction launch per locus-count
//      group and generation; groups on their own streams, so they overlap).
// A job stops at its own generation count on the device (the state's target),
// so jobs of any length share launches; its Philox counters carry its own
// replicate id, so its results are identical alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <memory>
#include <new>
#include <thread>
#include <vector>

#include "spegg.h"
#include "spegg_engine.h"
#include "spegg_internal.h"

using namespace spg;

namespace {

// Groups by locus count (L = 32, 64, 128, 256: index 0-3) and variant: the
// index for plain jobs, 4 + 4v + index for v = 0 linkage map, 1 parent
// weights, 2 both, 16 + index for continuous values (variants: one shape).
constexpr int kGroups = 20;

struct Job {
    spg_pop_desc desc{};
    std::vector<int16_t> effects, dominance;
    std::vector<uint32_t> table, founders, attack;
    std::unique_ptr<LinkParams> link;       // linkage-map tables (built at submission)
    std::unique_ptr<WeightParams> weights;  // parent acceptance thresholds (built at submission)
    bool has_eco = false;
    spg_ecology eco{};
    uint32_t n_gen = 0;
    double t_arrival = 0, t_admit = -1, t_finish = -1;
    uint32_t state = SPG_JOB_QUEUED;
    // while resident
    char *arena = nullptr;
    size_t footprint = 0;
    PopView v;
    std::unique_ptr<PopParams> prm;
    uint32_t gen = 0;  // generations enqueued (host bookkeeping)
    // once finished
    std::vector<spg_stats> stats;
    int32_t status = SPG_OK;
    uint32_t final_gen = 0;
};

uint32_t group_of(uint32_t n_loci, bool linked, bool weighted, bool continuous) {
    const uint32_t l = n_loci == 32 ? 0u : n_loci == 64 ? 1u : n_loci == 128 ? 2u : 3u;
    return continuous ? 16u + l : l + 4u * ((linked ? 1u : 0u) + (weighted ? 2u : 0u));
}
bool continuous_job(const spg_pop_desc &d) { return d.allele_model == 1u; }
uint32_t job_words(const spg_pop_desc &d) { return continuous_job(d) ? d.n_loci / 2 : d.n_loci / 32; }

}  // namespace

struct spg_server {
    spg_server_config cfg{};
    Allocator alloc;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t group_stream[kGroups] = {};
    cudaEvent_t tick_start = nullptr, group_done[kGroups] = {};
    std::vector<std::unique_ptr<Job>> jobs;  // by id
    std::deque<uint64_t> queue;
    std::vector<uint64_t> resident;
    size_t used = 0, peak_used = 0;
    uint32_t peak_resident = 0;
    char *table[kGroups] = {};
    size_t table_cap[kGroups] = {};
    GenLaunch gl[kGroups];
    bool dirty = true;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

int server_sync(spg_server *s) {
    const cudaError_t e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? SPG_OK : cuda_fail(e, "cudaStreamSynchronize");
}

int retire(spg_server *s, Job &j) {
    DevState st;
    int rc = view_state(j.v, st);
    if (rc != SPG_OK) return rc;
    j.final_gen = st.gen;
    j.status = st.status;
    j.stats.resize(st.gen);
    if (st.gen) {
        rc = view_read_stats(j.v, 1, st.gen, j.stats.data());
        if (rc != SPG_OK) return rc;
    }
    s->alloc.release(j.arena, s->stream);
    j.arena = nullptr;
    j.prm.reset();
    j.link.reset();
    j.weights.reset();
    s->used -= j.footprint;
    j.state = SPG_JOB_FINISHED;
    j.t_finish = s->now();
    std::vector<uint32_t>().swap(j.founders);
    return SPG_OK;
}

// Try to make job j resident; returns 1 if admitted, 0 if it must wait.
int admit(spg_server *s, Job &j) {
    if (s->resident.size() >= s->cfg.max_resident) return 0;
    if (s->used + j.footprint > s->cfg.memory_budget) return 0;
    j.arena = static_cast<char *>(s->alloc.alloc(j.footprint, s->stream));
    if (!j.arena) return 0;  // the allocator is full right now; retry next tick
    const uint32_t words = job_words(j.desc);
    j.prm.reset(new (std::nothrow) PopParams());
    if (!j.prm) return fail(SPG_ERR_OOM, "host allocation failed");
    int rc = build_params(&j.desc, *j.prm);
    if (rc != SPG_OK) return rc;
    j.prm->linked = j.link ? 1u : 0u;
    j.prm->weighted = j.weights ? 1u : 0u;
    j.v.base = j.arena;
    j.v.n = j.desc.n;
    j.v.words = words;
    j.v.cap = j.prm->stats_cap;
    j.v.nbuckets = bucket_count(j.desc.n);
    j.v.L = layout_for(j.desc.n, words, j.v.nbuckets, j.v.cap, j.weights != nullptr, !continuous_job(j.desc));
    j.v.stream = s->stream;
    cudaError_t e = cudaSuccess;
    if (j.link) {  // the variant tables in the job's memory (read by its parameters)
        j.prm->link = reinterpret_cast<const LinkParams *>(j.arena + j.v.L.link);
        e = cudaMemcpyAsync(j.arena + j.v.L.link, j.link.get(), sizeof(LinkParams), cudaMemcpyHostToDevice, s->stream);
    }
    if (e == cudaSuccess && j.weights) {
        j.prm->weights = reinterpret_cast<const WeightParams *>(j.arena + j.v.L.weights);
        e = cudaMemcpyAsync(j.arena + j.v.L.weights, j.weights.get(), sizeof(WeightParams), cudaMemcpyHostToDevice,
                            s->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "upload a job's variant tables");
    rc = view_init(j.v, *j.prm, j.founders.empty() ? nullptr : j.founders.data(), j.desc.p0_q32);
    if (rc == SPG_OK && j.has_eco) rc = view_set_ecology(j.v, *j.prm, &j.eco);
    DevState st;
    if (rc == SPG_OK) rc = view_state(j.v, st);
    if (rc == SPG_OK) rc = view_set_state(j.v, st.gen, st.S, st.f, st.R, st.status, j.n_gen);
    if (rc != SPG_OK) return rc;
    j.state = SPG_JOB_RESIDENT;
    j.t_admit = s->now();
    s->used += j.footprint;
    s->peak_used = std::max(s->peak_used, s->used);
    return 1;
}

int rebuild(spg_server *s) {
    int rc = server_sync(s);
    if (rc != SPG_OK) return rc;
    for (int gi = 0; gi < kGroups; ++gi) {
        std::vector<const PopView *> views;
        uint64_t offspring = 0;
        uint32_t buckets = 0;
        bool eco = false, dom = false;
        const bool continuous = gi >= 16;
        const uint32_t words = continuous ? (32u << (gi % 4)) / 2u : 1u << (gi % 4);
        const bool linked = !continuous && ((gi / 4) & 1) != 0, weighted = !continuous && ((gi / 4) & 2) != 0;
        for (uint64_t id : s->resident) {
            const Job &j = *s->jobs[id];
            if (group_of(j.desc.n_loci, j.link != nullptr, j.weights != nullptr, continuous_job(j.desc)) !=
                (uint32_t)gi)
                continue;
            views.push_back(&j.v);
            offspring += j.v.n;
            buckets += j.v.nbuckets;
            eco |= j.prm->has_eco != 0u;
            dom |= j.prm->has_dom != 0u;
        }
        const size_t need = group_table_bytes((uint32_t)views.size(), offspring, buckets);
        if (need > s->table_cap[gi]) {
            if (s->table[gi]) s->alloc.release(s->table[gi], s->stream);
            s->table[gi] = nullptr;
            s->table_cap[gi] = 0;
            const size_t cap = std::max<size_t>(need * 2, 1 << 16);
            s->table[gi] = static_cast<char *>(s->alloc.alloc(cap, s->stream));
            if (!s->table[gi]) return fail(SPG_ERR_OOM, "launch table allocation failed");
            s->table_cap[gi] = cap;
        }
        const Shape shape = (linked || weighted || continuous) ? Shape{(uint32_t)kBlock, 1u, 1u} : default_shape(words);
        rc = build_group_launch(views, words, shape, eco, dom, s->table[gi], s->table_cap[gi], s->gl[gi], linked,
                                weighted, continuous);
        if (rc != SPG_OK) return rc;
    }
    s->dirty = false;
    return SPG_OK;
}

int advance(spg_server *s, uint32_t k) {
    cudaError_t e = cudaEventRecord(s->tick_start, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    for (int gi = 0; gi < kGroups; ++gi) {
        if (s->gl[gi].blocks == 0) continue;
        e = cudaStreamWaitEvent(s->group_stream[gi], s->tick_start, 0);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
        for (uint32_t i = 0; i < k; ++i) {
            const int rc = launch_generation(s->gl[gi], s->group_stream[gi]);
            if (rc != SPG_OK) return rc;
        }
        e = cudaEventRecord(s->group_done[gi], s->group_stream[gi]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->group_done[gi], 0);
        if (e != cudaSuccess) return cuda_fail(e, "join group stream");
    }
    for (uint64_t id : s->resident) {
        Job &j = *s->jobs[id];
        j.gen = std::min(j.n_gen, j.gen + k);
    }
    return server_sync(s);
}

}  // namespace

extern "C" {

int spg_server_create(const spg_server_config *cfg, const spg_allocator *alloc, void *stream, spg_server **out) {
    if (!out) return fail(SPG_ERR_INVALID, "out is NULL");
    *out = nullptr;
    std::unique_ptr<spg_server> s(new (std::nothrow) spg_server());
    if (!s) return fail(SPG_ERR_OOM, "host allocation failed");
    if (cfg) s->cfg = *cfg;
    if (s->cfg.max_resident == 0) s->cfg.max_resident = 1024;
    if (s->cfg.gens_per_tick == 0) s->cfg.gens_per_tick = 16;
    if (s->cfg.memory_budget == 0) {
        size_t free_b = 0, total_b = 0;
        const cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
        s->cfg.memory_budget = free_b / 10 * 8;
    }
    if (alloc) s->alloc.hooks = *alloc;
    cudaError_t e = cudaSuccess;
    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        s->own_stream = e == cudaSuccess;
    }
    for (int gi = 0; gi < kGroups && e == cudaSuccess; ++gi) {
        e = cudaStreamCreateWithFlags(&s->group_stream[gi], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->group_done[gi], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->tick_start, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        spg_server_destroy(s.release());
        return cuda_fail(e, "server streams");
    }
    *out = s.release();
    return SPG_OK;
}

int spg_server_submit(spg_server *s, const spg_pop_desc *desc, const spg_ecology *eco, uint32_t n_gen,
                      double t_arrival, uint64_t *job) {
    if (!s || !job) return fail(SPG_ERR_INVALID, "NULL argument");
    int rc = validate_desc(desc);
    if (rc != SPG_OK) return rc;
    if (eco && (rc = check_ecology(eco)) != SPG_OK) return rc;
    if (n_gen == 0) return fail(SPG_ERR_INVALID, "a job needs at least one generation");
    std::unique_ptr<Job> j(new (std::nothrow) Job());
    if (!j) return fail(SPG_ERR_OOM, "host allocation failed");
    if (desc->map_morgans) {  // built (and checked) now: the caller's arrays need not outlive the call
        j->link.reset(new (std::nothrow) LinkParams());
        if (!j->link) return fail(SPG_ERR_OOM, "host allocation failed");
        if ((rc = build_link(desc->map_morgans, desc->n_loci, *j->link)) != SPG_OK) return rc;
    }
    if (desc->mother_weights || desc->father_weights) {
        j->weights.reset(new (std::nothrow) WeightParams());
        if (!j->weights) return fail(SPG_ERR_OOM, "host allocation failed");
        if ((rc = build_weights(desc->mother_weights, desc->father_weights, *j->weights)) != SPG_OK) return rc;
    }
    j->desc = *desc;
    j->desc.map_morgans = nullptr;
    j->desc.mother_weights = j->desc.father_weights = nullptr;
    j->effects.assign(desc->effects, desc->effects + desc->n_loci);
    j->table.assign(desc->surv_table, desc->surv_table + SPG_N_BINS);
    if (desc->init_genotypes)
        j->founders.assign(desc->init_genotypes, desc->init_genotypes + (size_t)desc->n * 2 * (desc->n_loci / 32));
    if (continuous_job(*desc) && desc->init_values) {  // [N * 2L] int16, kept as the records' words
        j->founders.resize((size_t)desc->n * desc->n_loci);
        std::memcpy(j->founders.data(), desc->init_values, j->founders.size() * 4);
    }
    j->desc.effects = j->effects.data();
    if (desc->dominance) {
        j->dominance.assign(desc->dominance, desc->dominance + desc->n_loci);
        j->desc.dominance = j->dominance.data();
    }
    j->desc.surv_table = j->table.data();
    j->desc.init_genotypes = nullptr;
    j->desc.init_values = nullptr;
    j->desc.stats_capacity = n_gen;  // every generation's statistics stay readable
    if (eco) {
        j->has_eco = true;
        j->eco = *eco;
        j->attack.assign(eco->attack, eco->attack + SPG_N_BINS);
        j->eco.attack = j->attack.data();
    }
    j->n_gen = n_gen;
    j->t_arrival = t_arrival;
    j->footprint = align_up(layout_for(desc->n, job_words(*desc), bucket_count(desc->n), n_gen, j->weights != nullptr,
                                       !continuous_job(*desc))
                                .total,
                            256);
    if (j->footprint > s->cfg.memory_budget)
        return fail(SPG_ERR_BUDGET, "job needs %zu bytes, the budget is %zu", j->footprint, s->cfg.memory_budget);
    *job = s->jobs.size();
    s->jobs.push_back(std::move(j));
    s->queue.push_back(*job);
    return SPG_OK;
}

int spg_server_tick(spg_server *s, uint32_t *resident, uint32_t *queued) {
    if (!s) return fail(SPG_ERR_INVALID, "server is NULL");
    int rc = SPG_OK;
    // 1. retire
    for (size_t i = 0; i < s->resident.size();) {
        Job &j = *s->jobs[s->resident[i]];
        if (j.gen >= j.n_gen) {
            rc = retire(s, j);
            if (rc != SPG_OK) return rc;
            s->resident.erase(s->resident.begin() + (long)i);
            s->dirty = true;
        } else {
            ++i;
        }
    }
    // 2. admit in arrival order
    while (!s->queue.empty()) {
        Job &j = *s->jobs[s->queue.front()];
        rc = admit(s, j);
        if (rc < 0) return rc;
        if (rc == 0) break;
        s->resident.push_back(s->queue.front());
        s->queue.pop_front();
        s->dirty = true;
    }
    s->peak_resident = std::max<uint32_t>(s->peak_resident, (uint32_t)s->resident.size());
    // 3. launch tables, 4. advance
    if (!s->resident.empty()) {
        if (s->dirty && (rc = rebuild(s)) != SPG_OK) return rc;
        uint32_t k = 0;
        for (uint64_t id : s->resident) {
            const Job &j = *s->jobs[id];
            k = std::max(k, j.n_gen - j.gen);
        }
        rc = advance(s, std::min(k, s->cfg.gens_per_tick));
        if (rc != SPG_OK) return rc;
    }
    if (resident) *resident = (uint32_t)s->resident.size();
    if (queued) *queued = (uint32_t)s->queue.size();
    return SPG_OK;
}

int spg_server_drain(spg_server *s) {
    if (!s) return fail(SPG_ERR_INVALID, "server is NULL");
    while (!s->queue.empty() || !s->resident.empty()) {
        const size_t before = s->queue.size() + s->resident.size();
        uint32_t r = 0, q = 0;
        const int rc = spg_server_tick(s, &r, &q);
        if (rc != SPG_OK) return rc;
        if (r == 0 && q == before && q > 0) return fail(SPG_ERR_BUDGET, "queued jobs cannot be admitted");
    }
    return SPG_OK;
}

int spg_server_run_trace(spg_server *s, const spg_pop_desc *descs, const spg_ecology *ecos, const uint8_t *has_eco,
                         const uint32_t *n_gen, const double *arrivals, uint32_t count, uint64_t *jobs) {
    if (!s || !descs || !n_gen || !arrivals || !jobs) return fail(SPG_ERR_INVALID, "NULL argument");
    for (uint32_t i = 1; i < count; ++i)
        if (arrivals[i] < arrivals[i - 1]) return fail(SPG_ERR_INVALID, "arrivals must be non-decreasing");
    const double base = s->now();
    uint32_t next = 0;
    while (true) {
        const double t = s->now() - base;
        while (next < count && arrivals[next] <= t) {
            const spg_ecology *eco = (ecos && has_eco && has_eco[next]) ? ecos + next : nullptr;
            const int rc = spg_server_submit(s, descs + next, eco, n_gen[next], base + arrivals[next], jobs + next);
            if (rc != SPG_OK) return rc;
            ++next;
        }
        if (s->queue.empty() && s->resident.empty()) {
            if (next == count) break;
            const double wait = arrivals[next] - (s->now() - base);
            if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait));
            continue;
        }
        const size_t before = s->queue.size();
        uint32_t r = 0, q = 0;
        const int rc = spg_server_tick(s, &r, &q);
        if (rc != SPG_OK) return rc;
        if (r == 0 && q == before && q > 0 && next == count)
            return fail(SPG_ERR_BUDGET, "queued jobs cannot be admitted");
    }
    return SPG_OK;
}

int spg_server_job_info(spg_server *s, uint64_t job, spg_job_info *out) {
    if (!s || !out) return fail(SPG_ERR_INVALID, "NULL argument");
    if (job >= s->jobs.size()) return fail(SPG_ERR_INVALID, "unknown job %llu", (unsigned long long)job);
    const Job &j = *s->jobs[job];
    out->job = job;
    out->state = j.state;
    out->gen = j.state == SPG_JOB_FINISHED ? j.final_gen : j.gen;
    out->status = j.status;
    out->n_gen = j.n_gen;
    out->t_arrival = j.t_arrival;
    out->t_admit = j.t_admit;
    out->t_finish = j.t_finish;
    out->footprint = j.footprint;
    return SPG_OK;
}

int spg_server_job_stats(spg_server *s, uint64_t job, uint32_t first_gen, uint32_t count, spg_stats *out) {
    if (!s || (!out && count)) return fail(SPG_ERR_INVALID, "NULL argument");
    if (job >= s->jobs.size()) return fail(SPG_ERR_INVALID, "unknown job %llu", (unsigned long long)job);
    const Job &j = *s->jobs[job];
    if (j.state != SPG_JOB_FINISHED) return fail(SPG_ERR_RANGE, "job %llu has not finished", (unsigned long long)job);
    if (first_gen == 0 || (uint64_t)first_gen + count - 1 > j.stats.size())
        return fail(SPG_ERR_RANGE, "job %llu ran %zu generations", (unsigned long long)job, j.stats.size());
    std::copy(j.stats.begin() + (first_gen - 1), j.stats.begin() + (first_gen - 1 + count), out);
    return SPG_OK;
}

int spg_server_stats(spg_server *s, spg_server_counters *out) {
    if (!s || !out) return fail(SPG_ERR_INVALID, "NULL argument");
    out->submitted = s->jobs.size();
    out->queued = s->queue.size();
    out->resident = s->resident.size();
    out->peak_resident = s->peak_resident;
    out->memory_budget = s->cfg.memory_budget;
    out->memory_used = s->used;
    out->peak_memory_used = s->peak_used;
    return SPG_OK;
}

double spg_server_clock(spg_server *s) { return s ? s->now() : 0.0; }

void spg_server_destroy(spg_server *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (auto &jp : s->jobs)
        if (jp && jp->arena) s->alloc.release(jp->arena, s->stream);
    for (int gi = 0; gi < kGroups; ++gi) {
        if (s->table[gi]) s->alloc.release(s->table[gi], s->stream);
        if (s->group_stream[gi]) cudaStreamDestroy(s->group_stream[gi]);
        if (s->group_done[gi]) cudaEventDestroy(s->group_done[gi]);
    }
    if (s->tick_start) cudaEventDestroy(s->tick_start);
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
