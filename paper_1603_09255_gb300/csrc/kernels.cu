// Device kernels of the per-generation update (sm_103a).
//
// One launch advances every population of a launch group by one generation
// (Fig. 1 A-F of the paper): each block takes a tile of kBlock*ITEMS
// offspring of one population and, in one pass,
//   draws both parents from the previous survivors,            (Fig. 1A)
//   forms the two gametes by crossover masks + mutation XOR,   (Fig. 1B)
//   sums the additive phenotype with bit-plane popcounts,      (Fig. 1C)
//   decides survival from the threshold table,                  (Fig. 1D)
//   writes the survivors' indices in offspring order through a
//   ballot + block scan + decoupled look-back compaction,      (Fig. 1E)
// and the last block of a population to finish reduces nothing more than a
// few scalars: it closes the statistics record and updates the resource
// (Fig. 1F) in IEEE double with explicitly rounded basic operations.
//
// All random numbers are Philox4x32-10 lanes at counters that name
// (individual, generation, replicate, purpose<<24 | sub); see spegg.h.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "spegg_internal.h"

namespace spg {
namespace {

// ---------------------------------------------------------------- Philox
// Philox4x32-10 from its published definition (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of
// (c0,c1,c2,c3) -> (hi(B*c2)^c1^k0, lo(B*c2), hi(A*c0)^c3^k1, lo(A*c0)),
// the key advanced by the Weyl increments between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
    constexpr uint32_t A = 0xD2511F53u, B = 0xCD9E8D57u;
    constexpr uint32_t WA = 0x9E3779B9u, WB = 0xBB67AE85u;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t hi0 = __umulhi(A, c.x), lo0 = A * c.x;
        const uint32_t hi1 = __umulhi(B, c.z), lo1 = B * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += WA;
        k1 += WB;
    }
    return c;
}

__device__ __forceinline__ uint32_t lane_of(const uint4 &d, int lane) {
    return lane == 0 ? d.x : lane == 1 ? d.y : lane == 2 ? d.z : d.w;
}

// ------------------------------------------------- relaxed gpu-scope access
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ double ld_relaxed_f64(const double *p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}

// --------------------------------------------------- packed record access
template <int W>
__device__ __forceinline__ void load_record(const uint32_t *__restrict__ p, uint32_t (&r)[2 * W]) {
    if constexpr (W == 1) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        r[0] = v.x;
        r[1] = v.y;
    } else {
#pragma unroll
        for (int q = 0; q < W / 2; ++q) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p) + q);
            r[4 * q + 0] = v.x;
            r[4 * q + 1] = v.y;
            r[4 * q + 2] = v.z;
            r[4 * q + 3] = v.w;
        }
    }
}

template <int W>
__device__ __forceinline__ void store_record(uint32_t *__restrict__ p, const uint32_t (&r)[2 * W]) {
    if constexpr (W == 1) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(r[0], r[1]);
    } else {
#pragma unroll
        for (int q = 0; q < W / 2; ++q)
            reinterpret_cast<uint4 *>(p)[q] = make_uint4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
    }
}

// Flip K distinct uniformly drawn allele positions (per-locus mutation,
// S2 "Genetics").  Rare path; indices are resolved by unrolled compares so
// the record stays in registers.
template <int W>
__device__ __forceinline__ void mutate(uint32_t (&c)[2 * W], uint32_t k, uint32_t j, uint32_t g, uint32_t rep,
                                    uint32_t k0, uint32_t k1) {
    uint32_t seen[2 * W];
#pragma unroll
    for (int w = 0; w < 2 * W; ++w) seen[w] = 0u;
    uint32_t chosen = 0;
    for (uint32_t a4 = 0; a4 < kMutDraws / 4 && chosen < k; ++a4) {
        const uint4 d = philox(make_uint4(j, g, rep, (kMutPos << 24) | a4), k0, k1);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            if (chosen < k) {
                const uint32_t pos = __umulhi(lane_of(d, l), 64u * W);  // [0, 2L)
                const uint32_t wi = pos >> 5, bit = 1u << (pos & 31u);
                bool dup = false;
#pragma unroll
                for (int w = 0; w < 2 * W; ++w)
                    if ((uint32_t)w == wi) dup = (seen[w] & bit) != 0u;
                if (!dup) {
#pragma unroll
                    for (int w = 0; w < 2 * W; ++w)
                        if ((uint32_t)w == wi) {
                            seen[w] |= bit;
                            c[w] ^= bit;
                        }
                    ++chosen;
                }
            }
        }
    }
}

// Additive phenotype (Fig. 1C, eq. S2-phenval) with effects in offset
// binary: e_l = e_min + sum_b 2^b * bit_b(e_l - e_min), so
// raw = e_min * (copies) + sum_b 2^b * popc(plane_b & copies).
template <int W>
__device__ __forceinline__ int32_t phenotype(const uint32_t (&c)[2 * W], const uint32_t *s_planes,
                                             uint32_t nplanes, int32_t e_min, uint32_t &allele,
                                             uint32_t &het) {
    uint32_t total = 0, hz = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        total += __popc(c[w]) + __popc(c[W + w]);
        hz += __popc(c[w] ^ c[W + w]);
    }
    int32_t raw = e_min * (int32_t)total;
    for (uint32_t b = 0; b < nplanes; ++b) {
        int32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t pl = s_planes[b * W + w];
            cnt += __popc(pl & c[w]) + __popc(pl & c[W + w]);
        }
        raw += cnt << b;
    }
    allele = total;
    het = hz;
    return raw;
}

// ------------------------------------------------- decoupled look-back
// Status word: [63:62] flag (1 aggregate, 2 inclusive prefix), [61:32] the
// generation tag, [31:0] value.  Words of older generations never match.
constexpr unsigned long long kFlagAgg = 1ull << 62, kFlagPrefix = 2ull << 62;
constexpr uint32_t kTagMask = 0x3FFFFFFFu;

__device__ __forceinline__ unsigned long long status_word(unsigned long long flag, uint32_t tag, uint32_t v) {
    return flag | ((unsigned long long)(tag & kTagMask) << 32) | (unsigned long long)v;
}

// Exclusive prefix of tile t, computed by one full warp: each round reads the
// status words of the 32 nearest unread predecessors, waits (bounded) until
// every one of them up to the nearest inclusive prefix has been published,
// and adds their values.  Sets *timed_out if the wait exceeded spin_limit
// polls; the tile then publishes its own count as if it were first, so its
// successors do not wait on it.
__device__ uint32_t look_back(unsigned long long *status, uint32_t t, uint32_t count, uint32_t tag,
                              uint32_t spin_limit, bool *timed_out) {
    const uint32_t lane = threadIdx.x & 31u;
    if (t == 0) {
        if (lane == 0) st_relaxed(&status[0], status_word(kFlagPrefix, tag, count));
        return 0;
    }
    if (lane == 0) st_relaxed(&status[t], status_word(kFlagAgg, tag, count));
    uint32_t excl = 0, spins = 0;
    long long nearest = (long long)t - 1;  // predecessor read by lane 0 this round
    while (true) {
        const long long idx = nearest - (long long)lane;
        unsigned long long s = 0;
        uint32_t upto, prefix;
        while (true) {
            s = idx >= 0 ? ld_relaxed(&status[idx]) : status_word(kFlagPrefix, tag, 0);
            const bool ready = (uint32_t)((s >> 32) & kTagMask) == (tag & kTagMask) && (s >> 62) != 0ull;
            const uint32_t not_ready = __ballot_sync(0xFFFFFFFFu, !ready);
            prefix = __ballot_sync(0xFFFFFFFFu, ready && (s >> 62) == 2ull);
            upto = prefix ? (((prefix & (0u - prefix)) << 1) - 1u) : 0xFFFFFFFFu;  // lanes <= nearest prefix
            if ((not_ready & upto) == 0u) break;
            if (++spins > spin_limit) {
                *timed_out = true;
                if (lane == 0) st_relaxed(&status[t], status_word(kFlagPrefix, tag, count));
                return 0;
            }
            __nanosleep(32);
        }
        uint32_t v = ((upto >> lane) & 1u) ? (uint32_t)s : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        excl += v;
        if (prefix != 0u) break;
        nearest -= 32;
    }
    if (lane == 0) st_relaxed(&status[t], status_word(kFlagPrefix, tag, excl + count));
    return excl;
}

// ------------------------------------------------------ ecology (Fig. 1F)
__device__ double resource_update(double R, double r, double K, unsigned long long C) {
    const double ratio = __ddiv_rn(R, K);
    const double room = __dsub_rn(1.0, ratio);
    const double rR = __dmul_rn(r, R);
    const double growth = __dmul_rn(rR, room);
    const double grown = __dadd_rn(R, growth);
    const double eaten = __dmul_rn(__ull2double_rn(C), 1.0 / 65536.0);
    double next = __dsub_rn(grown, eaten);
    if (!(next > 0.0)) next = 0.0;
    return next;
}

__device__ uint32_t factor_q32(double R, double R_half) {
    const double den = __dadd_rn(R, R_half);
    const double q = __ddiv_rn(R, den);
    const double scaled = __dmul_rn(q, 4294967296.0);
    if (scaled >= 4294967294.0) return 0xFFFFFFFEu;
    if (!(scaled > 0.0)) return 0u;
    return __double2uint_rz(scaled);
}

__device__ void init_record(spg_stats *rec) {
    rec->gen = 0;
    rec->n = 0;
    rec->s = 0;
    rec->status = 0;
    rec->sum_raw = 0;
    rec->sum_raw2 = 0;
    rec->sum_raw_surv = 0;
    rec->min_raw = INT_MAX;
    rec->max_raw = INT_MIN;
    rec->het = 0;
    rec->allele = 0;
    rec->consumption = 0;
    rec->R = 0.0;
    rec->f = 0;
    rec->pad = 0;
}

// Close generation g of one population (run by one thread of the block that
// finished last): statistics header, resource update, new state, next slot.
__device__ void finalize(DevState *st, spg_stats *ring, const PopParams *P, uint32_t g, uint32_t f_used) {
    const uint32_t cap = P->stats_cap;
    spg_stats *rec = ring + (g - 1) % cap;
    const uint32_t S_new = ld_relaxed_u32(&rec->s);
    rec->gen = g;
    rec->n = P->n;
    uint32_t f_next = f_used;
    double R = 0.0;
    if (P->has_eco) {
        const unsigned long long C =
            ld_relaxed(reinterpret_cast<const unsigned long long *>(&rec->consumption));
        R = resource_update(ld_relaxed_f64(&st->R), P->r, P->K, C);
        f_next = factor_q32(R, P->R_half);
        st->R = R;
    }
    rec->R = R;
    rec->f = f_next;
    const int32_t status = (S_new == 0u) ? SPG_EXTINCT : SPG_OK;
    if (st->status == SPG_OK) st->status = status;
    rec->status = (uint32_t)status;
    st->f = f_next;
    st->S = S_new;
    init_record(ring + g % cap);
    st->done = 0;
    __threadfence();
    st->gen = g;
}

// --------------------------------------------------- the generation kernel
template <int W, int ITEMS>
__global__ void __launch_bounds__(kBlock) k_generation(GenArgs a) {
    static_assert(ITEMS * (kBlock / 32) <= 32, "scan of per-warp counts uses one warp");
    constexpr int NW = kBlock / 32;
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_planes[kMaxPlanes * W];
    __shared__ uint32_t s_cdf[kMaxKmax];
    __shared__ uint32_t s_cnt[ITEMS][NW];
    __shared__ uint32_t s_excl;
    __shared__ long long s_red_ll[3][NW];
    __shared__ unsigned long long s_red_ull[4][NW];
    __shared__ uint32_t s_total;
    __shared__ int s_red_i[2][NW];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(&a.ctl->ticket, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;

    // population of this tile: last segment whose first tile <= tile
    uint32_t lo = 0, hi = a.nsegs - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (a.segs[mid].tile_begin <= tile) lo = mid;
        else hi = mid - 1;
    }
    const Segment sg = a.segs[lo];
    const PopParams *__restrict__ P = sg.prm;
    const uint32_t t_local = tile - sg.tile_begin;

    const uint32_t gen = ld_relaxed_u32(&sg.state->gen);
    const uint32_t S = ld_relaxed_u32(&sg.state->S);
    const uint32_t f = ld_relaxed_u32(&sg.state->f);
    const int32_t status0 = (int32_t)ld_relaxed_u32(reinterpret_cast<const uint32_t *>(&sg.state->status));
    const bool active = (S > 0u) && (status0 == SPG_OK) && (t_local < sg.ntiles);

    if (active) {
        const uint32_t n = P->n, nplanes = P->nplanes, kmax = P->kmax, rep = P->rep;
        const uint32_t k0 = P->key0, k1 = P->key1;
        const int32_t e_min = P->e_min, bias = P->bias;
        const uint32_t shift = P->shift;
        const bool has_eco = P->has_eco != 0u;
        const uint32_t g = gen + 1;
        const uint32_t *__restrict__ par = sg.geno[gen & 1u];
        uint32_t *__restrict__ chi = sg.geno[(gen + 1u) & 1u];
        const uint32_t *__restrict__ sin = sg.surv[gen & 1u];
        uint32_t *__restrict__ sout = sg.surv[(gen + 1u) & 1u];

        for (uint32_t i = tid; i < nplanes * W; i += kBlock) s_planes[i] = P->planes[i];
        if (tid < kMaxKmax) s_cdf[tid] = tid < kmax ? P->cdf[tid] : 0u;
        __syncthreads();

        const uint32_t base = t_local * (uint32_t)(kBlock * ITEMS);

        // (A) parents: Philox draws, then the survivor-list gathers
        uint32_t mom[ITEMS], dad[ITEMS], u_surv[ITEMS], u_mut[ITEMS];
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
            const uint32_t j = base + it * kBlock + tid;
            mom[it] = dad[it] = u_surv[it] = u_mut[it] = 0u;
            if (j < n) {
                const uint4 d = philox(make_uint4(j, g, rep, kMate << 24), k0, k1);
                mom[it] = __ldg(sin + __umulhi(d.x, S));
                dad[it] = __ldg(sin + __umulhi(d.y, S));
                u_surv[it] = d.z;
                u_mut[it] = d.w;
            }
        }
        uint32_t pm[ITEMS][2 * W], pf[ITEMS][2 * W];
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
            const uint32_t j = base + it * kBlock + tid;
            if (j < n) {
                load_record<W>(par + (size_t)mom[it] * (2 * W), pm[it]);
                load_record<W>(par + (size_t)dad[it] * (2 * W), pf[it]);
            }
        }

        long long sum_raw = 0, sum_raw_s = 0;
        unsigned long long sum_raw2 = 0, cons = 0, het_sum = 0, allele_sum = 0;
        int mn = INT_MAX, mx = INT_MIN;
        uint32_t alive_bits = 0;

#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
            const uint32_t j = base + it * kBlock + tid;
            if (j < n) {
                // (B) gametes: stream q = 2w + parent is lane q%4 of sub q/4
                uint32_t c[2 * W];
#pragma unroll
                for (int q4 = 0; q4 < (2 * W + 3) / 4; ++q4) {
                    const uint4 d = philox(make_uint4(j, g, rep, (kRecomb << 24) | (uint32_t)q4), k0, k1);
#pragma unroll
                    for (int l = 0; l < 4; ++l) {
                        const int q = 4 * q4 + l;
                        if (q < 2 * W) {
                            const int w = q >> 1;
                            const uint32_t m = lane_of(d, l);
                            if ((q & 1) == 0) c[w] = (pm[it][w] & ~m) | (pm[it][W + w] & m);
                            else c[W + w] = (pf[it][w] & ~m) | (pf[it][W + w] & m);
                        }
                    }
                }
                // (B) mutation count from the CDF, positions on the rare path
                uint32_t k = 0;
                for (uint32_t i = 0; i < kmax; ++i) k += (u_mut[it] >= s_cdf[i]) ? 1u : 0u;
                if (k != 0u) mutate<W>(c, k, j, g, rep, k0, k1);
                store_record<W>(chi + (size_t)j * (2 * W), c);

                // (C) phenotype, (D) survival
                uint32_t allele, hz;
                const int32_t raw = phenotype<W>(c, s_planes, nplanes, e_min, allele, hz);
                const long long v = (long long)raw + (long long)bias;
                const uint32_t bin = v < 0 ? 0u : (uint32_t)min(v >> shift, (long long)(kBins - 1));
                uint32_t thr = __ldg(&P->table[bin]);
                if (f != kCertain) thr = __umulhi(thr, f);
                const bool alive = (thr == kCertain) || (u_surv[it] < thr);

                sum_raw += raw;
                sum_raw2 += (unsigned long long)((long long)raw * (long long)raw);
                mn = min(mn, raw);
                mx = max(mx, raw);
                het_sum += hz;
                allele_sum += allele;
                if (alive) {
                    alive_bits |= 1u << it;
                    sum_raw_s += raw;
                    if (has_eco) cons += __ldg(&P->attack[bin]);
                }
            }
        }

        // (E) compaction: per-(item, warp) ballots scanned in offspring order
        uint32_t bal[ITEMS];
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
            bal[it] = __ballot_sync(0xFFFFFFFFu, (alive_bits >> it) & 1u);
            if (lane == 0) s_cnt[it][warp] = __popc(bal[it]);
        }
        __syncthreads();
        if (warp == 0) {
            const uint32_t v = lane < ITEMS * NW ? s_cnt[lane / NW][lane % NW] : 0u;
            uint32_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane < ITEMS * NW) s_cnt[lane / NW][lane % NW] = incl - v;
            const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
            bool timed_out = false;
            const uint32_t excl = look_back(sg.tile_status, t_local, total, g, a.spin_limit, &timed_out);
            if (lane == 0) {
                s_total = total;
                s_excl = excl;
                if (timed_out)
                    atomicExch(reinterpret_cast<int *>(&sg.state->status), (int)SPG_ERR_TIMEOUT);
            }
        }
        __syncthreads();
        const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
            if ((alive_bits >> it) & 1u) {
                const uint32_t j = base + it * kBlock + tid;
                sout[s_excl + s_cnt[it][warp] + __popc(bal[it] & lt_mask)] = j;
            }
        }

        // statistics: warp, then block reduction, then one atomic per field
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sum_raw += __shfl_xor_sync(0xFFFFFFFFu, sum_raw, o);
            sum_raw_s += __shfl_xor_sync(0xFFFFFFFFu, sum_raw_s, o);
            sum_raw2 += __shfl_xor_sync(0xFFFFFFFFu, sum_raw2, o);
            cons += __shfl_xor_sync(0xFFFFFFFFu, cons, o);
            het_sum += __shfl_xor_sync(0xFFFFFFFFu, het_sum, o);
            allele_sum += __shfl_xor_sync(0xFFFFFFFFu, allele_sum, o);
            mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
            mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
        }
        if (lane == 0) {
            s_red_ll[0][warp] = sum_raw;
            s_red_ll[1][warp] = sum_raw_s;
            s_red_ull[0][warp] = sum_raw2;
            s_red_ull[1][warp] = cons;
            s_red_ull[2][warp] = het_sum;
            s_red_ull[3][warp] = allele_sum;
            s_red_i[0][warp] = mn;
            s_red_i[1][warp] = mx;
        }
        __syncthreads();
        if (tid == 0) {
            long long a0 = 0, a1 = 0;
            unsigned long long b0 = 0, b1 = 0, hz = 0, al = 0;
            int m0 = INT_MAX, m1 = INT_MIN;
            for (int w = 0; w < NW; ++w) {
                a0 += s_red_ll[0][w];
                a1 += s_red_ll[1][w];
                b0 += s_red_ull[0][w];
                b1 += s_red_ull[1][w];
                hz += s_red_ull[2][w];
                al += s_red_ull[3][w];
                m0 = min(m0, s_red_i[0][w]);
                m1 = max(m1, s_red_i[1][w]);
            }
            spg_stats *rec = sg.ring + (g - 1) % P->stats_cap;
            atomicAdd(reinterpret_cast<unsigned long long *>(&rec->sum_raw), (unsigned long long)a0);
            atomicAdd(reinterpret_cast<unsigned long long *>(&rec->sum_raw_surv), (unsigned long long)a1);
            atomicAdd(reinterpret_cast<unsigned long long *>(&rec->sum_raw2), b0);
            if (b1) atomicAdd(reinterpret_cast<unsigned long long *>(&rec->consumption), b1);
            atomicAdd(reinterpret_cast<unsigned long long *>(&rec->het), hz);
            atomicAdd(reinterpret_cast<unsigned long long *>(&rec->allele), al);
            atomicMin(&rec->min_raw, m0);
            atomicMax(&rec->max_raw, m1);
            if (s_total) atomicAdd(&rec->s, s_total);
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            const uint32_t d = atomicAdd(&sg.state->done, 1u);
            if (d == sg.ntiles - 1u) {
                __threadfence();
                finalize(sg.state, sg.ring, P, g, f);
            }
        }
    }

    if (tid == 0) {
        __threadfence();
        const uint32_t d = atomicAdd(&a.ctl->done, 1u);
        if (d == a.total_tiles - 1u) {
            atomicExch(&a.ctl->done, 0u);
            atomicExch(&a.ctl->ticket, 0u);
        }
    }
}

// ---------------------------------------------------------- founders
template <int W>
__global__ void k_founders(uint32_t *__restrict__ geno, uint32_t *__restrict__ surv, uint32_t n, uint32_t k0,
                           uint32_t k1, uint32_t rep, uint32_t p0) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // allele copy q = h*L + l (L = 32W) lies in record word q/32 = h*W + l/32
#pragma unroll
    for (int hw = 0; hw < 2 * W; ++hw) {
        uint32_t word = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const uint4 d = philox(make_uint4(i, 0u, rep, (kFounder << 24) | (uint32_t)(hw * 8 + c)), k0, k1);
            word |= (uint32_t)(d.x < p0) << (4 * c + 0);
            word |= (uint32_t)(d.y < p0) << (4 * c + 1);
            word |= (uint32_t)(d.z < p0) << (4 * c + 2);
            word |= (uint32_t)(d.w < p0) << (4 * c + 3);
        }
        geno[(size_t)i * (2 * W) + hw] = word;
    }
    surv[i] = i;
}

__global__ void k_iota(uint32_t *__restrict__ surv, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) surv[i] = i;
}

__global__ void k_set_state(DevState *st, spg_stats *ring, uint32_t cap, uint32_t gen, uint32_t S, uint32_t f,
                            double R, int32_t status) {
    st->gen = gen;
    st->S = S;
    st->f = f;
    st->status = status;
    st->R = R;
    st->done = 0;
    init_record(ring + gen % cap);
}

__global__ void k_lookback_probe(unsigned long long *status, int32_t *out, uint32_t spin_limit) {
    // one warp: tile 1 of a generation whose tile 0 never publishes
    bool timed_out = false;
    (void)look_back(status, 1u, 5u, 7u, spin_limit, &timed_out);
    if (threadIdx.x == 0) *out = timed_out ? SPG_ERR_TIMEOUT : SPG_OK;
}

}  // namespace

bool supported_items(uint32_t items) { return items == 1 || items == 2 || items == 4; }
uint32_t tile_size(uint32_t items) { return (uint32_t)kBlock * items; }

GenKernel generation_kernel(uint32_t words, uint32_t items) {
#define SPG_CASE(Wv, Iv) \
    if (words == Wv && items == Iv) return &k_generation<Wv, Iv>;
    SPG_CASE(1, 1) SPG_CASE(1, 2) SPG_CASE(1, 4)
    SPG_CASE(2, 1) SPG_CASE(2, 2) SPG_CASE(2, 4)
    SPG_CASE(4, 1) SPG_CASE(4, 2) SPG_CASE(4, 4)
    SPG_CASE(8, 1) SPG_CASE(8, 2) SPG_CASE(8, 4)
#undef SPG_CASE
    return nullptr;
}

int launch_founders(uint32_t words, uint32_t *geno, uint32_t *surv, uint32_t n, uint32_t key0, uint32_t key1,
                    uint32_t rep, uint32_t p0_q32, void *stream) {
    const dim3 grid((n + 127) / 128), block(128);
    cudaStream_t s = (cudaStream_t)stream;
    switch (words) {
        case 1: k_founders<1><<<grid, block, 0, s>>>(geno, surv, n, key0, key1, rep, p0_q32); break;
        case 2: k_founders<2><<<grid, block, 0, s>>>(geno, surv, n, key0, key1, rep, p0_q32); break;
        case 4: k_founders<4><<<grid, block, 0, s>>>(geno, surv, n, key0, key1, rep, p0_q32); break;
        case 8: k_founders<8><<<grid, block, 0, s>>>(geno, surv, n, key0, key1, rep, p0_q32); break;
        default: return SPG_ERR_INVALID;
    }
    return cudaGetLastError() == cudaSuccess ? SPG_OK : SPG_ERR_CUDA;
}

int launch_iota(uint32_t *surv, uint32_t n, void *stream) {
    k_iota<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(surv, n);
    return cudaGetLastError() == cudaSuccess ? SPG_OK : SPG_ERR_CUDA;
}

int launch_set_state(DevState *st, spg_stats *ring, uint32_t cap, uint32_t gen, uint32_t S, uint32_t f, double R,
                     int32_t status, void *stream) {
    k_set_state<<<1, 1, 0, (cudaStream_t)stream>>>(st, ring, cap, gen, S, f, R, status);
    return cudaGetLastError() == cudaSuccess ? SPG_OK : SPG_ERR_CUDA;
}

int launch_lookback_probe(unsigned long long *status_words, int32_t *out, uint32_t spin_limit, void *stream) {
    k_lookback_probe<<<1, 32, 0, (cudaStream_t)stream>>>(status_words, out, spin_limit);
    return cudaGetLastError() == cudaSuccess ? SPG_OK : SPG_ERR_CUDA;
}

}  // namespace spg
