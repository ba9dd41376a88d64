// Device kernels of the per-generation update (sm_103a).
//
// A generation of every population in a launch group is two launches
// (Fig. 1 A-F of the paper):
//   k_offspring  one block per tile of kBlock*ITEMS offspring: draws both
//                parents from the previous survivors (A), forms the gametes
//                by crossover masks and mutation XOR (B), sums the additive
//                phenotype with bit-plane popcounts (C), decides survival
//                from the threshold table (D), and writes the child records,
//                the alive bitmap, per-bucket survivor counts and the exact
//                integer statistics;
//   k_compact    one block per bucket of kBucket offspring: turns the bitmap
//                into the ordered survivor list (E) with a two-level scan
//                (earlier buckets' counts + a block scan), and the block that
//                finishes a population's last bucket closes its generation:
//                statistics header, resource update in IEEE double with
//                explicitly rounded basic operations (F), new state.
// No block ever waits on another block.
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

// --------------------------------------------------- warp reductions
// Exact warp sums of per-lane integers through redux.sync on 16-bit limbs
// (every limb sum stays far below 2^32).
__device__ __forceinline__ long long warp_sum_i32(int v) {
    const uint32_t lo = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)v & 0xFFFFu);
    const int hi = __reduce_add_sync(0xFFFFFFFFu, v >> 16);
    return (long long)hi * 65536ll + (long long)lo;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
    unsigned long long r = 0;
#pragma unroll
    for (int q = 3; q >= 0; --q)
        r = (r << 16) + __reduce_add_sync(0xFFFFFFFFu, (uint32_t)(v >> (16 * q)) & 0xFFFFu);
    return r;
}

// Segment (population) owning launch-wide unit `u` given each segment's
// first unit: last segment with first <= u.
template <typename F>
__device__ __forceinline__ uint32_t find_segment(const Segment *segs, uint32_t nsegs, uint32_t u, F first) {
    uint32_t lo = 0, hi = nsegs - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (first(segs[mid]) <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct PopNow {
    uint32_t gen, S, f;
    bool active;
};

__device__ __forceinline__ PopNow read_state(const DevState *st) {
    PopNow s;
    s.gen = ld_relaxed_u32(&st->gen);
    s.S = ld_relaxed_u32(&st->S);
    s.f = ld_relaxed_u32(&st->f);
    const int32_t status = (int32_t)ld_relaxed_u32(reinterpret_cast<const uint32_t *>(&st->status));
    s.active = s.S > 0u && status == SPG_OK;
    return s;
}

// --------------------------------------------- offspring kernel (Fig. 1A-D)
// One block per tile of kBlock*ITEMS offspring; offspring j = base +
// it*kBlock + tid.  Writes the child records, the alive bitmap (word j/32 is
// the ballot of the warp holding j), the tile's survivor count into its
// compaction bucket, and the integer statistics.
template <int W, int ITEMS>
__global__ void __launch_bounds__(kBlock) k_offspring(GenArgs a) {
    constexpr int NW = kBlock / 32;
    constexpr uint32_t TILE = (uint32_t)(kBlock * ITEMS);
    __shared__ uint32_t s_planes[kMaxPlanes * W];
    __shared__ uint32_t s_cdf[kMaxKmax];
    __shared__ long long s_sum[2][NW];
    __shared__ unsigned long long s_sum64[2][NW];
    __shared__ uint32_t s_cnt[3][NW];
    __shared__ int s_mm[2][NW];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t tile = blockIdx.x;
    const Segment &sg = a.segs[find_segment(a.segs, a.nsegs, tile, [](const Segment &x) { return x.tile_begin; })];
    const PopNow now = read_state(sg.state);
    if (!now.active) return;
    const PopParams *__restrict__ P = sg.prm;
    const uint32_t t_local = tile - sg.tile_begin;
    const uint32_t n = P->n, nplanes = P->nplanes, kmax = P->kmax, rep = P->rep;
    const uint32_t k0 = P->key0, k1 = P->key1;
    const int32_t e_min = P->e_min, bias = P->bias;
    const uint32_t shift = P->shift, S = now.S, f = now.f;
    const bool has_eco = P->has_eco != 0u;
    const uint32_t gen = now.gen, g = gen + 1;
    const uint32_t *__restrict__ par = sg.geno[gen & 1u];
    uint32_t *__restrict__ chi = sg.geno[(gen + 1u) & 1u];
    const uint32_t *__restrict__ sin = sg.surv[gen & 1u];
    const uint32_t base = t_local * TILE;
    uint32_t *bucket_now = sg.bucket_sum + (g & 1u) * sg.nbuckets;
    uint32_t *bucket_next = sg.bucket_sum + ((g + 1u) & 1u) * sg.nbuckets;

    for (uint32_t i = tid; i < nplanes * W; i += kBlock) s_planes[i] = P->planes[i];
    if (tid < kMaxKmax) s_cdf[tid] = tid < kmax ? P->cdf[tid] : 0u;
    // the bucket this tile opens is cleared for the next generation
    if (tid == 0 && base % kBucket == 0u) bucket_next[base / kBucket] = 0u;
    __syncthreads();

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

    int sum_raw = 0, sum_raw_s = 0, mn = INT_MAX, mx = INT_MIN;
    unsigned long long sum_raw2 = 0, cons = 0;
    uint32_t het_sum = 0, allele_sum = 0, tile_alive = 0;

#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const uint32_t j = base + it * kBlock + tid;
        bool alive = false;
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
            alive = (thr == kCertain) || (u_surv[it] < thr);

            sum_raw += raw;
            sum_raw2 += (unsigned long long)((long long)raw * (long long)raw);
            mn = min(mn, raw);
            mx = max(mx, raw);
            het_sum += hz;
            allele_sum += allele;
            if (alive) {
                sum_raw_s += raw;
                if (has_eco) cons += __ldg(&P->attack[bin]);
            }
        }
        // (E, first half) the alive bitmap: word (base + it*kBlock + 32*warp)/32
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, alive);
        if (lane == 0) sg.alive[(base >> 5) + it * NW + warp] = bal;
        tile_alive += __popc(bal);
    }

    // statistics: exact warp sums, then one atomic per field and block
    const long long w_raw = warp_sum_i32(sum_raw), w_raw_s = warp_sum_i32(sum_raw_s);
    const unsigned long long w_raw2 = warp_sum_u64(sum_raw2), w_cons = warp_sum_u64(cons);
    const uint32_t w_het = __reduce_add_sync(0xFFFFFFFFu, het_sum);
    const uint32_t w_allele = __reduce_add_sync(0xFFFFFFFFu, allele_sum);
    const int w_mn = __reduce_min_sync(0xFFFFFFFFu, mn), w_mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if (lane == 0) {
        s_sum[0][warp] = w_raw;
        s_sum[1][warp] = w_raw_s;
        s_sum64[0][warp] = w_raw2;
        s_sum64[1][warp] = w_cons;
        s_cnt[0][warp] = w_het;
        s_cnt[1][warp] = w_allele;
        s_cnt[2][warp] = tile_alive;
        s_mm[0][warp] = w_mn;
        s_mm[1][warp] = w_mx;
    }
    __syncthreads();
    if (tid == 0) {
        long long a0 = 0, a1 = 0;
        unsigned long long b0 = 0, b1 = 0, hz = 0, al = 0;
        uint32_t alive_cnt = 0;
        int m0 = INT_MAX, m1 = INT_MIN;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            a0 += s_sum[0][w];
            a1 += s_sum[1][w];
            b0 += s_sum64[0][w];
            b1 += s_sum64[1][w];
            hz += s_cnt[0][w];
            al += s_cnt[1][w];
            alive_cnt += s_cnt[2][w];
            m0 = min(m0, s_mm[0][w]);
            m1 = max(m1, s_mm[1][w]);
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
        if (alive_cnt) {
            atomicAdd(&rec->s, alive_cnt);
            atomicAdd(&bucket_now[base / kBucket], alive_cnt);
        }
    }
}

// ---------------------------------------- compaction kernel (Fig. 1E, 1F)
// One block of kBucketWords threads per bucket of kBucket offspring: the
// survivors' indices, in offspring order, at offset (survivors of all earlier
// buckets) + (block scan of the bitmap words' popcounts).  The block that
// finishes a population's last bucket closes its generation.
__global__ void __launch_bounds__(kBucketWords) k_compact(GenArgs a) {
    constexpr int NW = kBucketWords / 32;
    __shared__ uint32_t s_warp[NW];
    __shared__ uint32_t s_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t bkt = blockIdx.x;
    const Segment &sg =
        a.segs[find_segment(a.segs, a.nsegs, bkt, [](const Segment &x) { return x.bucket_begin; })];
    const PopNow now = read_state(sg.state);
    if (!now.active) return;
    const PopParams *__restrict__ P = sg.prm;
    const uint32_t b = bkt - sg.bucket_begin;
    const uint32_t g = now.gen + 1u;
    const uint32_t valid_words = (P->n + 31u) >> 5;
    const uint32_t w = b * kBucketWords + tid;
    const uint32_t bits = w < valid_words ? __ldcg(sg.alive + w) : 0u;
    const uint32_t cnt = __popc(bits);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    if (warp == 0) {
        const uint32_t *bs = sg.bucket_sum + (g & 1u) * sg.nbuckets;
        uint32_t acc = 0;
        for (uint32_t i = lane; i < b; i += 32) acc += __ldcg(bs + i);
        acc = __reduce_add_sync(0xFFFFFFFFu, acc);
        if (lane == 0) s_base = acc;
    }
    __syncthreads();
    uint32_t excl = s_base + incl - cnt;
    for (int q = 0; q < warp; ++q) excl += s_warp[q];
    uint32_t *__restrict__ sout = sg.surv[(now.gen + 1u) & 1u];
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t w0 = b * kBucketWords + (uint32_t)warp * 32u;
    for (int k = 0; k < 32; ++k) {
        const uint32_t word = __shfl_sync(0xFFFFFFFFu, bits, k);
        const uint32_t r0 = __shfl_sync(0xFFFFFFFFu, excl, k);
        if ((word >> lane) & 1u) sout[r0 + __popc(word & lt)] = (w0 + (uint32_t)k) * 32u + (uint32_t)lane;
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const uint32_t d = atomicAdd(&sg.state->done, 1u);
        if (d == sg.nbuckets - 1u) {
            __threadfence();
            finalize(sg.state, sg.ring, P, g, now.f);
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

}  // namespace

bool supported_items(uint32_t items) { return items == 1 || items == 2 || items == 4; }
uint32_t tile_size(uint32_t items) { return (uint32_t)kBlock * items; }

GenKernel compact_kernel() { return &k_compact; }

GenKernel offspring_kernel(uint32_t words, uint32_t items) {
#define SPG_CASE(Wv, Iv) \
    if (words == Wv && items == Iv) return &k_offspring<Wv, Iv>;
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

}  // namespace spg
