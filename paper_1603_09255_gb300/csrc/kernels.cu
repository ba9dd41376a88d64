// Device kernels of the per-generation update (sm_103a).
//
// A generation of every population in a launch group is two launches
// (Fig. 1 A-F of the paper):
//   k_offspring  persistent: each resident block walks a contiguous range of
//                tiles of kBlock*ITEMS offspring.  Per offspring it draws both
//                parents from the previous survivors (A), forms the gametes
//                by crossover masks and mutation XOR (B), sums the additive
//                phenotype with bit-plane popcounts (C) and decides survival
//                from the threshold table (D); it writes the child records,
//                the alive bitmap, per-bucket survivor counts and exact
//                integer statistics.  The parents' survivor indices are
//                fetched two tiles ahead and their records are staged into
//                shared memory with cp.async one tile ahead, so the random
//                gathers overlap the arithmetic of the tile in hand;
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

// Minimum resident blocks per SM requested from the compiler for the
// offspring kernel (a register cap: 65536 / (256 * SPG_MIN_BLOCKS) per thread).
#ifndef SPG_MIN_BLOCKS
#define SPG_MIN_BLOCKS 2
#endif

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

// Linkage map in shared memory (see LinkParams) for one population.
struct LinkSmem {
    const uint32_t *cdf, *cum;
    const uint8_t *chrom;
    const uint16_t *first, *clast;
    const uint32_t *guide;
    uint32_t kmax, nchrom;
};

template <int W>
__device__ __forceinline__ void toggle_bit(uint32_t (&t)[W], uint32_t pos) {
#pragma unroll
    for (int w = 0; w < W; ++w)
        if ((uint32_t)w == (pos >> 5)) t[w] ^= 1u << (pos & 31u);
}

// Origin mask of one gamete under the linkage map (bit set: the locus comes
// from the parent's haplotype 1): every chromosome whose coin is 1 and every
// crossover flips the loci from its start to the chromosome's end.  Each
// flip is two toggles (at the first flipped locus and one past the last); a
// crossover toggles its start and flips its chromosome's parity bit, and the
// end toggles, which cancel in pairs, are applied once per chromosome whose
// coin and parity differ.  A prefix XOR over the L bits turns the toggles
// into the mask.
template <int W>
__device__ __forceinline__ void linked_mask(const LinkSmem &lk, uint32_t j, uint32_t g, uint32_t rep, uint32_t pi,
                                            uint32_t k0, uint32_t k1, uint32_t (&m)[W]) {
    constexpr uint32_t L = 32u * W;
    const uint4 d0 = philox(make_uint4(j, g, rep, (kLink << 24) | (pi << 8)), k0, k1);
    uint32_t t[W];
#pragma unroll
    for (int w = 0; w < W; ++w) t[w] = 0u;
    uint32_t par0 = 0, par1 = 0, par2 = 0;  // crossovers per chromosome, mod 2 (chromosomes 0-31, 32-63, 64-95)
    uint32_t K = 0;
    if (lk.kmax != 0u && d0.x >= lk.cdf[0]) {  // K = #{i < kmax : cdf[i] <= u} by bisection (the CDF is non-decreasing)
        K = 1u;
#pragma unroll
        for (uint32_t step = 16u; step > 0u; step >>= 1)
            if (K + step <= lk.kmax && lk.cdf[K + step - 1u] <= d0.x) K += step;
    }
    uint4 d = d0;
    for (uint32_t a = 0; a < K; ++a) {
        if ((a & 3u) == 0u) d = philox(make_uint4(j, g, rep, (kLink << 24) | (pi << 8) | (1u + a / 4u)), k0, k1);
        const uint32_t u = lane_of(d, (int)(a & 3u));
        // interval I = #{l <= L-2 : cum[l] <= u} and its chromosome: the guide
        // entry of u's top bits when no boundary lies inside that bucket, one
        // comparison when one does, a forward search otherwise
        const uint32_t ge = lk.guide[u >> (32 - kLinkGuideBits)], nb = ge >> 26;
        uint32_t I = ge & 0xFFu, ch = (ge >> 8) & 0x7Fu;
        if (nb == 1u) {
            if (lk.cum[I] <= u) {
                ++I;
                ch = (ge >> 15) & 0x7Fu;
            }
        } else if (nb > 1u) {
            while (I + 1u < L && lk.cum[I] <= u) ++I;
            ch = lk.chrom[I];
        }
        toggle_bit<W>(t, I);
        const uint32_t cb = 1u << (ch & 31u);
        par0 ^= ch < 32u ? cb : 0u;
        par1 ^= (ch >= 32u && ch < 64u) ? cb : 0u;
        par2 ^= ch >= 64u ? cb : 0u;
    }
    for (uint32_t c = 0; c < lk.nchrom; ++c) {
        const uint32_t coin = ((c < 32u ? d0.y : c < 64u ? d0.z : d0.w) >> (c & 31u)) & 1u;
        const uint32_t par = ((c < 32u ? par0 : c < 64u ? par1 : par2) >> (c & 31u)) & 1u;
        if (coin) toggle_bit<W>(t, lk.first[c]);
        if ((coin ^ par) && lk.clast[c] + 1u < L) toggle_bit<W>(t, lk.clast[c] + 1u);
    }
    uint32_t carry = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        uint32_t x = t[w];
        x ^= x << 1;
        x ^= x << 2;
        x ^= x << 4;
        x ^= x << 8;
        x ^= x << 16;
        x ^= 0u - carry;
        m[w] = x;
        carry = x >> 31;
    }
}

// Additive phenotype (Fig. 1C, eq. S2-phenval) with effects in offset
// binary: e_l = e_min + sum_b 2^b * bit_b(e_l - e_min), so
// raw = e_min * (copies) + sum_b 2^b * popc(plane_b & copies).
// Words of plane b (W consecutive words, 8-byte aligned for W = 2 and
// 16-byte aligned for W >= 4) in one or two vector shared-memory loads.
template <int W>
__device__ __forceinline__ void plane_words(const uint32_t *s_planes, uint32_t b, uint32_t (&pl)[W]) {
    if constexpr (W == 1) {
        pl[0] = s_planes[b];
    } else if constexpr (W == 2) {
        const uint2 v = reinterpret_cast<const uint2 *>(s_planes)[b];
        pl[0] = v.x;
        pl[1] = v.y;
    } else {
#pragma unroll
        for (int q = 0; q < W / 4; ++q) {
            const uint4 v = reinterpret_cast<const uint4 *>(s_planes)[b * (W / 4) + q];
            pl[4 * q + 0] = v.x;
            pl[4 * q + 1] = v.y;
            pl[4 * q + 2] = v.z;
            pl[4 * q + 3] = v.w;
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
#pragma unroll 4
    for (uint32_t b = 0; b < nplanes; ++b) {
        uint32_t pl[W];
        plane_words<W>(s_planes, b, pl);
        int32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) cnt += __popc(pl[w] & c[w]) + __popc(pl[w] & c[W + w]);
        raw += cnt << b;
    }
    allele = total;
    het = hz;
    return raw;
}

// Dominance part of the genetic value: heterozygous loci x = h0 ^ h1 add
// their deviations, d_min * popc(x) + sum_b 2^b * popc(dplane_b & x)
// (zero when the population has no dominance: d_min = 0, no planes).
template <int W>
__device__ __forceinline__ int32_t dominance_part(const uint32_t (&c)[2 * W], const uint32_t *s_dplanes,
                                                  uint32_t ndplanes, int32_t d_min, uint32_t het) {
    int32_t raw = d_min * (int32_t)het;
    for (uint32_t b = 0; b < ndplanes; ++b) {
        uint32_t pl[W];
        plane_words<W>(s_dplanes, b, pl);
        int32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) cnt += __popc(pl[w] & (c[w] ^ c[W + w]));
        raw += cnt << b;
    }
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

// Beverton-Holt variant: R' = (r' R) / (1 + R/K) - C 2^-16, clamped at 0.
__device__ double resource_update_bh(double R, double rg, double K, unsigned long long C) {
    const double grown_num = __dmul_rn(rg, R);
    const double ratio = __ddiv_rn(R, K);
    const double den = __dadd_rn(1.0, ratio);
    const double grown = __ddiv_rn(grown_num, den);
    const double eaten = __dmul_rn(__ull2double_rn(C), 1.0 / 65536.0);
    double next = __dsub_rn(grown, eaten);
    if (!(next > 0.0)) next = 0.0;
    return next;
}

// Growth rate of generation g: r + r_sd * z, z the Irwin-Hall(12) normal
// (sum of twelve Philox lanes of counter (0, g, rep, 7<<24 | k/4)) * 2^-32 - 6.
__device__ double growth_rate(const PopParams *P, uint32_t g) {
    if (P->r_sd == 0.0) return P->r;
    unsigned long long sum = 0;
#pragma unroll
    for (uint32_t k = 0; k < 3; ++k) {
        const uint4 d = philox(make_uint4(0u, g, P->rep, (kGrowth << 24) | k), P->key0, P->key1);
        sum += (unsigned long long)d.x + d.y + d.z + d.w;
    }
    const double u = __dmul_rn(__ull2double_rn(sum), 1.0 / 4294967296.0);
    const double z = __dsub_rn(u, 6.0);
    return __dadd_rn(P->r, __dmul_rn(P->r_sd, z));
}

__device__ uint32_t factor_q32(double R, double R_half) {
    const double den = __dadd_rn(R, R_half);
    const double q = __ddiv_rn(R, den);
    const double scaled = __dmul_rn(q, 4294967296.0);
    if (scaled >= 4294967294.0) return 0xFFFFFFFEu;
    if (!(scaled > 0.0)) return 0u;
    return __double2uint_rz(scaled);
}

__device__ __forceinline__ void clear_acc(StatAcc *a) {
    a->s = 0;
    a->sum_raw = 0;
    a->sum_raw_s = 0;
    a->sum_raw2 = 0;
    a->cons = 0;
    a->het = 0;
    a->allele = 0;
    a->mn = INT_MAX;
    a->mx = INT_MIN;
}

// --------------------------------------------------- warp reductions
// Exact warp sums of per-lane integers through redux.sync on 16-bit limbs
// (every limb sum stays far below 2^32; the top limb carries the sign).
__device__ __forceinline__ long long warp_sum_i64(long long v) {
    const uint32_t l0 = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)v & 0xFFFFu);
    const uint32_t l1 = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)(v >> 16) & 0xFFFFu);
    const uint32_t l2 = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)(v >> 32) & 0xFFFFu);
    const int l3 = __reduce_add_sync(0xFFFFFFFFu, (int)(v >> 48));
    return ((long long)l3 << 48) + ((long long)l2 << 32) + ((long long)l1 << 16) + (long long)l0;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
    unsigned long long r = 0;
#pragma unroll
    for (int q = 3; q >= 0; --q)
        r = (r << 16) + __reduce_add_sync(0xFFFFFFFFu, (uint32_t)(v >> (16 * q)) & 0xFFFFu);
    return r;
}
__device__ __forceinline__ unsigned long long shfl_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Close generation g of one population (run by one full warp while the
// population's survivors are being compacted; everything it reads was final
// when the offspring launch ended).  The statistics accumulators (kAccCopies
// copies) are summed, the resource is updated, the statistics record is
// written, the accumulators are reset for the next generation, and the new
// survivor count, factor, resource and status are left in the state's next_*
// fields for commit_state.
__device__ void finalize_warp(const Segment &sg, const PopParams *P, uint32_t g, uint32_t f_used) {
    const uint32_t lane = threadIdx.x & 31u;
    DevState *st = sg.state;
    // state loads issued together with the accumulator loads
    const double R_prev = ld_relaxed_f64(&st->R);
    StatAcc mine;
    clear_acc(&mine);
    if (lane < (uint32_t)kAccCopies) {
        StatAcc *src = sg.acc + lane;
        mine.s = __ldcg(&src->s);
        mine.sum_raw = __ldcg(&src->sum_raw);
        mine.sum_raw_s = __ldcg(&src->sum_raw_s);
        mine.sum_raw2 = __ldcg(&src->sum_raw2);
        mine.cons = __ldcg(&src->cons);
        mine.het = __ldcg(&src->het);
        mine.allele = __ldcg(&src->allele);
        mine.mn = __ldcg(&src->mn);
        mine.mx = __ldcg(&src->mx);
        clear_acc(src);
    }
    const unsigned long long S_new = shfl_sum_u64(mine.s);
    const unsigned long long sum_raw = shfl_sum_u64((unsigned long long)mine.sum_raw);
    const unsigned long long sum_raw_s = shfl_sum_u64((unsigned long long)mine.sum_raw_s);
    const unsigned long long sum_raw2 = shfl_sum_u64(mine.sum_raw2);
    const unsigned long long cons = shfl_sum_u64(mine.cons);
    const unsigned long long het = shfl_sum_u64(mine.het);
    const unsigned long long allele = shfl_sum_u64(mine.allele);
    const int mn = __reduce_min_sync(0xFFFFFFFFu, mine.mn), mx = __reduce_max_sync(0xFFFFFFFFu, mine.mx);
    if (lane == 0) {
        spg_stats *rec = sg.ring + (g - 1) % P->stats_cap;
        uint32_t f_next = f_used;
        double R = 0.0;
        if (P->has_eco) {
            R = P->eco_model == 1u ? resource_update_bh(R_prev, growth_rate(P, g), P->K, cons)
                                   : resource_update(R_prev, P->r, P->K, cons);
            f_next = factor_q32(R, P->R_half);
        }
        const int32_t status = (S_new == 0ull) ? SPG_EXTINCT : SPG_OK;
        rec->gen = g;
        rec->n = sg.n;
        rec->s = (uint32_t)S_new;
        rec->status = (uint32_t)status;
        rec->sum_raw = (long long)sum_raw;
        rec->sum_raw2 = sum_raw2;
        rec->sum_raw_surv = (long long)sum_raw_s;
        rec->min_raw = mn;
        rec->max_raw = mx;
        rec->het = het;
        rec->allele = allele;
        rec->consumption = P->has_eco ? cons : 0ull;
        rec->R = R;
        rec->f = f_next;
        rec->pad = 0;
        st->next_S = (uint32_t)S_new;
        st->next_f = f_next;
        st->next_R = P->has_eco ? R : R_prev;
        st->next_status = status;
    }
}

// Make generation g the population's current one (one thread of the block
// that finished the last compaction bucket, after every block has read the
// state and the closing warp's next_* values are visible).
__device__ void commit_state(DevState *st, uint32_t g) {
    const uint32_t S = ld_relaxed_u32(&st->next_S), f = ld_relaxed_u32(&st->next_f);
    const int32_t status = (int32_t)ld_relaxed_u32(reinterpret_cast<const uint32_t *>(&st->next_status));
    const double R = ld_relaxed_f64(&st->next_R);
    if (st->status == SPG_OK) st->status = status;
    st->f = f;
    st->S = S;
    st->R = R;
    st->done = 0;
    st->gen = g;
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
    const uint32_t target = ld_relaxed_u32(&st->target);
    s.active = s.S > 0u && status == SPG_OK && s.gen < target;
    return s;
}

// ------------------------------------------------------- async copies
__device__ __forceinline__ void cp_async_16(uint32_t saddr, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_8(uint32_t saddr, const void *g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Shared-memory staging of parent records: a ring of kStages stages; per
// stage, item, parent (0 mother, 1 father) and chunk q one chunk per thread,
// chunks of consecutive threads adjacent (conflict-free 8/16-byte accesses),
// followed by each item's survival and mutation-count draws.  A thread only
// ever reads the slots it wrote itself, so the ring needs no block barrier.
template <int W, int ITEMS>
struct Staging {
    static constexpr int kChunkBytes = (W == 1) ? 8 : 16;
    static constexpr int kChunks = (W == 1) ? 1 : W / 2;  // per record
    static constexpr uint32_t kRecBytes = (uint32_t)ITEMS * 2u * kChunks * kBlock * kChunkBytes;
    static constexpr uint32_t kDrawBytes = (uint32_t)ITEMS * kBlock * 8u;
    static constexpr uint32_t kStageBytes = kRecBytes + kDrawBytes;
    // as many stages (2..4) as fit in ~110 KB, so two blocks share an SM
    static constexpr int kStages = (4u * kStageBytes <= 112640u) ? 4 : (3u * kStageBytes <= 112640u) ? 3 : 2;
    static constexpr uint32_t kBytes = (uint32_t)kStages * kStageBytes;
    __device__ static __forceinline__ uint32_t offset(int stage, int it, int parent, int q, int tid) {
        return (uint32_t)stage * kStageBytes +
               ((((uint32_t)it * 2u + (uint32_t)parent) * kChunks + (uint32_t)q) * kBlock + (uint32_t)tid) *
                   kChunkBytes;
    }
    __device__ static __forceinline__ uint32_t draw_offset(int stage, int it, int tid) {
        return (uint32_t)stage * kStageBytes + kRecBytes + ((uint32_t)it * kBlock + (uint32_t)tid) * 8u;
    }
};

// Parents of one tile: indices into the previous generation and the
// survival / mutation-count draws of each item.
template <int ITEMS>
struct TileDraws {
    uint32_t mom[ITEMS], dad[ITEMS], u_surv[ITEMS], u_mut[ITEMS];
};

struct SegCtx {
    const PopParams *P;
    const uint32_t *par;
    uint32_t *chi;
    const uint32_t *sin;
    uint32_t *alive;
    uint32_t *bucket_now;
    const unsigned long long *survw;   // weighted parents: [2][n] survivor index | role threshold << 32
    uint16_t *obin;                    // weighted parents: bins of the offspring formed
    uint32_t n, S, f, g, rep, k0, k1, kmax, nplanes, shift, ndplanes;
    int32_t e_min, bias, d_min;
    bool has_eco;
};

// Weighted parents (pi = 0 mother, 1 father) by bounded rejection sampling:
// proposal k draws a uniform survivor rank and an acceptance value (lanes
// 2(k%2), 2(k%2)+1 of Philox sub pi<<8 | k/2) and is taken when the
// survivor's bin threshold is certain or above the value; the last proposal
// stands if all kMateAttempts are rejected.  Proposals go in pairs (one
// Philox block), both roles together, so four gathers are in flight at once;
// the first accepted proposal in order is the parent, as if they were tried
// one at a time.  A gathered word carries the survivor's threshold for the
// role (looked up once per survivor by the compaction), so a proposal is one
// 8-byte read and a comparison.
static_assert(kMateAttempts % 2 == 0, "whole Philox blocks of proposals");

// Proposals k and k+1 of one role: whether one was taken, and the parent (the
// first taken, else proposal k+1).
__device__ __forceinline__ bool weighted_pair(const uint4 &d, unsigned long long e0, unsigned long long e1,
                                              uint32_t &parent) {
    const uint32_t t0 = (uint32_t)(e0 >> 32), t1 = (uint32_t)(e1 >> 32);
    const bool a0 = t0 == kCertain || d.y < t0, a1 = t1 == kCertain || d.w < t1;
    parent = a0 ? (uint32_t)e0 : (uint32_t)e1;
    return a0 || a1;
}

__device__ __forceinline__ void weighted_parents(const SegCtx &c, uint32_t j, uint32_t &mom, uint32_t &dad) {
    bool open_m = true, open_f = true;
    for (uint32_t k = 0; k < kMateAttempts && (open_m || open_f); k += 2) {
        const uint32_t sub = (kMateW << 24) | (k >> 1);
        uint4 dm = make_uint4(0u, 0u, 0u, 0u), df = dm;
        unsigned long long em0 = 0, em1 = 0, ef0 = 0, ef1 = 0;
        if (open_m) {
            dm = philox(make_uint4(j, c.g, c.rep, sub), c.k0, c.k1);
            em0 = __ldcg(c.survw + __umulhi(dm.x, c.S));
            em1 = __ldcg(c.survw + __umulhi(dm.z, c.S));
        }
        if (open_f) {
            df = philox(make_uint4(j, c.g, c.rep, sub | (1u << 8)), c.k0, c.k1);
            ef0 = __ldcg(c.survw + c.n + __umulhi(df.x, c.S));
            ef1 = __ldcg(c.survw + c.n + __umulhi(df.z, c.S));
        }
        if (open_m) open_m = !weighted_pair(dm, em0, em1, mom);
        if (open_f) open_f = !weighted_pair(df, ef0, ef1, dad);
    }
}

template <int ITEMS, bool WEIGHTED = false>
__device__ __forceinline__ void draw_parents(const SegCtx &c, uint32_t base, int tid, TileDraws<ITEMS> &d) {
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const uint32_t j = base + (uint32_t)(it * kBlock + tid);
        d.mom[it] = d.dad[it] = d.u_surv[it] = d.u_mut[it] = 0u;
        if (j < c.n) {
            const uint4 r = philox(make_uint4(j, c.g, c.rep, kMate << 24), c.k0, c.k1);
            // survivor indices through L2 only: random 4-byte reads would
            // evict the threshold table from L1
            if constexpr (WEIGHTED) {
                weighted_parents(c, j, d.mom[it], d.dad[it]);
            } else {
                d.mom[it] = __ldcg(c.sin + __umulhi(r.x, c.S));
                d.dad[it] = __ldcg(c.sin + __umulhi(r.y, c.S));
            }
            d.u_surv[it] = r.z;
            d.u_mut[it] = r.w;
        }
    }
}

template <int W, int ITEMS>
__device__ __forceinline__ void stage_parents(const SegCtx &c, uint32_t base, int tid, const TileDraws<ITEMS> &d,
                                              unsigned char *s_dyn, uint32_t s_base, int stage) {
    using St = Staging<W, ITEMS>;
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const uint32_t j = base + (uint32_t)(it * kBlock + tid);
        if (j < c.n) {
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const uint32_t *src = c.par + (size_t)(p ? d.dad[it] : d.mom[it]) * (2 * W);
#pragma unroll
                for (int q = 0; q < St::kChunks; ++q) {
                    const uint32_t sa = s_base + St::offset(stage, it, p, q, tid);
                    if constexpr (W == 1) cp_async_8(sa, src);
                    else cp_async_16(sa, src + 4 * q);
                }
            }
            *reinterpret_cast<uint2 *>(s_dyn + St::draw_offset(stage, it, tid)) =
                make_uint2(d.u_surv[it], d.u_mut[it]);
        }
    }
}

template <int W, int ITEMS>
__device__ __forceinline__ void read_parent(const unsigned char *s_dyn, int stage, int it, int p, int tid,
                                            uint32_t (&r)[2 * W]) {
    using St = Staging<W, ITEMS>;
    if constexpr (W == 1) {
        const uint2 v = *reinterpret_cast<const uint2 *>(s_dyn + St::offset(stage, it, p, 0, tid));
        r[0] = v.x;
        r[1] = v.y;
    } else {
#pragma unroll
        for (int q = 0; q < St::kChunks; ++q) {
            const uint4 v = *reinterpret_cast<const uint4 *>(s_dyn + St::offset(stage, it, p, q, tid));
            r[4 * q + 0] = v.x;
            r[4 * q + 1] = v.y;
            r[4 * q + 2] = v.z;
            r[4 * q + 3] = v.w;
        }
    }
}

struct ThreadStats {
    long long sum_raw = 0, sum_raw_s = 0;
    unsigned long long sum_raw2 = 0, cons = 0;
    uint32_t het = 0, allele = 0;
    int mn = INT_MAX, mx = INT_MIN;
};

// One tile: gametes (B), phenotype (C), survival (D), bitmap (E, first half).
template <int W, int ITEMS, bool LINKED, bool WEIGHTED>
__device__ __forceinline__ uint32_t offspring_tile(const SegCtx &c, uint32_t base, int tid, int lane, int warp,
                                                   const unsigned char *s_dyn, int stage, const uint32_t *s_planes,
                                                   const uint32_t *s_cdf, ThreadStats &ts, const LinkSmem &lk,
                                                   const uint32_t *s_dplanes) {
    constexpr int NW = kBlock / 32;
    using St = Staging<W, ITEMS>;
    uint32_t alive_count = 0;  // the warp's survivors (same in every lane)
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const uint32_t j = base + (uint32_t)(it * kBlock + tid);
        bool alive = false;
        if (j < c.n) {
            const uint2 u = *reinterpret_cast<const uint2 *>(s_dyn + St::draw_offset(stage, it, tid));
            uint32_t pm[2 * W], pf[2 * W], ch[2 * W];
            read_parent<W, ITEMS>(s_dyn, stage, it, 0, tid, pm);
            read_parent<W, ITEMS>(s_dyn, stage, it, 1, tid, pf);
            if constexpr (LINKED) {
                // (B) gametes under the linkage map
                uint32_t mm[W], mf[W];
                linked_mask<W>(lk, j, c.g, c.rep, 0u, c.k0, c.k1, mm);
                linked_mask<W>(lk, j, c.g, c.rep, 1u, c.k0, c.k1, mf);
#pragma unroll
                for (int w = 0; w < W; ++w) {
                    ch[w] = (pm[w] & ~mm[w]) | (pm[W + w] & mm[w]);
                    ch[W + w] = (pf[w] & ~mf[w]) | (pf[W + w] & mf[w]);
                }
            } else {
            // (B) gametes: stream q = 2w + parent is lane q%4 of sub q/4
#pragma unroll
            for (int q4 = 0; q4 < (2 * W + 3) / 4; ++q4) {
                const uint4 d = philox(make_uint4(j, c.g, c.rep, (kRecomb << 24) | (uint32_t)q4), c.k0, c.k1);
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const int q = 4 * q4 + l;
                    if (q < 2 * W) {
                        const int w = q >> 1;
                        const uint32_t m = lane_of(d, l);
                        if ((q & 1) == 0) ch[w] = (pm[w] & ~m) | (pm[W + w] & m);
                        else ch[W + w] = (pf[w] & ~m) | (pf[W + w] & m);
                    }
                }
            }
            }
            // (B) mutation count from the CDF (none below its first entry,
            // the common case), positions on the rare path
            if (c.kmax != 0u && u.y >= s_cdf[0]) {
                uint32_t k = 0;
                for (uint32_t i = 0; i < c.kmax; ++i) k += (u.y >= s_cdf[i]) ? 1u : 0u;
                mutate<W>(ch, k, j, c.g, c.rep, c.k0, c.k1);
            }
            store_record<W>(c.chi + (size_t)j * (2 * W), ch);

            // (C) phenotype, (D) survival
            uint32_t allele, hz;
            int32_t raw = phenotype<W>(ch, s_planes, c.nplanes, c.e_min, allele, hz);
            raw += dominance_part<W>(ch, s_dplanes, c.ndplanes, c.d_min, hz);  // hz is set by the line above
            const long long v = (long long)raw + (long long)c.bias;
            const uint32_t bin = v < 0 ? 0u : (uint32_t)min(v >> c.shift, (long long)(kBins - 1));
            if constexpr (WEIGHTED) c.obin[j] = (uint16_t)bin;
            uint32_t thr = __ldg(&c.P->table[bin]);
            if (c.f != kCertain) thr = __umulhi(thr, c.f);
            alive = (thr == kCertain) || (u.x < thr);

            ts.sum_raw += raw;
            ts.sum_raw2 += (unsigned long long)((long long)raw * (long long)raw);
            ts.mn = min(ts.mn, raw);
            ts.mx = max(ts.mx, raw);
            ts.het += hz;
            ts.allele += allele;
            if (alive) {
                ts.sum_raw_s += raw;
                if (c.has_eco) ts.cons += __ldg(&c.P->attack[bin]);
            }
        }
        // (E, first half) alive bitmap word (base + it*kBlock + 32*warp)/32
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, alive);
        if (lane == 0) c.alive[(base >> 5) + (uint32_t)(it * NW + warp)] = bal;
        alive_count += __popc(bal);
    }
    return alive_count;
}

// --------------------------------------------- offspring kernel (Fig. 1A-D)
template <int W, int ITEMS, bool LINKED, bool WEIGHTED>
__global__ void __launch_bounds__(kBlock, SPG_MIN_BLOCKS) k_offspring(const __grid_constant__ GenArgs a) {
    constexpr int NW = kBlock / 32;
    constexpr uint32_t TILE = (uint32_t)(kBlock * ITEMS);
    static_assert(kBucket % TILE == 0, "tiles must not straddle compaction buckets");
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ __align__(16) uint32_t s_planes[kMaxPlanes * W];
    __shared__ __align__(16) uint32_t s_dplanes[kMaxPlanes * W];
    __shared__ uint32_t s_cdf[kMaxKmax];
    __shared__ long long s_ll[2][NW];
    __shared__ unsigned long long s_ull[2][NW];
    __shared__ uint32_t s_u32[3][NW];
    __shared__ int s_mm[2][NW];
    constexpr int LK = LINKED ? 1 : 0;  // linkage-map tables only in the linked variant
    __shared__ uint32_t s_lcdf[LK * kMaxKmax + 1], s_lcum[LK * kMaxLoci + 1];
    __shared__ uint8_t s_lchrom[LK * kMaxLoci + 1];
    __shared__ uint16_t s_lfirst[LK * kMaxChrom + 1], s_lclast[LK * kMaxChrom + 1];
    __shared__ uint32_t s_lguide[LK * kLinkGuide + 1];
    LinkSmem lk{s_lcdf, s_lcum, s_lchrom, s_lfirst, s_lclast, s_lguide, 0u, 0u};

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(s_dyn);
    const uint32_t T = a.total_tiles, G = gridDim.x;
    uint32_t t = (uint32_t)(((unsigned long long)T * blockIdx.x) / G);
    const uint32_t t_end = (uint32_t)(((unsigned long long)T * (blockIdx.x + 1)) / G);
    if (t >= t_end) return;
    uint32_t si = a.nsegs == 1u ? 0u : __ldg(a.tile_seg + t);

    while (t < t_end) {
        const Segment &sg = a.nsegs == 1u ? a.one : a.segs[si];
        const uint32_t seg_end = min(t_end, sg.tile_begin + sg.ntiles);
        const PopNow now = read_state(sg.state);
        if (now.active) {
            SegCtx c;
            c.P = sg.prm;
            c.n = sg.n;
            c.S = now.S;
            c.f = now.f;
            c.g = now.gen + 1u;
            c.par = sg.geno[now.gen & 1u];
            c.chi = sg.geno[(now.gen + 1u) & 1u];
            c.sin = sg.surv[now.gen & 1u];
            c.alive = sg.alive;
            c.survw = sg.survw;
            c.obin = sg.obin;
            c.bucket_now = sg.bucket_sum + (c.g & 1u) * sg.nbuckets;
            uint32_t *bucket_next = sg.bucket_sum + ((c.g + 1u) & 1u) * sg.nbuckets;
            c.rep = c.P->rep;
            c.k0 = c.P->key0;
            c.k1 = c.P->key1;
            c.kmax = c.P->kmax;
            c.nplanes = c.P->nplanes;
            c.shift = c.P->shift;
            c.e_min = c.P->e_min;
            c.d_min = c.P->d_min;
            c.ndplanes = c.P->ndplanes;
            c.bias = c.P->bias;
            c.has_eco = c.P->has_eco != 0u;

            __syncthreads();  // the previous population's tables are no longer read
            for (uint32_t i = tid; i < c.nplanes * W; i += kBlock) s_planes[i] = c.P->planes[i];
            for (uint32_t i = tid; i < c.ndplanes * W; i += kBlock) s_dplanes[i] = c.P->dplanes[i];
            if (tid < kMaxKmax) s_cdf[tid] = (uint32_t)tid < c.kmax ? c.P->cdf[tid] : 0u;
            if constexpr (LINKED) {
                const LinkParams *lp = c.P->link;
                lk.kmax = lp->kmax;
                lk.nchrom = lp->nchrom;
                for (uint32_t i = tid; i < 32u * W; i += kBlock) {
                    s_lcum[i] = lp->cum[i];
                    s_lchrom[i] = lp->chrom[i];
                }
                if (tid < kMaxKmax) s_lcdf[tid] = lp->cdf[tid];
                for (uint32_t i = tid; i < (uint32_t)kLinkGuide; i += kBlock) s_lguide[i] = lp->guide[i];
                if (tid < kMaxChrom) {
                    s_lfirst[tid] = lp->first[tid];
                    s_lclast[tid] = lp->clast[tid];
                }
            }
            __syncthreads();

            const uint32_t lt0 = t - sg.tile_begin, lt1 = seg_end - sg.tile_begin;
            ThreadStats ts;
            uint32_t warp_alive = 0, bucket_alive = 0, bucket_cur = (lt0 * TILE) / kBucket;

            // software pipeline over the block's tiles: parent records (and
            // each item's draws) are staged kStages-1 tiles ahead; survivor
            // indices are fetched two iterations before they are staged.
            // Every iteration commits one cp.async group (empty near the end),
            // so waiting for all but the newest R groups completes tile lt's.
            using St = Staging<W, ITEMS>;
            constexpr int R = St::kStages - 1;
            TileDraws<ITEMS> dA, dB;
            for (int k = 0; k < R; ++k) {
                const uint32_t tk = lt0 + (uint32_t)k;
                if (tk < lt1) {
                    draw_parents<ITEMS, WEIGHTED>(c, tk * TILE, tid, dA);
                    stage_parents<W, ITEMS>(c, tk * TILE, tid, dA, s_dyn, s_base, k);
                }
                cp_async_commit();
            }
            if (lt0 + R < lt1) draw_parents<ITEMS, WEIGHTED>(c, (lt0 + R) * TILE, tid, dA);
            if (lt0 + R + 1 < lt1) draw_parents<ITEMS, WEIGHTED>(c, (lt0 + R + 1) * TILE, tid, dB);
            int stage = 0;
            for (uint32_t lt = lt0; lt < lt1; ++lt) {
                const uint32_t base = lt * TILE;
                const int ahead = stage == 0 ? R : stage - 1;  // (stage + R) % kStages
                if (lt + R < lt1) stage_parents<W, ITEMS>(c, base + R * TILE, tid, dA, s_dyn, s_base, ahead);
                cp_async_commit();
                dA = dB;
                if (lt + R + 2 < lt1) draw_parents<ITEMS, WEIGHTED>(c, base + (R + 2) * TILE, tid, dB);
                cp_async_wait<R>();
                if (tid == 0 && base % kBucket == 0u) bucket_next[base / kBucket] = 0u;
                const uint32_t bkt = base / kBucket;
                if (bkt != bucket_cur) {
                    if (lane == 0 && bucket_alive) atomicAdd(&c.bucket_now[bucket_cur], bucket_alive);
                    bucket_alive = 0;
                    bucket_cur = bkt;
                }
                const uint32_t cnt =
                    offspring_tile<W, ITEMS, LINKED, WEIGHTED>(c, base, tid, lane, warp, s_dyn, stage, s_planes, s_cdf,
                                                               ts, lk, s_dplanes);
                bucket_alive += cnt;
                warp_alive += cnt;
                stage = stage + 1 == St::kStages ? 0 : stage + 1;
            }
            cp_async_wait<0>();
            if (lane == 0 && bucket_alive) atomicAdd(&c.bucket_now[bucket_cur], bucket_alive);

            // statistics of this block's tiles: exact warp sums, one atomic
            // per field into one of the population's accumulator copies
            const long long w_raw = warp_sum_i64(ts.sum_raw), w_raw_s = warp_sum_i64(ts.sum_raw_s);
            const unsigned long long w_raw2 = warp_sum_u64(ts.sum_raw2), w_cons = warp_sum_u64(ts.cons);
            const uint32_t w_het = __reduce_add_sync(0xFFFFFFFFu, ts.het);
            const uint32_t w_allele = __reduce_add_sync(0xFFFFFFFFu, ts.allele);
            const int w_mn = __reduce_min_sync(0xFFFFFFFFu, ts.mn), w_mx = __reduce_max_sync(0xFFFFFFFFu, ts.mx);
            if (lane == 0) {
                s_ll[0][warp] = w_raw;
                s_ll[1][warp] = w_raw_s;
                s_ull[0][warp] = w_raw2;
                s_ull[1][warp] = w_cons;
                s_u32[0][warp] = w_het;
                s_u32[1][warp] = w_allele;
                s_u32[2][warp] = warp_alive;
                s_mm[0][warp] = w_mn;
                s_mm[1][warp] = w_mx;
            }
            __syncthreads();
            if (tid == 0) {
                long long a0 = 0, a1 = 0;
                unsigned long long b0 = 0, b1 = 0, hz = 0, al = 0, sv = 0;
                int m0 = INT_MAX, m1 = INT_MIN;
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    a0 += s_ll[0][w];
                    a1 += s_ll[1][w];
                    b0 += s_ull[0][w];
                    b1 += s_ull[1][w];
                    hz += s_u32[0][w];
                    al += s_u32[1][w];
                    sv += s_u32[2][w];
                    m0 = min(m0, s_mm[0][w]);
                    m1 = max(m1, s_mm[1][w]);
                }
                StatAcc *acc = sg.acc + blockIdx.x % kAccCopies;
                atomicAdd(&acc->s, sv);
                atomicAdd(reinterpret_cast<unsigned long long *>(&acc->sum_raw), (unsigned long long)a0);
                atomicAdd(reinterpret_cast<unsigned long long *>(&acc->sum_raw_s), (unsigned long long)a1);
                atomicAdd(&acc->sum_raw2, b0);
                if (b1) atomicAdd(&acc->cons, b1);
                atomicAdd(&acc->het, hz);
                atomicAdd(&acc->allele, al);
                atomicMin(&acc->mn, m0);
                atomicMax(&acc->mx, m1);
            }
        }
        t = seg_end;
        ++si;
    }
}

// ------------------------------------------------ continuous allelic values
// A normal step in raw units from twelve Philox lanes (Irwin-Hall(12)): the
// lanes of subs sub0..sub0+2 summed, t = sum - 6 * 2^32, step =
// ((t >> 8) * s) >> 40 for a Q16 scale s (see spegg.h).
__device__ __forceinline__ int32_t irwin_hall_step(uint32_t j, uint32_t g, uint32_t rep, uint32_t purpose,
                                                   uint32_t sub0, long long s, uint32_t k0, uint32_t k1) {
    unsigned long long sum = 0;
#pragma unroll
    for (uint32_t q = 0; q < 3; ++q) {
        const uint4 d = philox(make_uint4(j, g, rep, (purpose << 24) | (sub0 + q)), k0, k1);
        sum += (unsigned long long)d.x + d.y + d.z + d.w;
    }
    const long long t = (long long)sum - 6LL * 4294967296LL;
    return (int32_t)(((t >> 8) * s) >> 40);
}

// Eight packed int16 values (one 16-byte access) per lane and haplotype.
// val16: value `half` (0 low, 1 high) of a packed word, sign-extended.
__device__ __forceinline__ int32_t val16(uint32_t w, uint32_t half) {
    return half ? (int32_t)w >> 16 : (int32_t)(int16_t)(w & 0xFFFFu);
}
__device__ __forceinline__ uint32_t word_of(const uint4 &c, uint32_t q) {
    return q == 0u ? c.x : q == 1u ? c.y : q == 2u ? c.z : c.w;
}
__device__ __forceinline__ void set_word(uint4 &c, uint32_t q, uint32_t v) {
    if (q == 0u) c.x = v;
    else if (q == 1u) c.y = v;
    else if (q == 2u) c.z = v;
    else c.w = v;
}
// the values of b where bit k (k = 0..7, value k of the eight) of `bits` is set, of a elsewhere
__device__ __forceinline__ uint4 pick8(const uint4 &a, const uint4 &b, uint32_t bits) {
    auto sel = [](uint32_t x, uint32_t y, uint32_t two) {
        const uint32_t m = ((two & 1u) ? 0x0000FFFFu : 0u) | ((two & 2u) ? 0xFFFF0000u : 0u);
        return (x & ~m) | (y & m);
    };
    return make_uint4(sel(a.x, b.x, bits), sel(a.y, b.y, bits >> 2), sel(a.z, b.z, bits >> 4),
                      sel(a.w, b.w, bits >> 6));
}
// value k of the eight moved by `step`, clamped to the int16 range
__device__ __forceinline__ void add_step(uint4 &c, uint32_t k, int32_t step) {
    const uint32_t q = k >> 1, half = k & 1u, w = word_of(c, q);
    const int32_t nv = min(max(val16(w, half) + step, -32768), 32767);
    set_word(c, q, half ? (w & 0xFFFFu) | ((uint32_t)nv << 16) : (w & 0xFFFF0000u) | ((uint32_t)nv & 0xFFFFu));
}

// Generation kernel of a continuous-allele population (S2 "Genetics").  A
// group of G = L/8 lanes forms one offspring, lane li owning loci
// 8li .. 8li+7 of both haplotypes, so parent and child records (2L int16)
// move in coalesced 16-byte accesses; a warp holds 32/G groups, each forming
// U offspring at a time with all their parent loads issued before any is
// used.  The per-offspring draws (parents, survival and mutation uniforms,
// environmental step, gamete-mask streams) are made once per warp, one
// offspring per lane, and handed to the groups by shuffles.  Parents, gamete
// bits, mutation counts and positions follow the biallelic model's draws;
// mutated values take Irwin-Hall steps; the phenotype is the group sum of the
// values plus the environmental step.  Survivors, statistics and the bitmap
// feed the same compaction kernel as the biallelic model.
constexpr int kContInFlight = 1;  // offspring a group of lanes forms at a time (four blocks per SM)

template <int G, int U>
__global__ void __launch_bounds__(kBlock, 4) k_offspring_cont(const __grid_constant__ GenArgs a) {
    constexpr uint32_t L = 8u * G;
    constexpr int NW = kBlock / 32, NO = 32 / G;
    constexpr int NST = G >= 8 ? G / 8 : 1;  // gamete-mask streams per offspring (2 words per parent each)
    constexpr int PER_T = NO * NST;          // (offspring, stream) pairs one step of the warp uses
    constexpr int T_PER_SLOT = 32 / PER_T;   // steps served by one register slot of those pairs
    static_assert(G >= 4 && G <= 32 && (G & (G - 1)) == 0 && G % U == 0, "group of 4..32 lanes");
    __shared__ uint32_t s_cdf[kMaxKmax];
    __shared__ uint32_t s_mpos[NW * NO][kMaxKmax];
    __shared__ long long s_ll[2][NW];
    __shared__ unsigned long long s_ull[4][NW];
    __shared__ uint32_t s_u32[2][NW];
    __shared__ int s_mm[2][NW];
    const Segment &sg = a.one;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const PopNow now = read_state(sg.state);
    if (!now.active) return;
    const PopParams *P = sg.prm;
    const uint32_t n = sg.n, S = now.S, g = now.gen + 1u, f = now.f;
    const uint32_t rep = P->rep, k0 = P->key0, k1 = P->key1, kmax = P->kmax, shift_bin = P->shift;
    const int32_t bias = P->bias;
    const long long s_mut = P->s_mut, s_env = P->s_env;
    const bool has_eco = P->has_eco != 0u;
    const uint4 *par = reinterpret_cast<const uint4 *>(sg.geno[now.gen & 1u]);
    uint4 *chi = reinterpret_cast<uint4 *>(sg.geno[g & 1u]);
    const uint32_t *sin = sg.surv[now.gen & 1u];
    uint32_t *bucket_now = sg.bucket_sum + (g & 1u) * sg.nbuckets;
    uint32_t *bucket_next = sg.bucket_sum + ((g + 1u) & 1u) * sg.nbuckets;
    if (tid < kMaxKmax) s_cdf[tid] = (uint32_t)tid < kmax ? P->cdf[tid] : 0u;
    __syncthreads();
    const uint32_t base = blockIdx.x * (uint32_t)kBlock;
    if (tid == 0 && base % kBucket == 0u) bucket_next[base / kBucket] = 0u;
    const uint32_t wbase = base + (uint32_t)warp * 32u;
    const uint32_t grp = (uint32_t)lane / G, li = (uint32_t)lane % G;
    const uint32_t gmask = G == 32 ? 0xFFFFFFFFu : ((1u << G) - 1u) << (grp * G);
    const uint32_t wv = li >> 2, sh = (li & 3u) * 8u;  // this lane's mask word and first bit
    uint32_t *mpos = s_mpos[warp * NO + grp];
    constexpr uint32_t R4 = L / 4;  // 16-byte units per record

    // (A) the draws of offspring wbase + lane and its parents' indices
    const uint32_t jl = wbase + (uint32_t)lane;
    const uint4 rl = philox(make_uint4(jl, g, rep, kMate << 24), k0, k1);
    const uint32_t mom_l = jl < n ? __ldcg(sin + __umulhi(rl.x, S)) : 0u;
    const uint32_t dad_l = jl < n ? __ldcg(sin + __umulhi(rl.y, S)) : 0u;
    const int32_t env_l = s_env != 0 ? irwin_hall_step(jl, g, rep, kEnv, 0u, s_env, k0, k1) : 0;
    // (B) gamete-mask streams: slot q of lane k holds pair 32q + k, i.e. step
    // (32q + k) / PER_T, group ((32q + k) % PER_T) / NST, stream (32q + k) % NST
    uint4 dml[NST];
#pragma unroll
    for (int q = 0; q < NST; ++q) {
        const uint32_t pr = 32u * (uint32_t)q + (uint32_t)lane, t = pr / PER_T, rem = pr % PER_T;
        dml[q] = philox(make_uint4(wbase + t * NO + rem / NST, g, rep, (kRecomb << 24) | (rem % NST)), k0, k1);
    }

    long long sum_raw = 0, sum_raw_s = 0;
    unsigned long long sum_raw2 = 0, cons = 0, lane_allele = 0;
    uint32_t lane_het = 0, alive_bits = 0, nsurv = 0;
    int mn = INT_MAX, mx = INT_MIN;
    for (uint32_t it = 0; it < (uint32_t)(G / U); ++it) {
        uint32_t bit[U], rz[U], rw[U];
        int32_t env[U];
        uint4 m0[U], m1[U], f0[U], f1[U];
        // the group's U offspring: parents and draws from their lanes, then all the records
#pragma unroll
        for (int u = 0; u < U; ++u) {
            bit[u] = (it * U + (uint32_t)u) * NO + grp;
            const uint32_t mom = __shfl_sync(0xFFFFFFFFu, mom_l, bit[u]), dad = __shfl_sync(0xFFFFFFFFu, dad_l, bit[u]);
            rz[u] = __shfl_sync(0xFFFFFFFFu, rl.z, bit[u]);
            rw[u] = __shfl_sync(0xFFFFFFFFu, rl.w, bit[u]);
            env[u] = __shfl_sync(0xFFFFFFFFu, env_l, bit[u]);
            const uint4 z = make_uint4(0u, 0u, 0u, 0u);
            const bool ok = wbase + bit[u] < n;
            const uint4 *pm = par + (size_t)mom * R4, *pf = par + (size_t)dad * R4;
            m0[u] = ok ? __ldg(pm + li) : z;
            m1[u] = ok ? __ldg(pm + G + li) : z;
            f0[u] = ok ? __ldg(pf + li) : z;
            f1[u] = ok ? __ldg(pf + G + li) : z;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t j = wbase + bit[u], t = it * U + (uint32_t)u;
            const bool ok = j < n;
            // (B) gametes: mask word wv of the mother (stream 2wv) and father (2wv + 1)
            const uint32_t q = t / T_PER_SLOT;
            uint4 dsrc = dml[0];
#pragma unroll
            for (int qq = 1; qq < NST; ++qq)
                if (q == (uint32_t)qq) dsrc = dml[qq];
            const uint32_t src = (t % T_PER_SLOT) * PER_T + grp * NST + (wv >> 1);
            const uint32_t dx = __shfl_sync(0xFFFFFFFFu, dsrc.x, src), dy = __shfl_sync(0xFFFFFFFFu, dsrc.y, src);
            const uint32_t dz = __shfl_sync(0xFFFFFFFFu, dsrc.z, src), dw = __shfl_sync(0xFFFFFFFFu, dsrc.w, src);
            const uint32_t mm = (wv & 1u) ? dz : dx, mf = (wv & 1u) ? dw : dy;
            uint4 c0 = pick8(m0[u], m1[u], (mm >> sh) & 0xFFu), c1 = pick8(f0[u], f1[u], (mf >> sh) & 0xFFu);
            // (B) mutation: the biallelic count and distinct positions, each
            // mutated value moved by an Irwin-Hall step by the lane owning it
            const uint32_t u_mut = rw[u];
            if (ok && kmax != 0u && u_mut >= s_cdf[0]) {  // the same in the whole group
                uint32_t K = 0;
                for (uint32_t qk = 0; qk < kmax; ++qk) K += u_mut >= s_cdf[qk] ? 1u : 0u;
                uint32_t chosen = 0;
                uint4 dp = make_uint4(0u, 0u, 0u, 0u);
                for (uint32_t d = 0; d < (uint32_t)kMutDraws && chosen < K; ++d) {
                    if ((d & 3u) == 0u) dp = philox(make_uint4(j, g, rep, (kMutPos << 24) | (d >> 2)), k0, k1);
                    const uint32_t pos = __umulhi(lane_of(dp, (int)(d & 3u)), 2u * L);
                    bool dup = false;
                    for (uint32_t qk = 0; qk < chosen; ++qk) dup |= mpos[qk] == pos;
                    if (!dup) {
                        if (li == 0u) mpos[chosen] = pos;
                        __syncwarp(gmask);
                        ++chosen;
                    }
                }
                for (uint32_t m = 0; m < chosen; ++m) {
                    const uint32_t pos = mpos[m], locus = pos >= L ? pos - L : pos;
                    if ((locus >> 3) == li) {
                        const int32_t step = irwin_hall_step(j, g, rep, kMutSize, 3u * m, s_mut, k0, k1);
                        if (pos >= L) add_step(c1, locus & 7u, step);
                        else add_step(c0, locus & 7u, step);
                    }
                }
                __syncwarp(gmask);  // positions are rewritten by the group's next offspring
            }
            if (ok) {
                chi[(size_t)j * R4 + li] = c0;
                chi[(size_t)j * R4 + G + li] = c1;
            }
            // this lane's part of the phenotype sum, its heterozygous loci and squares
            int32_t part = 0;
            uint32_t het = 0;
            unsigned long long sq = 0;
#pragma unroll
            for (uint32_t k = 0; k < 8u; ++k) {
                const int32_t x = val16(word_of(c0, k >> 1), k & 1u), y = val16(word_of(c1, k >> 1), k & 1u);
                part += x + y;
                het += x != y ? 1u : 0u;
                sq += (uint32_t)(x * x) + (uint32_t)(y * y);
            }
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
            // (C) phenotype: the sum of all values, plus the environmental step
            const int32_t raw = part + env[u];
            // (D) survival
            const long long v = (long long)raw + (long long)bias;
            const uint32_t bin = v < 0 ? 0u : (uint32_t)min(v >> shift_bin, (long long)(kBins - 1));
            uint32_t thr = __ldg(&P->table[bin]);
            if (f != kCertain) thr = __umulhi(thr, f);
            const bool alive = (thr == kCertain) || (rz[u] < thr);
            if (ok) {
                lane_het += het;
                lane_allele += sq;
                mn = min(mn, raw);
                mx = max(mx, raw);
                if (alive) alive_bits |= 1u << bit[u];
                if (li == 0u) {  // per-offspring sums once per group
                    sum_raw += raw;
                    sum_raw2 += (unsigned long long)((long long)raw * (long long)raw);
                    if (alive) {
                        ++nsurv;
                        sum_raw_s += raw;
                        if (has_eco) cons += __ldg(&P->attack[bin]);
                    }
                }
            }
        }
    }
    alive_bits = __reduce_or_sync(0xFFFFFFFFu, alive_bits);
    const uint32_t w_surv = __reduce_add_sync(0xFFFFFFFFu, nsurv);
    if (lane == 0 && wbase < n) {
        sg.alive[wbase >> 5] = alive_bits;
        if (w_surv) atomicAdd(&bucket_now[wbase / kBucket], w_surv);
    }
    // statistics over the warp: the per-offspring sums sit in the group
    // leaders, the het and allele sums in every lane
    const uint32_t w_het = __reduce_add_sync(0xFFFFFFFFu, lane_het);
    const unsigned long long w_allele = warp_sum_u64(lane_allele);
    const long long w_raw = (long long)warp_sum_u64((unsigned long long)sum_raw);
    const long long w_raw_s = (long long)warp_sum_u64((unsigned long long)sum_raw_s);
    const unsigned long long w_raw2 = warp_sum_u64(sum_raw2), w_cons = warp_sum_u64(cons);
    const int w_mn = __reduce_min_sync(0xFFFFFFFFu, mn), w_mx = __reduce_max_sync(0xFFFFFFFFu, mx);
    if (lane == 0) {
        s_ll[0][warp] = w_raw;
        s_ll[1][warp] = w_raw_s;
        s_ull[0][warp] = w_raw2;
        s_ull[1][warp] = w_cons;
        s_ull[2][warp] = w_allele;
        s_ull[3][warp] = w_surv;
        s_u32[0][warp] = w_het;
        s_mm[0][warp] = w_mn;
        s_mm[1][warp] = w_mx;
    }
    __syncthreads();
    if (tid == 0) {
        long long a0 = 0, a1 = 0;
        unsigned long long b0 = 0, b1 = 0, al = 0, sv = 0, hz = 0;
        int m0 = INT_MAX, m1 = INT_MIN;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            a0 += s_ll[0][w];
            a1 += s_ll[1][w];
            b0 += s_ull[0][w];
            b1 += s_ull[1][w];
            al += s_ull[2][w];
            sv += s_ull[3][w];
            hz += s_u32[0][w];
            m0 = min(m0, s_mm[0][w]);
            m1 = max(m1, s_mm[1][w]);
        }
        if (sv | hz | (unsigned long long)(m1 != INT_MIN)) {
            StatAcc *acc = sg.acc + blockIdx.x % kAccCopies;
            atomicAdd(&acc->s, sv);
            atomicAdd(reinterpret_cast<unsigned long long *>(&acc->sum_raw), (unsigned long long)a0);
            atomicAdd(reinterpret_cast<unsigned long long *>(&acc->sum_raw_s), (unsigned long long)a1);
            atomicAdd(&acc->sum_raw2, b0);
            if (b1) atomicAdd(&acc->cons, b1);
            atomicAdd(&acc->het, hz);
            atomicAdd(&acc->allele, al);
            atomicMin(&acc->mn, m0);
            atomicMax(&acc->mx, m1);
        }
    }
}

// Continuous founders: value of copy q = h*L + l is effect[l] (decoded from the
// offset-binary planes) when the biallelic founder draw of q is below p0.
template <int C>
__global__ void k_founders_cont(const PopParams *__restrict__ P, uint32_t *__restrict__ geno,
                                uint32_t *__restrict__ surv, uint32_t n, uint32_t p0) {
    constexpr uint32_t L = 32u * C, W = C;  // W = L / 32 words of the planes
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int16_t *rec = reinterpret_cast<int16_t *>(geno + (size_t)i * L);
    for (uint32_t q4 = 0; q4 < 2u * L / 4u; ++q4) {
        const uint4 d = philox(make_uint4(i, 0u, P->rep, (kFounder << 24) | q4), P->key0, P->key1);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const uint32_t q = 4u * q4 + (uint32_t)c, l = q % L;
            int32_t e = P->e_min;
            for (uint32_t b = 0; b < P->nplanes; ++b) e += (int32_t)((P->planes[b * W + l / 32u] >> (l % 32u)) & 1u) << b;
            rec[q] = (int16_t)(lane_of(d, c) < p0 ? e : 0);
        }
    }
    surv[i] = i;
}

// ---------------------------------------- compaction kernel (Fig. 1E, 1F)
// One block of kCompactThreads threads per bucket of kBucket offspring: its
// first kBucketWords threads write the survivors' indices, in offspring order,
// at offset (survivors of all earlier buckets) + (block scan of the bitmap
// words' popcounts); in a population's first bucket the extra warp closes the
// generation meanwhile (finalize_warp).  The block that finishes the last
// bucket commits the new state.  Every load that does not depend on the
// population state is issued together with it (both parities of the bucket
// counts are summed; the state picks one).
__device__ __forceinline__ void compaction_barrier() {
    asm volatile("bar.sync 1, %0;" ::"n"(kBucketWords) : "memory");  // the kBucketWords compaction threads
}

__device__ __forceinline__ void compact_bucket(const Segment &sg, uint32_t b) {
    constexpr int NW = kBucketWords / 32;
    __shared__ uint32_t s_warp[NW];
    __shared__ uint32_t s_prev[NW];
    __shared__ uint32_t s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool closer = tid >= (int)kBucketWords;  // the generation-closing warp
    const uint32_t valid_words = (sg.n + 31u) >> 5;
    const uint32_t w = b * kBucketWords + (uint32_t)tid;
    const uint32_t bits = (!closer && w < valid_words) ? __ldcg(sg.alive + w) : 0u;
    uint32_t prev0 = 0, prev1 = 0;
    for (uint32_t i = (uint32_t)tid; !closer && i < b; i += kBucketWords) {
        prev0 += __ldcg(sg.bucket_sum + i);
        prev1 += __ldcg(sg.bucket_sum + sg.nbuckets + i);
    }
    const PopNow now = read_state(sg.state);
    if (!now.active) return;
    const uint32_t g = now.gen + 1u;
    if (closer) {
        if (b == 0u) finalize_warp(sg, sg.prm, g, now.f);
        __threadfence();
    } else {
    const uint32_t prev = __reduce_add_sync(0xFFFFFFFFu, (g & 1u) ? prev1 : prev0);
    const uint32_t cnt = __popc(bits);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    if (lane == 0) s_prev[warp] = prev;
    compaction_barrier();
    uint32_t excl = incl - cnt;
#pragma unroll
    for (int q = 0; q < NW; ++q) {
        excl += q < warp ? s_warp[q] : 0u;
        excl += s_prev[q];
    }
    uint32_t *__restrict__ sout = sg.surv[(now.gen + 1u) & 1u];
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t w0 = b * kBucketWords + (uint32_t)warp * 32u;
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
        const uint32_t word = __shfl_sync(0xFFFFFFFFu, bits, k);
        const uint32_t r0 = __shfl_sync(0xFFFFFFFFu, excl, k);
        if ((word >> lane) & 1u) {
            const uint32_t rank = r0 + __popc(word & lt), idx = (w0 + (uint32_t)k) * 32u + (uint32_t)lane;
            sout[rank] = idx;
            if (sg.survw) {  // the survivor's acceptance thresholds as mother and as father
                const uint32_t bin = __ldcg(sg.obin + idx);
                const WeightParams *wt = sg.prm->weights;
                sg.survw[rank] = (unsigned long long)idx | ((unsigned long long)__ldg(&wt->acc[0][bin]) << 32);
                sg.survw[sg.n + rank] = (unsigned long long)idx | ((unsigned long long)__ldg(&wt->acc[1][bin]) << 32);
            }
        }
    }
    }
    // every block has read the state by now (its values fed the stores
    // above), and the closing warp of bucket 0 has published the next state
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&sg.state->done, 1u) == sg.nbuckets - 1u) ? 1u : 0u;
    __syncthreads();
    if (s_last && tid == 0) {
        __threadfence();
        commit_state(sg.state, g);
    }
}

__global__ void __launch_bounds__(kCompactThreads) k_compact(const __grid_constant__ GenArgs a) {
    const uint32_t bkt = blockIdx.x;
    if (a.nsegs == 1u) {
        compact_bucket(a.one, bkt);
    } else {
        const Segment &sg = a.segs[__ldg(a.bucket_seg + bkt)];
        compact_bucket(sg, bkt - sg.bucket_begin);
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

// survw[pi * n + r] = surv[r] | (role pi's threshold for the survivor's bin)
// << 32 for the current survivors, each bin from its record's genetic value
// (planes read from the parameters).
template <int W>
__global__ void k_survivor_bins(const PopParams *__restrict__ P, const uint32_t *__restrict__ geno,
                                const uint32_t *__restrict__ surv, uint32_t S, uint32_t n,
                                unsigned long long *__restrict__ survw) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= S) return;
    const uint32_t idx = surv ? surv[r] : r;
    uint32_t rec[2 * W];
    load_record<W>(geno + (size_t)idx * (2 * W), rec);
    uint32_t total = 0, het = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        total += __popc(rec[w]) + __popc(rec[W + w]);
        het += __popc(rec[w] ^ rec[W + w]);
    }
    int32_t raw = P->e_min * (int32_t)total + P->d_min * (int32_t)het;
    for (uint32_t b = 0; b < P->nplanes; ++b) {
        int32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t pl = P->planes[b * W + w];
            cnt += __popc(pl & rec[w]) + __popc(pl & rec[W + w]);
        }
        raw += cnt << b;
    }
    for (uint32_t b = 0; b < P->ndplanes; ++b) {
        int32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) cnt += __popc(P->dplanes[b * W + w] & (rec[w] ^ rec[W + w]));
        raw += cnt << b;
    }
    const long long v = (long long)raw + (long long)P->bias;
    const uint32_t bin = v < 0 ? 0u : (uint32_t)min(v >> P->shift, (long long)(kBins - 1));
    survw[r] = (unsigned long long)idx | ((unsigned long long)P->weights->acc[0][bin] << 32);
    survw[(size_t)n + r] = (unsigned long long)idx | ((unsigned long long)P->weights->acc[1][bin] << 32);
}

__global__ void k_set_state(DevState *st, StatAcc *acc, uint32_t gen, uint32_t S, uint32_t f, double R,
                            int32_t status, uint32_t target) {
    if (threadIdx.x == 0) {
        st->target = target;
        st->gen = gen;
        st->S = S;
        st->f = f;
        st->status = status;
        st->R = R;
        st->done = 0;
    }
    if (threadIdx.x < (unsigned)kAccCopies) clear_acc(acc + threadIdx.x);
}

}  // namespace

bool supported_items(uint32_t words, uint32_t items) {
    if (!(items == 1 || items == 2 || items == 4)) return false;
    return !(words == 8 && items == 4);
}
uint32_t tile_size(uint32_t items) { return (uint32_t)kBlock * items; }

GenKernel compact_kernel() { return &k_compact; }

OffspringKernel continuous_kernel(uint32_t n_loci) {
    OffspringKernel k;
    switch (n_loci) {
        case 32: k.fn = &k_offspring_cont<4, kContInFlight>; break;
        case 64: k.fn = &k_offspring_cont<8, kContInFlight>; break;
        case 128: k.fn = &k_offspring_cont<16, kContInFlight>; break;
        case 256: k.fn = &k_offspring_cont<32, kContInFlight>; break;
        default: return OffspringKernel{};
    }
    k.smem = 0;
    k.resident = 0;  // not persistent: one block per 256 offspring
    return k;
}

int launch_founders_cont(const PopParams *prm, uint32_t n_loci, uint32_t *geno, uint32_t *surv, uint32_t n,
                         uint32_t p0_q32, void *stream) {
    const dim3 grid((n + 127) / 128), block(128);
    cudaStream_t s = (cudaStream_t)stream;
    switch (n_loci) {
        case 32: k_founders_cont<1><<<grid, block, 0, s>>>(prm, geno, surv, n, p0_q32); break;
        case 64: k_founders_cont<2><<<grid, block, 0, s>>>(prm, geno, surv, n, p0_q32); break;
        case 128: k_founders_cont<4><<<grid, block, 0, s>>>(prm, geno, surv, n, p0_q32); break;
        case 256: k_founders_cont<8><<<grid, block, 0, s>>>(prm, geno, surv, n, p0_q32); break;
        default: return SPG_ERR_INVALID;
    }
    return cudaGetLastError() == cudaSuccess ? SPG_OK : SPG_ERR_CUDA;
}

namespace {
template <int W, int I, bool LINKED = false, bool WEIGHTED = false>
OffspringKernel make_offspring() {
    OffspringKernel k;
    k.fn = &k_offspring<W, I, LINKED, WEIGHTED>;
    k.smem = Staging<W, I>::kBytes;
    return k;
}

template <bool LINKED, bool WEIGHTED>
OffspringKernel variant_kernel(uint32_t words) {
    switch (words) {
        case 1: return make_offspring<1, 1, LINKED, WEIGHTED>();
        case 2: return make_offspring<2, 1, LINKED, WEIGHTED>();
        case 4: return make_offspring<4, 1, LINKED, WEIGHTED>();
        case 8: return make_offspring<8, 1, LINKED, WEIGHTED>();
        default: return OffspringKernel{};
    }
}
}  // namespace

OffspringKernel offspring_kernel(uint32_t words, uint32_t items, bool linked, bool weighted) {
    if (linked || weighted) {  // linkage maps and weighted parents: one offspring per thread
        if (items != 1u) return OffspringKernel{};
        if (linked && weighted) return variant_kernel<true, true>(words);
        return linked ? variant_kernel<true, false>(words) : variant_kernel<false, true>(words);
    }
#define SPG_CASE(Wv, Iv) \
    if (words == Wv && items == Iv) return make_offspring<Wv, Iv>();
    SPG_CASE(1, 1) SPG_CASE(1, 2) SPG_CASE(1, 4)
    SPG_CASE(2, 1) SPG_CASE(2, 2) SPG_CASE(2, 4)
    SPG_CASE(4, 1) SPG_CASE(4, 2) SPG_CASE(4, 4)
    SPG_CASE(8, 1) SPG_CASE(8, 2)
#undef SPG_CASE
    return OffspringKernel{};
}

int prepare_offspring(OffspringKernel &k) {
    if (!k.fn) return SPG_ERR_INVALID;
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(k.fn),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
    if (e != cudaSuccess) return SPG_ERR_CUDA;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void *>(k.fn), kBlock,
                                                      k.smem);
    if (e != cudaSuccess || per_sm <= 0) return SPG_ERR_CUDA;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return SPG_ERR_CUDA;
    k.resident = (uint32_t)per_sm * (uint32_t)sms;
    return SPG_OK;
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

int launch_survivor_bins(const PopParams *prm, uint32_t words, const uint32_t *geno, const uint32_t *surv,
                         uint32_t S, uint32_t n, unsigned long long *survw, void *stream) {
    if (S == 0) return SPG_OK;
    const dim3 grid((S + 255) / 256), block(256);
    cudaStream_t s = (cudaStream_t)stream;
    switch (words) {
        case 1: k_survivor_bins<1><<<grid, block, 0, s>>>(prm, geno, surv, S, n, survw); break;
        case 2: k_survivor_bins<2><<<grid, block, 0, s>>>(prm, geno, surv, S, n, survw); break;
        case 4: k_survivor_bins<4><<<grid, block, 0, s>>>(prm, geno, surv, S, n, survw); break;
        case 8: k_survivor_bins<8><<<grid, block, 0, s>>>(prm, geno, surv, S, n, survw); break;
        default: return SPG_ERR_INVALID;
    }
    return cudaGetLastError() == cudaSuccess ? SPG_OK : SPG_ERR_CUDA;
}

int launch_set_state(DevState *st, StatAcc *acc, uint32_t gen, uint32_t S, uint32_t f, double R, int32_t status,
                     uint32_t target, void *stream) {
    k_set_state<<<1, 32, 0, (cudaStream_t)stream>>>(st, acc, gen, S, f, R, status, target);
    return cudaGetLastError() == cudaSuccess ? SPG_OK : SPG_ERR_CUDA;
}

}  // namespace spg
