// Spatial, age-structured multi-species community (spg_space_*): species on
// an X x Y torus of patches, individuals of age class 0/1/2, births from the
// adults of a deme, per-age survival scaled by an interaction factor from
// all species' counts in the patch, dispersal to the four neighbours
// (the migration among patches of the paper's Main text and S3, Fig. 1 A-F
// per deme, Fig. S5 B flattening over demes).
//
// Layout: all demes d = s*P + p concatenated; a deme stores adults first
// (age 2, then 1, then 0).  One step is eight launches, none of which waits
// on another block:
//   k_sp_plan      one thread per deme: interaction factor f, births B;
//   k_sp_scan      (x2) one block: exclusive scans of births (offsets of
//                  each deme's newborns in the step's newborn arrays) and of
//                  the new deme sizes;
//   k_sp_classify  one block per deme: survival, ageing and direction of
//                  every member, direction of every newborn, and each
//                  item's stable rank within its (age class, direction)
//                  class by block scans of per-class counts;
//   k_sp_totals    one thread per destination deme: offsets of the five
//                  source slots (stay, from N, S, E, W) per age class;
//   k_sp_births    grid-stride over all newborns: records formed and
//                  written with age and phenotype to their final positions;
//   k_sp_scatter   one block per deme: surviving members' records, ages and
//                  phenotypes to their final positions;
//   k_sp_finish    one thread: statistics record, step counter.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "spegg.h"
#include "spegg_engine.h"
#include "spegg_internal.h"

namespace spg {
namespace {

constexpr int kSpBlock = 256;
constexpr int kSpClassBlock = 128;  // threads of the per-deme classify blocks
constexpr uint32_t kMaxSpecies = 4;
enum SpPurpose : uint32_t { kSpFounder = 1, kSpMate = 2, kSpRecomb = 3, kSpMutPos = 4, kSpSurv = 5, kSpDisp = 6 };
constexpr uint32_t kDead = 15u;

struct alignas(16) SpeciesParams {
    uint32_t table[3][kBins];
    uint32_t planes[kMaxPlanes * kMaxWords];
    uint32_t cdf[kMaxKmax];
    int32_t e_min;
    uint32_t nplanes, kmax;
    int32_t bias;
    uint32_t shift;
    uint32_t D, A[kMaxSpecies], G, P[kMaxSpecies], E, C[kMaxSpecies], beta_q16, bmax;
};

struct alignas(16) SpAcc {
    unsigned long long n_before, adults_before, births, survivors, movers, n_after, adults_after;
    long long sum_raw_surv;
    unsigned long long het_newborn, allele_newborn;
};

struct alignas(16) SpState {
    uint32_t t;        // steps completed
    int32_t status;    // SPG_OK or an error
    uint32_t total;    // individuals in the current layout
    uint32_t births;   // newborns of the step in progress
};

struct SpaceArgs {
    const SpeciesParams *sp;
    uint32_t X, Y, P, ns, nd;
    uint32_t key0, key1, disp_q32;
    uint32_t cap, staging_cap, ring_cap;
    uint32_t *geno[2];   // [cap][2W] by step parity
    uint8_t *age[2];     // [cap]
    int32_t *raw[2];     // [cap] additive phenotype of each record, set at birth
    uint32_t *off[2];    // [nd + 1]
    uint32_t *adults[2]; // [nd]
    uint32_t *f, *births, *nb_off;   // [nd], [nd], [nd + 1]
    uint32_t *nb_deme;               // [staging_cap] demes of the step's newborns
    uint8_t *cls, *nb_cls;           // [cap], [staging_cap]
    uint32_t *rank, *nb_rank;        // [cap], [staging_cap]
    uint32_t *cnt;                   // [nd][15] per source deme and (age class, direction)
    uint32_t *slotoff;               // [nd][15] per destination deme and (age class, slot)
    uint32_t *nnew;                  // [nd]
    SpState *state;
    SpAcc *acc;                      // [ns]
    spg_space_stats *ring;           // [ring_cap][ns]
};

// ---------------------------------------------------------------- Philox
// Philox4x32-10 from its published definition (Salmon et al., SC'11).
__device__ __forceinline__ uint4 sp_philox(uint4 c, uint32_t k0, uint32_t k1) {
    constexpr uint32_t A = 0xD2511F53u, B = 0xCD9E8D57u, WA = 0x9E3779B9u, WB = 0xBB67AE85u;
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
__device__ __forceinline__ uint32_t sp_lane(const uint4 &d, int l) {
    return l == 0 ? d.x : l == 1 ? d.y : l == 2 ? d.z : d.w;
}

__device__ __forceinline__ uint32_t sp_dest(const SpaceArgs &a, uint32_t p, uint32_t dir) {
    uint32_t x = p % a.X, y = p / a.X;
    if (dir == 1) y = (y + a.Y - 1) % a.Y;
    else if (dir == 2) y = (y + 1) % a.Y;
    else if (dir == 3) x = (x + 1) % a.X;
    else if (dir == 4) x = (x + a.X - 1) % a.X;
    return y * a.X + x;
}
// slot of a move in the destination's order (stay, from N, from S, from E, from W)
__device__ __forceinline__ uint32_t sp_slot(uint32_t dir) { return dir == 0 ? 0u : dir == 1 ? 2u : dir == 2 ? 1u : dir == 3 ? 4u : 3u; }
// source patch and direction of slot `slot` of destination patch q
__device__ __forceinline__ void sp_slot_source(const SpaceArgs &a, uint32_t q, uint32_t slot, uint32_t &src,
                                               uint32_t &dir) {
    // from N means the mover went S (dir 2) out of north(q), etc.
    const uint32_t back[5] = {0, 1, 2, 3, 4};      // the neighbour of q on that side
    const uint32_t moved[5] = {0, 2, 1, 4, 3};     // the direction the mover took
    src = sp_dest(a, q, back[slot]);
    dir = moved[slot];
}

// One record (2W words; 8W bytes, 16-byte aligned for W >= 2) in vector accesses.
template <int W>
__device__ __forceinline__ void sp_load_rec(const uint32_t *p, uint32_t (&r)[2 * W]) {
    if constexpr (W == 1) {
        const uint2 v = *reinterpret_cast<const uint2 *>(p);
        r[0] = v.x;
        r[1] = v.y;
    } else {
#pragma unroll
        for (int q = 0; q < W / 2; ++q) {
            const uint4 v = reinterpret_cast<const uint4 *>(p)[q];
            r[4 * q] = v.x;
            r[4 * q + 1] = v.y;
            r[4 * q + 2] = v.z;
            r[4 * q + 3] = v.w;
        }
    }
}
template <int W>
__device__ __forceinline__ void sp_store_rec(uint32_t *p, const uint32_t (&r)[2 * W]) {
    if constexpr (W == 1) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(r[0], r[1]);
    } else {
#pragma unroll
        for (int q = 0; q < W / 2; ++q)
            reinterpret_cast<uint4 *>(p)[q] = make_uint4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
    }
}

// Effect planes of one species staged in shared memory (plane b, word w at
// [b * W + w]) by the whole block.
template <int W>
__device__ __forceinline__ void sp_stage_planes(const SpeciesParams *sp, uint32_t *s_planes) {
    for (uint32_t i = threadIdx.x; i < kMaxPlanes * W; i += blockDim.x) s_planes[i] = sp->planes[i];
}

template <int W>
__device__ __forceinline__ int32_t sp_phenotype(const uint32_t (&c)[2 * W], const SpeciesParams *sp,
                                                const uint32_t *s_planes) {
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) total += __popc(c[w]) + __popc(c[W + w]);
    int32_t raw = sp->e_min * (int32_t)total;
    for (uint32_t b = 0; b < sp->nplanes; ++b) {
        int32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t pl = s_planes[b * W + w];
            cnt += __popc(pl & c[w]) + __popc(pl & c[W + w]);
        }
        raw += cnt << b;
    }
    return raw;
}

__device__ __forceinline__ uint32_t sp_bin(const SpeciesParams *sp, int32_t raw) {
    const long long v = (long long)raw + (long long)sp->bias;
    return v < 0 ? 0u : (uint32_t)min(v >> sp->shift, (long long)(kBins - 1));
}

// ------------------------------------------------------------- founders
template <int W>
__global__ void k_sp_founders(SpaceArgs a, const uint32_t *n0, const uint32_t *p0) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t total = a.off[0][a.nd];
    if (i >= total) return;
    // deme of item i: founders are n0[s] per patch
    uint32_t s = 0, base = 0;
    while (s + 1 < a.ns && i >= base + n0[s] * a.P) base += n0[s++] * a.P;
    const uint32_t within = i - base, p = within / n0[s], r = within % n0[s], d = s * a.P + p;
    uint32_t rec[2 * W];
#pragma unroll
    for (int hw = 0; hw < 2 * W; ++hw) {
        uint32_t word = 0;
        for (int c = 0; c < 8; ++c) {
            const uint4 u = sp_philox(make_uint4(r, 0u, d, (kSpFounder << 24) | (uint32_t)(hw * 8 + c)), a.key0, a.key1);
            word |= (uint32_t)(u.x < p0[s]) << (4 * c + 0);
            word |= (uint32_t)(u.y < p0[s]) << (4 * c + 1);
            word |= (uint32_t)(u.z < p0[s]) << (4 * c + 2);
            word |= (uint32_t)(u.w < p0[s]) << (4 * c + 3);
        }
        rec[hw] = word;
    }
#pragma unroll
    for (int hw = 0; hw < 2 * W; ++hw) a.geno[0][(size_t)i * 2 * W + hw] = rec[hw];
    a.raw[0][i] = sp_phenotype<W>(rec, a.sp + s, a.sp[s].planes);
    const uint32_t half = n0[s] / 2, quarter = n0[s] / 4;
    a.age[0][i] = r < half ? 2 : (r < half + quarter ? 1 : 0);
}

// ------------------------------------------------------------- planning
__global__ void k_sp_plan(SpaceArgs a) {
    const uint32_t par = a.state->t & 1u;
    const uint32_t d = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nb = 0, nad = 0, nbirth = 0;
    uint32_t s = 0;
    if (d < a.nd && a.state->status == SPG_OK) {
        s = d / a.P;
        const uint32_t p = d % a.P;
        const SpeciesParams *sp = a.sp + s;
        const uint32_t *off = a.off[par];
        unsigned long long pressure = 0, benefit = sp->G, cost = sp->E;
        for (uint32_t k = 0; k < a.ns; ++k) {
            const uint32_t dk = k * a.P + p;
            const unsigned long long nk = off[dk + 1] - off[dk];
            pressure += (unsigned long long)sp->A[k] * nk;
            benefit += (unsigned long long)sp->P[k] * nk;
            cost += (unsigned long long)sp->C[k] * nk;
        }
        uint32_t f = kCertain;
        if (pressure) {
            const unsigned __int128 q =
                ((unsigned __int128)sp->D << 32) / (unsigned __int128)((unsigned long long)sp->D + pressure);
            f = q > 0xFFFFFFFEull ? 0xFFFFFFFEu : (uint32_t)q;
        }
        const unsigned long long den = benefit + cost;
        unsigned long long g = 0;
        if (den) g = (unsigned long long)(((unsigned __int128)benefit << 32) / (unsigned __int128)den);
        const uint32_t m = a.adults[par][d];
        const unsigned __int128 prod = (unsigned __int128)((unsigned long long)m * sp->beta_q16) * g;
        const unsigned long long b = (unsigned long long)(prod >> 48);
        const uint32_t B = b > sp->bmax ? sp->bmax : (uint32_t)b;
        a.f[d] = f;
        a.births[d] = B;
        nb = off[d + 1] - off[d];
        nad = m;
        nbirth = B;
    }
    // per-species sums: demes of one block belong to at most two species
    for (uint32_t k = 0; k < a.ns; ++k) {
        const bool mine = d < a.nd && s == k;
        const unsigned long long v0 = __reduce_add_sync(0xFFFFFFFFu, mine ? (uint32_t)nb : 0u);
        const unsigned long long v1 = __reduce_add_sync(0xFFFFFFFFu, mine ? (uint32_t)nad : 0u);
        const unsigned long long v2 = __reduce_add_sync(0xFFFFFFFFu, mine ? (uint32_t)nbirth : 0u);
        if ((threadIdx.x & 31) == 0 && (v0 | v2)) {
            atomicAdd(&a.acc[k].n_before, v0);
            atomicAdd(&a.acc[k].adults_before, v1);
            atomicAdd(&a.acc[k].births, v2);
        }
    }
}

// Exclusive scan of `in` (n values) into out[0..n] (out[n] = total) by one
// block; flags capacity overflow.  which = 0: births -> staging offsets,
// which = 1: new deme sizes -> offsets of the next layout.
__global__ void k_sp_scan(SpaceArgs a, int which) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    const uint32_t *in = which == 0 ? a.births : a.nnew;
    uint32_t *out = which == 0 ? a.nb_off : a.off[(a.state->t + 1u) & 1u];
    const uint32_t n = a.nd, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < n; base += blockDim.x) {
        const uint32_t i = base + tid;
        const uint32_t v = i < n ? in[i] : 0u;
        uint32_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if ((int)lane >= o) incl += y;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        uint32_t wbase = 0;
        for (uint32_t q = 0; q < warp; ++q) wbase += s_warp[q];
        const uint32_t carry = s_carry;
        if (i < n) out[i] = carry + wbase + incl - v;
        __syncthreads();
        if (tid == blockDim.x - 1) s_carry = carry + wbase + incl;
        __syncthreads();
    }
    if (tid == 0) {
        out[n] = s_carry;
        if (which == 0) {
            a.state->births = s_carry;
            if (s_carry > a.staging_cap) a.state->status = SPG_ERR_RANGE;
        } else if (s_carry > a.cap) {
            a.state->status = SPG_ERR_RANGE;
        }
    }
}

// Stable ranks of one pass of items, thread t holding items IPT t ..
// IPT t + IPT - 1 of the pass: rank = items of the same class in earlier
// passes (s_carry) + in earlier threads of this pass + earlier items of this
// thread.  The thread's own counts sit in 3-bit fields of one word; the scans
// over threads use 16-bit fields, two classes per word (classes 2Q0 ..
// 2Q1-1; a pass holds at most kSpBlock * IPT <= 65535 items); kDead is not
// counted.
template <int IPT, int Q0, int Q1>
__device__ __forceinline__ void class_ranks(const uint32_t (&cls)[IPT], uint32_t (&rk)[IPT], uint32_t *s_carry,
                                            uint32_t (*s_wt)[8]) {
    constexpr int NQ = Q1 - Q0, NW = kSpClassBlock / 32;
    constexpr uint32_t C0 = 2u * Q0;
    static_assert(kSpClassBlock * IPT <= 65535 && Q1 <= 8 && IPT <= 7 && NQ <= 5, "field widths");
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t mine = 0, before[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const uint32_t c = cls[i], sh = 3u * (c - C0);
        const bool counted = c < kDead && c - C0 < 2u * NQ;
        before[i] = counted ? (mine >> sh) & 7u : 0u;
        if (counted) mine += 1u << sh;
    }
    uint32_t own[NQ], x[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        own[q] = ((mine >> (6 * q)) & 7u) | (((mine >> (6 * q + 3)) & 7u) << 16);
        x[q] = own[q];
    }
#pragma unroll
    for (int step = 0; step < 5; ++step) {
        const int o = 1 << step;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x[q], o);
            if ((int)lane >= o) x[q] += y;
        }
    }
    if (lane == 31u)
#pragma unroll
        for (int q = 0; q < NQ; ++q) s_wt[warp][q] = x[q];
    __syncthreads();
    // earlier warps' totals: lane q of each warp sums word q, then shares it
    uint32_t wp = 0;
    if (lane < (uint32_t)NQ)
        for (uint32_t v = 0; v < warp; ++v) wp += s_wt[v][lane];
#pragma unroll
    for (int q = 0; q < NQ; ++q) x[q] += __shfl_sync(0xFFFFFFFFu, wp, q) - own[q];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const uint32_t c = cls[i];
        rk[i] = 0;
        if (c < kDead && c - C0 < 2u * NQ) {
            uint32_t sel = x[0];
#pragma unroll
            for (int q = 1; q < NQ; ++q)
                if ((c >> 1) == (uint32_t)(Q0 + q)) sel = x[q];
            rk[i] = s_carry[c] + ((sel >> ((c & 1u) * 16u)) & 0xFFFFu) + before[i];
        }
    }
    __syncthreads();  // s_carry and s_wt read by every thread
    if (threadIdx.x < 2u * NQ) {
        const uint32_t c = C0 + threadIdx.x, q = threadIdx.x >> 1;
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) tot += (s_wt[w][q] >> ((c & 1u) * 16u)) & 0xFFFFu;
        s_carry[c] += tot;
    }
    __syncthreads();
}

// ----------------------------------------------- survival and births (A-E)
// One block per deme: survival, ageing and direction of every member, the
// direction of every newborn (its mate and dispersal draws), and each item's
// stable rank within its (age class, direction) class.  Members (classes
// 0-9) go kSpIPT consecutive ones per thread, so all their loads are in
// flight together; newborns (classes 10-14) kSpNbIPT per thread.  A block
// of kSpClassBlock threads ranks a typical deme (~800 members, ~150
// newborns) in one pass each, so the fixed cost of the two class scans is
// spread over all of its items.  The newborns' records are formed by
// k_sp_births.
constexpr int kSpIPT = 7;
constexpr int kSpNbIPT = 2;  // newborns per thread

__global__ void __launch_bounds__(kSpClassBlock) k_sp_classify(SpaceArgs a) {
    __shared__ uint32_t s_carry[16];
    __shared__ uint32_t s_wt[kSpClassBlock / 32][8];
    if (a.state->status != SPG_OK) return;
    const uint32_t d = blockIdx.x, s = d / a.P, tid = threadIdx.x;
    const uint32_t t = a.state->t + 1u, par = a.state->t & 1u;
    const SpeciesParams *sp = a.sp + s;
    const uint8_t *age = a.age[par];
    const int32_t *rawp = a.raw[par];
    const uint32_t base = a.off[par][d], n = a.off[par][d + 1] - base;
    const uint32_t f = a.f[d], B = a.births[d], nb0 = a.nb_off[d];
    if (tid < 16) s_carry[tid] = 0;
    __syncthreads();
    long long sum_raw = 0;
    uint32_t surv = 0, moved = 0;
    // pre-existing members, in rank order
    for (uint32_t p0 = 0; p0 < n; p0 += kSpClassBlock * kSpIPT) {
        const uint32_t r0 = p0 + tid * kSpIPT;
        uint32_t ag[kSpIPT], cls[kSpIPT], rk[kSpIPT];
        int32_t raw[kSpIPT];
        // a genotype is fixed for life, so its phenotype was computed once at birth
#pragma unroll
        for (int i = 0; i < kSpIPT; ++i) {
            ag[i] = r0 + i < n ? age[base + r0 + i] : 0u;
            raw[i] = r0 + i < n ? rawp[base + r0 + i] : 0;
        }
#pragma unroll
        for (int i = 0; i < kSpIPT; ++i) {
            const uint32_t r = r0 + (uint32_t)i;
            cls[i] = kDead;
            if (r < n) {
                const uint4 u = sp_philox(make_uint4(r, t, d, kSpSurv << 24), a.key0, a.key1);
                uint32_t thr = __ldg(&sp->table[ag[i]][sp_bin(sp, raw[i])]);
                if (f != kCertain) thr = __umulhi(thr, f);
                if (thr == kCertain || u.x < thr) {
                    const uint32_t na = ag[i] + 1 > 2 ? 2u : ag[i] + 1;
                    const uint32_t dir = u.y < a.disp_q32 ? 1u + __umulhi(u.z, 4u) : 0u;
                    cls[i] = (2u - na) * 5u + dir;
                    ++surv;
                    sum_raw += raw[i];
                    moved += dir != 0;
                }
            }
        }
        class_ranks<kSpIPT, 0, 5>(cls, rk, s_carry, s_wt);
#pragma unroll
        for (int i = 0; i < kSpIPT; ++i)
            if (r0 + i < n) {
                a.cls[base + r0 + i] = (uint8_t)cls[i];
                a.rank[base + r0 + i] = rk[i];
            }
    }
    // newborns, in birth order: dispersal from the mate draw's third lane,
    // direction from the dispersal draw
    for (uint32_t c0 = 0; c0 < B; c0 += kSpClassBlock * kSpNbIPT) {
        uint32_t cls[kSpNbIPT], rk[kSpNbIPT];
#pragma unroll
        for (int i = 0; i < kSpNbIPT; ++i) {
            const uint32_t k = c0 + tid * kSpNbIPT + (uint32_t)i;
            cls[i] = kDead;
            if (k < B && nb0 + k < a.staging_cap) {
                const uint4 u = sp_philox(make_uint4(k, t, d, kSpMate << 24), a.key0, a.key1);
                uint32_t dir = 0;
                if (u.z < a.disp_q32)
                    dir = 1u + __umulhi(sp_philox(make_uint4(k, t, d, kSpDisp << 24), a.key0, a.key1).x, 4u);
                cls[i] = 2u * 5u + dir;
                moved += dir != 0;
            }
        }
        class_ranks<kSpNbIPT, 5, 8>(cls, rk, s_carry, s_wt);
#pragma unroll
        for (int i = 0; i < kSpNbIPT; ++i) {
            const uint32_t k = c0 + tid * kSpNbIPT + (uint32_t)i;
            if (k < B && nb0 + k < a.staging_cap) {
                a.nb_cls[nb0 + k] = (uint8_t)cls[i];
                a.nb_rank[nb0 + k] = rk[i];
                a.nb_deme[nb0 + k] = d;
            }
        }
    }
    if (tid < 15) a.cnt[(size_t)d * 15 + tid] = s_carry[tid];
    // statistics
    const uint32_t w_s = __reduce_add_sync(0xFFFFFFFFu, surv), w_m = __reduce_add_sync(0xFFFFFFFFu, moved);
    long long w_raw = sum_raw;
    for (int o = 16; o > 0; o >>= 1) w_raw += __shfl_xor_sync(0xFFFFFFFFu, w_raw, o);
    if ((tid & 31) == 0) {
        SpAcc *ac = a.acc + s;
        if (w_s) atomicAdd(&ac->survivors, (unsigned long long)w_s);
        if (w_m) atomicAdd(&ac->movers, (unsigned long long)w_m);
        if (w_raw) atomicAdd(reinterpret_cast<unsigned long long *>(&ac->sum_raw_surv), (unsigned long long)w_raw);
    }
}

// Newborn records (A-C), one thread per newborn over all demes: parents
// among the deme's m adults, free recombination, mutation, written with
// their age and phenotype straight to their places in the new layout (after
// k_sp_totals and the second scan); heterozygosity and allele counts per
// species.
template <int W>
__global__ void __launch_bounds__(kSpBlock) k_sp_births(SpaceArgs a) {
    __shared__ __align__(16) uint32_t s_planes[kMaxSpecies][kMaxPlanes * W];
    if (a.state->status != SPG_OK) return;
    const uint32_t tid = threadIdx.x;
    const uint32_t t = a.state->t + 1u, par = a.state->t & 1u;
    const uint32_t total = min(a.state->births, a.staging_cap);
    for (uint32_t k = 0; k < a.ns; ++k) sp_stage_planes<W>(a.sp + k, s_planes[k]);
    __syncthreads();
    uint32_t het_s[kMaxSpecies] = {0u, 0u, 0u, 0u}, allele_s[kMaxSpecies] = {0u, 0u, 0u, 0u};
    const uint32_t *geno = a.geno[par];
    uint32_t *ngeno = a.geno[par ^ 1u];
    const uint32_t *noff = a.off[par ^ 1u];
    for (uint32_t i = blockIdx.x * kSpBlock + tid; i < total; i += gridDim.x * kSpBlock) {
        const uint32_t d = a.nb_deme[i], s = d / a.P, k = i - a.nb_off[d];
        const uint32_t dir = a.nb_cls[i] % 5u, rk = a.nb_rank[i];  // class 10 + dir: age 0
        const SpeciesParams *sp = a.sp + s;
        const uint32_t base = a.off[par][d], m = a.adults[par][d];
        const uint4 u = sp_philox(make_uint4(k, t, d, kSpMate << 24), a.key0, a.key1);
        uint32_t mo[2 * W], fa[2 * W], ch[2 * W];
        sp_load_rec<W>(geno + (size_t)(base + __umulhi(u.x, m)) * 2 * W, mo);
        sp_load_rec<W>(geno + (size_t)(base + __umulhi(u.y, m)) * 2 * W, fa);
#pragma unroll
        for (int q4 = 0; q4 < (2 * W + 3) / 4; ++q4) {
            const uint4 dm = sp_philox(make_uint4(k, t, d, (kSpRecomb << 24) | (uint32_t)q4), a.key0, a.key1);
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int q = 4 * q4 + l;
                if (q < 2 * W) {
                    const int w = q >> 1;
                    const uint32_t mk = sp_lane(dm, l);
                    if ((q & 1) == 0) ch[w] = (mo[w] & ~mk) | (mo[W + w] & mk);
                    else ch[W + w] = (fa[w] & ~mk) | (fa[W + w] & mk);
                }
            }
        }
        uint32_t kmut = 0;  // none below the CDF's first entry (the common case)
        if (sp->kmax != 0u && u.w >= __ldg(&sp->cdf[0]))
            for (uint32_t q = 0; q < sp->kmax; ++q) kmut += u.w >= __ldg(&sp->cdf[q]) ? 1u : 0u;
        if (kmut) {
            uint32_t seen[2 * W];
#pragma unroll
            for (int w = 0; w < 2 * W; ++w) seen[w] = 0;
            uint32_t chosen = 0;
            for (uint32_t a4 = 0; a4 < kMutDraws / 4 && chosen < kmut; ++a4) {
                const uint4 dp = sp_philox(make_uint4(k, t, d, (kSpMutPos << 24) | a4), a.key0, a.key1);
                for (int l = 0; l < 4; ++l) {
                    if (chosen >= kmut) break;
                    const uint32_t pos = __umulhi(sp_lane(dp, l), 64u * W);
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
                                ch[w] ^= bit;
                            }
                        ++chosen;
                    }
                }
            }
        }
        const uint32_t q = s * a.P + sp_dest(a, d % a.P, dir);
        const uint32_t pos = noff[q] + a.slotoff[(size_t)q * 15 + 2u * 5u + sp_slot(dir)] + rk;
        if (pos < a.cap) {
            sp_store_rec<W>(ngeno + (size_t)pos * 2 * W, ch);
            a.age[par ^ 1u][pos] = 0;
            a.raw[par ^ 1u][pos] = sp_phenotype<W>(ch, sp, s_planes[s]);
        }
        uint32_t het = 0, allele = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            het += __popc(ch[w] ^ ch[W + w]);
            allele += __popc(ch[w]) + __popc(ch[W + w]);
        }
#pragma unroll
        for (uint32_t q = 0; q < kMaxSpecies; ++q)
            if (q == s) {
                het_s[q] += het;
                allele_s[q] += allele;
            }
    }
    // a thread's sums stay below 2^32: at most 2L <= 512 per newborn, and a
    // thread forms at most staging_cap / (resident threads) < 2^23 newborns
#pragma unroll
    for (uint32_t q = 0; q < kMaxSpecies; ++q) {
        const uint32_t h = __reduce_add_sync(0xFFFFFFFFu, het_s[q]), al = __reduce_add_sync(0xFFFFFFFFu, allele_s[q]);
        if ((tid & 31) == 0 && (h | al)) {
            atomicAdd(&a.acc[q].het_newborn, (unsigned long long)h);
            atomicAdd(&a.acc[q].allele_newborn, (unsigned long long)al);
        }
    }
}

// ------------------------------------------------ destination offsets
__global__ void k_sp_totals(SpaceArgs a) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t total = 0, adults = 0, s = 0;
    const bool ok = q < a.nd && a.state->status == SPG_OK;
    if (ok) {
        s = q / a.P;
        const uint32_t pq = q % a.P;
        for (uint32_t ci = 0; ci < 3; ++ci) {
            for (uint32_t slot = 0; slot < 5; ++slot) {
                uint32_t src, dir;
                sp_slot_source(a, pq, slot, src, dir);
                const uint32_t c = a.cnt[(size_t)(s * a.P + src) * 15 + ci * 5 + dir];
                a.slotoff[(size_t)q * 15 + ci * 5 + slot] = total;
                total += c;
                if (ci == 0) adults += c;
            }
        }
        a.nnew[q] = total;
        a.adults[(a.state->t + 1u) & 1u][q] = adults;
    } else if (q < a.nd) {
        a.nnew[q] = 0;
    }
    for (uint32_t k = 0; k < a.ns; ++k) {
        const bool mine = ok && s == k;
        const uint32_t v0 = __reduce_add_sync(0xFFFFFFFFu, mine ? total : 0u);
        const uint32_t v1 = __reduce_add_sync(0xFFFFFFFFu, mine ? adults : 0u);
        if ((threadIdx.x & 31) == 0 && v0) {
            atomicAdd(&a.acc[k].n_after, (unsigned long long)v0);
            atomicAdd(&a.acc[k].adults_after, (unsigned long long)v1);
        }
    }
}

// ------------------------------------------------------ new layout
template <int W>
__global__ void __launch_bounds__(kSpBlock) k_sp_scatter(SpaceArgs a) {
    if (a.state->status != SPG_OK) return;
    const uint32_t d = blockIdx.x, s = d / a.P, p = d % a.P, tid = threadIdx.x;
    const uint32_t par = a.state->t & 1u, npar = par ^ 1u;
    const uint32_t *geno = a.geno[par];
    uint32_t *ngeno = a.geno[npar];
    uint8_t *nage = a.age[npar];
    int32_t *nraw = a.raw[npar];
    const uint32_t *noff = a.off[npar];
    const uint32_t base = a.off[par][d], n = a.off[par][d + 1] - base;
    for (uint32_t i = tid; i < n; i += kSpBlock) {
        const uint32_t cls = a.cls[base + i], rk = a.rank[base + i];
        const uint32_t *src = geno + (size_t)(base + i) * 2 * W;
        const int32_t *src_raw = a.raw[par] + base + i;
        if (cls >= kDead) continue;
        const uint32_t ci = cls / 5u, dir = cls % 5u;
        const uint32_t q = s * a.P + sp_dest(a, p, dir);
        const uint32_t pos = noff[q] + a.slotoff[(size_t)q * 15 + ci * 5 + sp_slot(dir)] + rk;
        if (pos >= a.cap) continue;
        uint32_t rec[2 * W];
        sp_load_rec<W>(src, rec);
        sp_store_rec<W>(ngeno + (size_t)pos * 2 * W, rec);
        nage[pos] = (uint8_t)(2u - ci);
        nraw[pos] = *src_raw;
    }
}

// ---------------------------------------------------------- step end
__global__ void k_sp_finish(SpaceArgs a) {
    const uint32_t k = threadIdx.x;
    SpState *st = a.state;
    const uint32_t t = st->t + 1u;
    if (k < a.ns) {
        SpAcc *ac = a.acc + k;
        spg_space_stats *rec = a.ring + (size_t)((t - 1u) % a.ring_cap) * a.ns + k;
        rec->t = t;
        rec->species = k;
        rec->n_before = (uint32_t)ac->n_before;
        rec->adults_before = (uint32_t)ac->adults_before;
        rec->births = (uint32_t)ac->births;
        rec->survivors = (uint32_t)ac->survivors;
        rec->movers = (uint32_t)ac->movers;
        rec->n_after = (uint32_t)ac->n_after;
        rec->adults_after = (uint32_t)ac->adults_after;
        rec->pad = 0;
        rec->sum_raw_surv = ac->sum_raw_surv;
        rec->het_newborn = ac->het_newborn;
        rec->allele_newborn = ac->allele_newborn;
        memset(ac, 0, sizeof(SpAcc));
    }
    __syncthreads();
    if (k == 0 && st->status == SPG_OK) {
        st->total = a.off[t & 1u][a.nd];
        st->t = t;
    }
}

__global__ void k_sp_clear(SpaceArgs a) {
    if (threadIdx.x < a.ns) memset(a.acc + threadIdx.x, 0, sizeof(SpAcc));
}

}  // namespace
}  // namespace spg

using namespace spg;

struct spg_space {
    uint32_t X = 0, Y = 0, P = 0, ns = 0, L = 0, W = 0, nd = 0, cap = 0, staging_cap = 0, ring_cap = 0;
    uint32_t births_grid = 0;  // resident blocks of k_sp_births
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;                     // the newborns' kernel, beside the survivors' move
    cudaEvent_t fork = nullptr, join = nullptr;     // side stream after the step's scans / stream after the newborns
    cudaGraphExec_t chunk = nullptr;                // kSpGraphSteps steps, captured on first use
    bool own_stream = false;
    Allocator alloc;
    char *arena = nullptr;
    SpaceArgs args{};
    std::vector<spg_space_stats> host_ring;
};

namespace {

int space_sync(spg_space *c) {
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? SPG_OK : cuda_fail(e, "cudaStreamSynchronize");
}

int space_state(spg_space *c, SpState &st) {
    int rc = space_sync(c);
    if (rc != SPG_OK) return rc;
    const cudaError_t e = cudaMemcpy(&st, c->args.state, sizeof st, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SPG_OK : cuda_fail(e, "read state");
}

// Resident blocks of k_sp_births on this device (a grid-stride kernel).
template <int W>
int births_grid_for(uint32_t &grid) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sp_births<W>, kSpBlock, 0);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "newborn kernel occupancy");
    grid = (uint32_t)std::max(per_sm, 1) * (uint32_t)std::max(sms, 1);
    return SPG_OK;
}

template <int W>
int launch_step(spg_space *c) {
    const SpaceArgs &a = c->args;
    cudaStream_t s = c->stream;
    const uint32_t g = (a.nd + 255) / 256;
    k_sp_plan<<<g, 256, 0, s>>>(a);
    k_sp_scan<<<1, 1024, 0, s>>>(a, 0);
    k_sp_classify<<<a.nd, kSpClassBlock, 0, s>>>(a);
    k_sp_totals<<<g, 256, 0, s>>>(a);
    k_sp_scan<<<1, 1024, 0, s>>>(a, 1);
    // the newborns on the side stream beside the survivors' move: both only
    // read the current generation and write disjoint places of the next; the
    // newborns' kernel goes first so that its resident grid is placed before
    // the move's blocks take the rest of each SM
    cudaError_t e = cudaEventRecord(c->fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->fork, 0);
    if (e != cudaSuccess) return cuda_fail(e, "space step fork");
    k_sp_births<W><<<c->births_grid, kSpBlock, 0, c->side>>>(a);
    e = cudaEventRecord(c->join, c->side);
    if (e != cudaSuccess) return cuda_fail(e, "space step join");
    k_sp_scatter<W><<<a.nd, kSpBlock, 0, s>>>(a);
    e = cudaStreamWaitEvent(s, c->join, 0);
    if (e != cudaSuccess) return cuda_fail(e, "space step join");
    k_sp_finish<<<1, 32, 0, s>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? SPG_OK : cuda_fail(e, "space step launch");
}

// Steps in a cached graph: every step's kernels take their parameters from
// the (fixed) SpaceArgs and their per-step state from device memory, so one
// captured chunk replays any kSpGraphSteps consecutive steps.
constexpr uint32_t kSpGraphSteps = 32;

int launch_steps(spg_space *c, uint32_t n) {
    for (uint32_t i = 0; i < n; ++i) {
        int rc;
        switch (c->W) {
            case 1: rc = launch_step<1>(c); break;
            case 2: rc = launch_step<2>(c); break;
            case 4: rc = launch_step<4>(c); break;
            default: rc = launch_step<8>(c); break;
        }
        if (rc != SPG_OK) return rc;
    }
    return SPG_OK;
}

// One chunk of kSpGraphSteps steps through the cached graph (captured from
// the step launches on first use).  A stream that is being captured already
// (the caller building a graph of its own) gets the launches themselves.
int launch_chunk(spg_space *c) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(c->stream, &cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    if (cs != cudaStreamCaptureStatusNone) return launch_steps(c, kSpGraphSteps);
    if (!c->chunk) {
        e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        const int rc = launch_steps(c, kSpGraphSteps);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(c->stream, &g);  // ends the capture whatever the launches returned
        if (rc != SPG_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return rc != SPG_OK ? rc : cuda_fail(e, "cudaStreamEndCapture");
        }
        e = cudaGraphInstantiate(&c->chunk, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->chunk = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
    }
    e = cudaGraphLaunch(c->chunk, c->stream);
    return e == cudaSuccess ? SPG_OK : cuda_fail(e, "cudaGraphLaunch");
}

}  // namespace

extern "C" {

int spg_space_create(const spg_space_desc *desc, const spg_allocator *alloc, void *stream, spg_space **out) {
    if (!out) return fail(SPG_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!desc || !desc->species) return fail(SPG_ERR_INVALID, "description is NULL");
    if (desc->X == 0 || desc->Y == 0 || (uint64_t)desc->X * desc->Y > (1u << 20))
        return fail(SPG_ERR_INVALID, "X and Y must be >= 1 with X*Y <= 2^20");
    if (desc->n_species == 0 || desc->n_species > kMaxSpecies)
        return fail(SPG_ERR_INVALID, "n_species must be 1..%u", kMaxSpecies);
    if (!(desc->n_loci == 32 || desc->n_loci == 64 || desc->n_loci == 128 || desc->n_loci == 256))
        return fail(SPG_ERR_INVALID, "n_loci must be 32, 64, 128 or 256");
    std::unique_ptr<spg_space> c(new (std::nothrow) spg_space());
    if (!c) return fail(SPG_ERR_OOM, "host allocation failed");
    c->X = desc->X;
    c->Y = desc->Y;
    c->P = desc->X * desc->Y;
    c->ns = desc->n_species;
    c->L = desc->n_loci;
    c->W = desc->n_loci / 32;
    c->nd = c->ns * c->P;
    c->seed = desc->seed;
    uint64_t founders = 0;
    std::vector<SpeciesParams> prm(c->ns);
    std::vector<uint32_t> n0(c->ns), p0(c->ns);
    for (uint32_t s = 0; s < c->ns; ++s) {
        const spg_species &sd = desc->species[s];
        if (!sd.effects || !sd.tables) return fail(SPG_ERR_INVALID, "species %u: effects and tables are required", s);
        if (sd.bin_shift > 31 || !(sd.mu >= 0.0 && sd.mu < 1.0))
            return fail(SPG_ERR_INVALID, "species %u: bin_shift <= 31 and 0 <= mu < 1", s);
        SpeciesParams &q = prm[s];
        std::memset(&q, 0, sizeof q);
        std::memcpy(q.table, sd.tables, sizeof q.table);
        PopParams tmp;
        effect_planes(sd.effects, c->L, tmp);
        if (tmp.nplanes > (uint32_t)kMaxPlanes) return fail(SPG_ERR_INVALID, "species %u: effects span > 16 bits", s);
        std::memcpy(q.planes, tmp.planes, sizeof q.planes);
        q.e_min = tmp.e_min;
        q.nplanes = tmp.nplanes;
        q.kmax = mutation_cdf(sd.mu, 2 * c->L, q.cdf);
        q.bias = sd.bin_bias;
        q.shift = sd.bin_shift;
        q.D = sd.D;
        q.G = sd.G;
        q.E = sd.E;
        q.beta_q16 = sd.beta_q16;
        q.bmax = sd.bmax;
        for (uint32_t k = 0; k < kMaxSpecies; ++k) {
            q.A[k] = sd.A[k];
            q.P[k] = sd.P[k];
            q.C[k] = sd.C[k];
        }
        if (q.D == 0 && std::any_of(q.A, q.A + kMaxSpecies, [](uint32_t x) { return x != 0; }))
            return fail(SPG_ERR_INVALID, "species %u: D must be > 0 when interactions are set", s);
        n0[s] = sd.n0;
        p0[s] = sd.p0_q32;
        founders += (uint64_t)sd.n0 * c->P;
    }
    const uint64_t cap = desc->capacity ? desc->capacity : std::max<uint64_t>(2 * founders, 1024);
    if (cap > 0x7FFFFFFFull || founders > cap) return fail(SPG_ERR_INVALID, "capacity must hold the founders (< 2^31)");
    c->cap = (uint32_t)cap;
    c->staging_cap = desc->staging_capacity ? desc->staging_capacity : std::max<uint32_t>(c->cap / 2, 1024);
    c->ring_cap = desc->stats_capacity ? desc->stats_capacity : 1024;
    // arena
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    const size_t o_sp = take(sizeof(SpeciesParams) * c->ns);
    const size_t o_g0 = take((size_t)c->cap * 2 * c->W * 4), o_g1 = take((size_t)c->cap * 2 * c->W * 4);
    const size_t o_a0 = take(c->cap), o_a1 = take(c->cap);
    const size_t o_r0 = take((size_t)c->cap * 4), o_r1 = take((size_t)c->cap * 4);
    const size_t o_nd = take((size_t)c->staging_cap * 4);
    const size_t o_off0 = take((size_t)(c->nd + 1) * 4), o_off1 = take((size_t)(c->nd + 1) * 4);
    const size_t o_ad0 = take((size_t)c->nd * 4), o_ad1 = take((size_t)c->nd * 4);
    const size_t o_f = take((size_t)c->nd * 4), o_b = take((size_t)c->nd * 4), o_nbo = take((size_t)(c->nd + 1) * 4);
    const size_t o_cls = take(c->cap), o_ncls = take(c->staging_cap);
    const size_t o_rk = take((size_t)c->cap * 4), o_nrk = take((size_t)c->staging_cap * 4);
    const size_t o_cnt = take((size_t)c->nd * 15 * 4), o_so = take((size_t)c->nd * 15 * 4), o_nn = take((size_t)c->nd * 4);
    const size_t o_st = take(sizeof(SpState)), o_acc = take(sizeof(SpAcc) * c->ns);
    const size_t o_ring = take((size_t)c->ring_cap * c->ns * sizeof(spg_space_stats));
    const size_t o_n0 = take(4 * c->ns), o_p0 = take(4 * c->ns);
    if (alloc) c->alloc.hooks = *alloc;
    cudaError_t e = cudaSuccess;
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        c->own_stream = true;
    }
    e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        spg_space_destroy(c.release());
        return cuda_fail(e, "side stream");
    }
    c->arena = static_cast<char *>(c->alloc.alloc(off, c->stream));
    if (!c->arena) {
        spg_space_destroy(c.release());
        return fail(SPG_ERR_OOM, "device allocation of %zu bytes failed", off);
    }
    char *b = c->arena;
    SpaceArgs &a = c->args;
    a.sp = reinterpret_cast<const SpeciesParams *>(b + o_sp);
    a.X = c->X;
    a.Y = c->Y;
    a.P = c->P;
    a.ns = c->ns;
    a.nd = c->nd;
    a.key0 = (uint32_t)(c->seed & 0xFFFFFFFFu);
    a.key1 = (uint32_t)(c->seed >> 32);
    a.disp_q32 = desc->disp_q32;
    a.cap = c->cap;
    a.staging_cap = c->staging_cap;
    a.ring_cap = c->ring_cap;
    a.geno[0] = reinterpret_cast<uint32_t *>(b + o_g0);
    a.geno[1] = reinterpret_cast<uint32_t *>(b + o_g1);
    a.age[0] = reinterpret_cast<uint8_t *>(b + o_a0);
    a.age[1] = reinterpret_cast<uint8_t *>(b + o_a1);
    a.raw[0] = reinterpret_cast<int32_t *>(b + o_r0);
    a.raw[1] = reinterpret_cast<int32_t *>(b + o_r1);
    a.nb_deme = reinterpret_cast<uint32_t *>(b + o_nd);
    a.off[0] = reinterpret_cast<uint32_t *>(b + o_off0);
    a.off[1] = reinterpret_cast<uint32_t *>(b + o_off1);
    a.adults[0] = reinterpret_cast<uint32_t *>(b + o_ad0);
    a.adults[1] = reinterpret_cast<uint32_t *>(b + o_ad1);
    a.f = reinterpret_cast<uint32_t *>(b + o_f);
    a.births = reinterpret_cast<uint32_t *>(b + o_b);
    a.nb_off = reinterpret_cast<uint32_t *>(b + o_nbo);
    a.cls = reinterpret_cast<uint8_t *>(b + o_cls);
    a.nb_cls = reinterpret_cast<uint8_t *>(b + o_ncls);
    a.rank = reinterpret_cast<uint32_t *>(b + o_rk);
    a.nb_rank = reinterpret_cast<uint32_t *>(b + o_nrk);
    a.cnt = reinterpret_cast<uint32_t *>(b + o_cnt);
    a.slotoff = reinterpret_cast<uint32_t *>(b + o_so);
    a.nnew = reinterpret_cast<uint32_t *>(b + o_nn);
    a.state = reinterpret_cast<SpState *>(b + o_st);
    a.acc = reinterpret_cast<SpAcc *>(b + o_acc);
    a.ring = reinterpret_cast<spg_space_stats *>(b + o_ring);
    // founder layout: offsets and adult counts on the host
    std::vector<uint32_t> offs(c->nd + 1), adults(c->nd);
    uint32_t run = 0;
    for (uint32_t s = 0; s < c->ns; ++s)
        for (uint32_t p = 0; p < c->P; ++p) {
            offs[s * c->P + p] = run;
            adults[s * c->P + p] = n0[s] / 2;
            run += n0[s];
        }
    offs[c->nd] = run;
    SpState st0{0, SPG_OK, run, 0};
    e = cudaMemcpy(b + o_sp, prm.data(), sizeof(SpeciesParams) * c->ns, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(a.off[0], offs.data(), offs.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(a.adults[0], adults.data(), adults.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(a.state, &st0, sizeof st0, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_n0, n0.data(), 4 * c->ns, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_p0, p0.data(), 4 * c->ns, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(a.ring, 0, (size_t)c->ring_cap * c->ns * sizeof(spg_space_stats));
    if (e != cudaSuccess) {
        spg_space_destroy(c.release());
        return cuda_fail(e, "initialise community");
    }
    int rc0;
    switch (c->W) {
        case 1: rc0 = births_grid_for<1>(c->births_grid); break;
        case 2: rc0 = births_grid_for<2>(c->births_grid); break;
        case 4: rc0 = births_grid_for<4>(c->births_grid); break;
        default: rc0 = births_grid_for<8>(c->births_grid); break;
    }
    if (rc0 != SPG_OK) {
        spg_space_destroy(c.release());
        return rc0;
    }
    const uint32_t grid = (run + 127) / 128;
    const uint32_t *dn0 = reinterpret_cast<const uint32_t *>(b + o_n0), *dp0 = reinterpret_cast<const uint32_t *>(b + o_p0);
    if (run) {
        switch (c->W) {
            case 1: k_sp_founders<1><<<grid, 128, 0, c->stream>>>(a, dn0, dp0); break;
            case 2: k_sp_founders<2><<<grid, 128, 0, c->stream>>>(a, dn0, dp0); break;
            case 4: k_sp_founders<4><<<grid, 128, 0, c->stream>>>(a, dn0, dp0); break;
            default: k_sp_founders<8><<<grid, 128, 0, c->stream>>>(a, dn0, dp0); break;
        }
    }
    k_sp_clear<<<1, 32, 0, c->stream>>>(a);
    e = cudaGetLastError();
    int rc = e == cudaSuccess ? space_sync(c.get()) : cuda_fail(e, "founder launch");
    if (rc != SPG_OK) {
        spg_space_destroy(c.release());
        return rc;
    }
    *out = c.release();
    return SPG_OK;
}

int spg_space_step(spg_space *c, uint32_t n_steps) {
    if (!c) return fail(SPG_ERR_INVALID, "community is NULL");
    uint32_t i = 0;
    for (; i + kSpGraphSteps <= n_steps; i += kSpGraphSteps) {
        const int rc = launch_chunk(c);
        if (rc != SPG_OK) return rc;
    }
    return launch_steps(c, n_steps - i);
}

int spg_space_get_state(spg_space *c, uint32_t *t, int32_t *status, uint32_t *total) {
    if (!c) return fail(SPG_ERR_INVALID, "community is NULL");
    SpState st;
    const int rc = space_state(c, st);
    if (rc != SPG_OK) return rc;
    if (t) *t = st.t;
    if (status) *status = st.status;
    if (total) *total = st.total;
    return SPG_OK;
}

int spg_space_read_stats(spg_space *c, uint32_t first_step, uint32_t count, spg_space_stats *out) {
    if (!c || (!out && count)) return fail(SPG_ERR_INVALID, "NULL argument");
    SpState st;
    int rc = space_state(c, st);
    if (rc != SPG_OK) return rc;
    const uint64_t last = (uint64_t)first_step + count - 1;
    if (count && (first_step == 0 || last > st.t || (uint64_t)st.t - first_step >= c->ring_cap))
        return fail(SPG_ERR_RANGE, "steps %u..%llu not in the ring (completed %u)", first_step,
                    (unsigned long long)last, st.t);
    for (uint32_t i = 0; i < count; ++i) {
        const uint32_t slot = (first_step - 1 + i) % c->ring_cap;
        const cudaError_t e = cudaMemcpy(out + (size_t)i * c->ns, c->args.ring + (size_t)slot * c->ns,
                                         c->ns * sizeof(spg_space_stats), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "read stats");
    }
    return st.status == SPG_OK ? SPG_OK : fail(st.status, "community status %d (capacity exceeded)", st.status);
}

int spg_space_sizes(spg_space *c, uint32_t *sizes, size_t count) {
    if (!c || !sizes) return fail(SPG_ERR_INVALID, "NULL argument");
    if (count < c->nd) return fail(SPG_ERR_INVALID, "need %u entries", c->nd);
    SpState st;
    int rc = space_state(c, st);
    if (rc != SPG_OK) return rc;
    std::vector<uint32_t> offs(c->nd + 1);
    const cudaError_t e = cudaMemcpy(offs.data(), c->args.off[st.t & 1u], offs.size() * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read offsets");
    for (uint32_t d = 0; d < c->nd; ++d) sizes[d] = offs[d + 1] - offs[d];
    return SPG_OK;
}

int spg_space_read_deme(spg_space *c, uint32_t species, uint32_t patch, uint32_t *rec, uint8_t *age, size_t capacity,
                        uint32_t *n) {
    if (!c || !n) return fail(SPG_ERR_INVALID, "NULL argument");
    if (species >= c->ns || patch >= c->P) return fail(SPG_ERR_INVALID, "no such deme");
    SpState st;
    int rc = space_state(c, st);
    if (rc != SPG_OK) return rc;
    const uint32_t d = species * c->P + patch, par = st.t & 1u;
    uint32_t o[2];
    cudaError_t e = cudaMemcpy(o, c->args.off[par] + d, 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read offsets");
    *n = o[1] - o[0];
    if (!rec && !age) return SPG_OK;
    if (capacity < *n) return fail(SPG_ERR_INVALID, "buffer holds %zu individuals, need %u", capacity, *n);
    if (rec)
        e = cudaMemcpy(rec, c->args.geno[par] + (size_t)o[0] * 2 * c->W, (size_t)*n * 2 * c->W * 4,
                       cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && age) e = cudaMemcpy(age, c->args.age[par] + o[0], *n, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SPG_OK : cuda_fail(e, "read deme");
}

int spg_space_synchronize(spg_space *c) {
    if (!c) return fail(SPG_ERR_INVALID, "community is NULL");
    return space_sync(c);
}

void spg_space_destroy(spg_space *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->arena) c->alloc.release(c->arena, c->stream);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->side) cudaStreamSynchronize(c->side);
    if (c->chunk) cudaGraphExecDestroy(c->chunk);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->join) cudaEventDestroy(c->join);
    delete c;
}

}  // extern "C"
