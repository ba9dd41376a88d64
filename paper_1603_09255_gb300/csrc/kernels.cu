// Device kernels of the per-generation update (sm_103a) other than the
// offspring kernel (offspring.cuh): the continuous-allele generation kernel,
// the compaction kernel that closes every generation, and the set-up kernels
// (founders, survivor words of weighted parents, state resets).
//
// A generation of every population in a launch group is two launches
// (Fig. 1 A-F of the paper):
//   k_offspring  (offspring.cuh) draws both parents of every offspring from
//                the previous survivors (A), forms the gametes by crossover
//                masks and mutation XOR (B), sums the genetic value (C) and
//                decides survival from the threshold table (D); it writes the
//                child records, the alive bitmap, per-bucket survivor counts
//                and exact integer statistics;
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

#include "device_common.cuh"
#include "spegg_internal.h"

namespace spg {
namespace {

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

template <int G, int U, bool GROUP>
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
    // the block's population and its tile there (GROUP: a launch group of
    // several populations, from the tile map, one block per launch-wide tile of
    // 256 offspring; otherwise the segment in the kernel parameters)
    const Segment *sgp = &a.one;
    uint32_t tile = blockIdx.x;
    if constexpr (GROUP) {
        sgp = a.segs + __ldg(a.tile_seg + tile);
        tile -= sgp->tile_begin;
    }
    const Segment &sg = *sgp;
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
    const uint32_t base = tile * (uint32_t)kBlock;
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
// One block per bucket of kBucket offspring.  Its first kBucketWords threads
// read the bucket's bitmap words and the survivor counts of all earlier
// buckets and scan the words' popcounts; then kCompactCopyThreads threads
// (8 warps) write every survivor's index, in offspring order, at its rank =
// (survivors of earlier buckets) + (survivors before it in the bucket), and,
// for populations with a dense parent buffer, its record at the same rank
// (the parents of the next generation, read by rank without an index hop).
// The bucket's child records reach shared memory by bulk asynchronous copies
// of kChunkBytes each into a ring of kRingSlots slots (issued by one thread
// before the scan, the next chunk into a slot as soon as the copy threads are
// done with it), so the record copy is a stream of large reads instead of a
// dependent load per survivor; the survivors are stored from shared memory
// with whole-sector stores.  In a population's first bucket an extra warp
// closes the generation meanwhile (finalize_warp).  The block that finishes
// the last bucket commits the new state.  Every load that does not depend on
// the population state is issued together with it (both parities of the
// bucket counts are summed; the state picks one).
// 32 KB of ring per block: rings of 64 KB and more measured up to 40%
// slower, alone and next to other launch groups' offspring kernels
constexpr uint32_t kChunkBytes = 16384;  // bytes of one bulk copy of child records (one ring slot)
constexpr uint32_t kRingSlots = 2;       // chunks in flight per block

__device__ __forceinline__ void compaction_barrier() {
    asm volatile("bar.sync 1, %0;" ::"n"(kCompactCopyThreads) : "memory");  // the compaction threads
}

// A record of 2W words from shared memory (16-byte chunks, 8-byte for W = 1).
template <int W>
__device__ __forceinline__ void ring_record(uint32_t addr, uint32_t (&r)[2 * W]) {
    if constexpr (W == 1) {
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(addr) : "memory");
    } else {
#pragma unroll
        for (int q = 0; q < W / 2; ++q)
            asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(r[4 * q]), "=r"(r[4 * q + 1]), "=r"(r[4 * q + 2]), "=r"(r[4 * q + 3])
                         : "r"(addr + 16u * q)
                         : "memory");
    }
}

template <int W>
__device__ __forceinline__ void compact_bucket(const Segment &sg, uint32_t b) {
    constexpr int NW = kBucketWords / 32;          // warps that scan the bitmap words
    constexpr uint32_t REC = 8u * W;               // bytes per record
    constexpr uint32_t CHUNK = kChunkBytes / REC;  // offspring per ring slot
    constexpr uint32_t SLOT = kChunkBytes;         // bytes per ring slot
    constexpr uint32_t NCHUNK = kBucket / CHUNK;   // ring fills per bucket
    constexpr int CW = (int)(CHUNK / 32);          // bitmap words per chunk
    constexpr int WPW = CW / (int)(kCompactCopyThreads / 32);  // bitmap words per copying warp and chunk
    static_assert(kBucket % CHUNK == 0 && WPW >= 1, "chunks split the bucket among the copying warps");
    extern __shared__ __align__(128) unsigned char s_ring[];  // [kRingSlots][SLOT]
    __shared__ alignas(8) unsigned long long s_bar[kRingSlots];
    __shared__ uint32_t s_warp[NW];
    __shared__ uint32_t s_prev[NW];
    __shared__ uint32_t s_bits[kBucketWords], s_incl[kBucketWords];
    __shared__ uint32_t s_last, s_timeout;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool closer = tid >= (int)kCompactCopyThreads;  // the generation-closing warp
    const bool scanner = tid < (int)kBucketWords;
    const uint32_t valid_words = (sg.n + 31u) >> 5;
    const uint32_t w = b * kBucketWords + (uint32_t)tid;
    const uint32_t bits = (scanner && w < valid_words) ? __ldcg(sg.alive + w) : 0u;
    uint32_t prev0 = 0, prev1 = 0;
    for (uint32_t i = (uint32_t)tid; scanner && i < b; i += kBucketWords) {
        prev0 += __ldcg(sg.bucket_sum + i);
        prev1 += __ldcg(sg.bucket_sum + sg.nbuckets + i);
    }
    const PopNow now = read_state(sg.state);
    const uint32_t g = now.gen + 1u;
    const uint32_t first = b * kBucket, nb = min(kBucket, sg.n - first);  // the bucket's offspring
    const uint32_t nchunks = (nb + CHUNK - 1u) / CHUNK;
    const bool ring = sg.dense != nullptr && now.active;
    const uint32_t ring0 = (uint32_t)__cvta_generic_to_shared(s_ring);
    const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&s_bar[0]);
    const uint32_t *__restrict__ chi = sg.geno[g & 1u];
    // chunk c of the bucket into ring slot c % kRingSlots (a partial last
    // chunk rounded up to 16 bytes: record buffers are padded to 256 bytes)
    auto fill = [&](uint32_t c) {
        const uint32_t off = first + c * CHUNK, cnt = min(CHUNK, nb - c * CHUNK);
        bulk_load(ring0 + (c % kRingSlots) * SLOT, chi + (size_t)off * (2 * W), (cnt * REC + 15u) & ~15u,
                  bar0 + 8u * (c % kRingSlots));
    };
    if (tid == 0) {
        s_timeout = 0u;
        if (ring) {
            for (uint32_t k = 0; k < kRingSlots; ++k) mbar_init(bar0 + 8u * k, 1u);
            mbar_init_fence();
            for (uint32_t c = 0; c < kRingSlots && c < nchunks; ++c) fill(c);
        }
    }
    __syncthreads();  // barriers initialised
    if (!now.active) return;
    if (closer) {
        if (b == 0u) finalize_warp(sg, sg.prm, g, now.f);
        __threadfence();
    } else {
        if (scanner) {
            const uint32_t prev = __reduce_add_sync(0xFFFFFFFFu, (g & 1u) ? prev1 : prev0);
            uint32_t incl = __popc(bits);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            s_bits[tid] = bits;
            s_incl[tid] = incl;
            if (lane == 31) s_warp[warp] = incl;
            if (lane == 0) s_prev[warp] = prev;
        }
        compaction_barrier();
        uint32_t before = 0;  // survivors of all earlier buckets
#pragma unroll
        for (int q = 0; q < NW; ++q) before += s_prev[q];
        uint32_t *__restrict__ sout = sg.surv[g & 1u];
        uint32_t *__restrict__ dense = sg.dense;
        const uint32_t lt = (1u << lane) - 1u;
        for (uint32_t c = 0; c < NCHUNK; ++c) {
            if (c >= nchunks) break;
            if (ring && !mbar_wait(bar0 + 8u * (c % kRingSlots), (c / kRingSlots) & 1u)) s_timeout = 1u;
            const uint32_t slot = ring0 + (c % kRingSlots) * SLOT;
#pragma unroll
            for (int k = 0; k < WPW; ++k) {
                const int q = (int)c * CW + warp * WPW + k;  // bitmap word of the bucket
                const uint32_t word = s_bits[q];
                uint32_t r0 = before + s_incl[q] - __popc(word);
#pragma unroll
                for (int v = 0; v < NW; ++v) r0 += v < q / 32 ? s_warp[v] : 0u;
                if ((word >> lane) & 1u) {
                    const uint32_t rank = r0 + __popc(word & lt), idx = first + (uint32_t)q * 32u + lane;
                    sout[rank] = idx;
                    if (ring) {
                        uint32_t rec[2 * W];
                        ring_record<W>(slot + ((uint32_t)(q - (int)c * CW) * 32u + lane) * REC, rec);
                        store_record<W>(dense + (size_t)rank * (2 * W), rec);
                    }
                    if (sg.survw) {  // the survivor's acceptance thresholds as mother and as father
                        const uint32_t bin = __ldcg(sg.obin + idx);
                        const WeightParams *wt = sg.prm->weights;
                        sg.survw[rank] = (unsigned long long)idx | ((unsigned long long)__ldg(&wt->acc[0][bin]) << 32);
                        sg.survw[sg.n + rank] =
                            (unsigned long long)idx | ((unsigned long long)__ldg(&wt->acc[1][bin]) << 32);
                    }
                }
            }
            if (ring && c + kRingSlots < nchunks) {  // the slot is free once every copying thread is past it
                compaction_barrier();
                if (tid == 0 && !s_timeout) fill(c + kRingSlots);
            }
        }
    }
    // every block has read the state by now (its values fed the stores
    // above), and the closing warp of bucket 0 has published the next state
    __syncthreads();
    if (tid == 0) {
        if (s_timeout) {  // a copy did not land in time: the generation fails; wait (bounded) for
                          // the last copy issued into each slot before the block's memory goes away
            atomicExch(reinterpret_cast<int *>(&sg.state->status), SPG_ERR_TIMEOUT);
            for (uint32_t k = 0; k < kRingSlots && k < nchunks; ++k) {
                uint32_t lastc = k;
                while (lastc + kRingSlots < nchunks) lastc += kRingSlots;
                mbar_wait(bar0 + 8u * k, (lastc / kRingSlots) & 1u);
            }
        }
        s_last = (atomicAdd(&sg.state->done, 1u) == sg.nbuckets - 1u) ? 1u : 0u;
    }
    __syncthreads();
    if (s_last && tid == 0) {
        __threadfence();
        commit_state(sg.state, g);
    }
}

template <int W>
__global__ void __launch_bounds__(kCompactThreads, 3) k_compact(const __grid_constant__ GenArgs a) {
    griddep_release();  // the next generation's blocks may take this grid's place as its blocks finish
    griddep_wait();     // everything below reads the offspring kernel's results
    const uint32_t bkt = blockIdx.x;
    if (a.nsegs == 1u) {
        compact_bucket<W>(a.one, bkt);
    } else {
        const Segment &sg = a.segs[__ldg(a.bucket_seg + bkt)];
        compact_bucket<W>(sg, bkt - sg.bucket_begin);
    }
}

// A record of 2W words read through L2 and written with whole-sector stores.
template <int W>
__device__ __forceinline__ void copy_record(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst) {
    uint32_t r[2 * W];
    if constexpr (W == 1) {
        const uint2 v = __ldcg(reinterpret_cast<const uint2 *>(src));
        r[0] = v.x;
        r[1] = v.y;
    } else if constexpr (W == 2) {
        const uint4 v = __ldcg(reinterpret_cast<const uint4 *>(src));
        r[0] = v.x;
        r[1] = v.y;
        r[2] = v.z;
        r[3] = v.w;
    } else {
#pragma unroll
        for (int q = 0; q < W / 4; ++q)
            asm volatile("ld.global.cg.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=r"(r[8 * q]), "=r"(r[8 * q + 1]), "=r"(r[8 * q + 2]), "=r"(r[8 * q + 3]),
                           "=r"(r[8 * q + 4]), "=r"(r[8 * q + 5]), "=r"(r[8 * q + 6]), "=r"(r[8 * q + 7])
                         : "l"(src + 8 * q));
    }
    store_record<W>(dst, r);
}

// dense[r] = geno[surv[r]] (surv null: r) for r < S: the dense parent buffer
// of founders or of a restored generation.
template <int W>
__global__ void k_dense_gather(const uint32_t *__restrict__ geno, const uint32_t *__restrict__ surv, uint32_t S,
                               uint32_t *__restrict__ dense) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= S) return;
    const uint32_t idx = surv ? surv[r] : r;
    copy_record<W>(geno + (size_t)idx * (2 * W), dense + (size_t)r * (2 * W));
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

OffspringKernel offspring_kernel_w1(const Shape &shape, bool linked, bool weighted, bool staged);
OffspringKernel offspring_kernel_w2(const Shape &shape, bool linked, bool weighted, bool staged);
OffspringKernel offspring_kernel_w4(const Shape &shape, bool linked, bool weighted, bool staged);
OffspringKernel offspring_kernel_w8(const Shape &shape, bool linked, bool weighted, bool staged);

bool supported_shape(uint32_t words, const Shape &s) {
    if (!(s.block == 128 || s.block == 256 || s.block == 512)) return false;
    if (s.lanes == 2) return words >= 4 && s.items == 1;
    if (s.lanes != 1) return false;
    return words <= 2 ? (s.items == 1 || s.items == 2) : s.items == 1;
}

uint32_t tile_size(const Shape &s) { return s.block * s.items / s.lanes; }

uint32_t compact_smem() { return kRingSlots * kChunkBytes; }

GenKernel compact_kernel(uint32_t words) {
    GenKernel k;
    switch (words) {
        case 2: k = &k_compact<2>; break;
        case 4: k = &k_compact<4>; break;
        case 8: k = &k_compact<8>; break;
        default: k = &k_compact<1>; break;  // and populations without a dense buffer (no record copies)
    }
    // the ring of bulk-copied child records is dynamic shared memory
    cudaFuncSetAttribute(reinterpret_cast<const void *>(k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)compact_smem());
    return k;
}

// ------------------------------------------------- per-locus allele counts
// 32 x 32 bit transpose across a warp: afterwards bit b of lane i is what bit
// i of lane b was.  Stage s swaps the off-diagonal s x s blocks between lanes
// i and i ^ s (masks keep the low s bits of each 2s-bit group).
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, uint32_t lane) {
    constexpr uint32_t M[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const uint32_t s = 16u >> k;
        const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, (int)s);
        x = (lane & s) ? (((y >> s) & M[k]) | (x & ~M[k])) : ((x & M[k]) | ((y << s) & ~M[k]));
    }
    return x;
}

// Allele-1 copies of every locus over both haplotypes of the generation just
// formed (all N offspring; S2 "Genetics": count / 2N is the locus's allele
// frequency).  A warp takes 32 records at a time, one per lane; each lane
// adds its record's words into bit-sliced counters (plane k holds bit k of
// every locus's count among the lane's records), and every kLocusPlanes
// records' worth of room (and at the end) the warp transposes each plane
// across its lanes, so that lane b holds bit b of the 32 lanes' planes, and
// adds 2^k times its population count to locus 32w + b; the warps of a block add theirs in
// shared memory, blocks add theirs into the accumulator row, and the block
// that finishes last moves the row to the generation's ring slot, clears it
// and re-arms the counter.  A generation already counted (a launch after the
// population has stopped forms none) is left as it is.
template <int W, bool GROUP>
__global__ void __launch_bounds__(kLocusBlock) k_locus_counts(const __grid_constant__ GenArgs a, const LocusArgs la_) {
    constexpr uint32_t L = 32u * W, NW = kLocusBlock / 32u;
    __shared__ uint32_t s_cnt[L];
    __shared__ uint32_t s_last;
    // the block's population, its arguments and the block's place among its
    // blocks (GROUP: a launch group, from the block map)
    const Segment *sgp = &a.one;
    const LocusArgs *lap = &la_;
    uint32_t blk = blockIdx.x, nblk = gridDim.x;
    if constexpr (GROUP) {
        const uint32_t m = __ldg(la_.block_member + blockIdx.x);
        sgp = a.segs + m;
        lap = la_.member + m;
        blk = blockIdx.x - lap->first;
        nblk = lap->blocks;
    }
    const Segment &sg = *sgp;
    const LocusArgs &la = *lap;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t g = ld_relaxed_u32(&sg.state->gen);  // the generation the compaction just committed
    if (g == 0u || ld_relaxed_u32(la.last) == g) return;  // the founders, or counted already
    for (uint32_t i = tid; i < L; i += kLocusBlock) s_cnt[i] = 0u;
    __syncthreads();
    const uint32_t *rec = sg.geno[g & 1u];
    constexpr int K = kLocusPlanes;
    uint32_t acc[W], v[2 * W][K];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = 0u;
#pragma unroll
    for (int c = 0; c < 2 * W; ++c)
#pragma unroll
        for (int k = 0; k < K; ++k) v[c][k] = 0u;
    auto flush = [&]() {  // the whole warp: every lane's planes into the counts
#pragma unroll
        for (int c = 0; c < 2 * W; ++c)
#pragma unroll
            for (int k = 0; k < K; ++k) {
                acc[c % W] += (uint32_t)__popc(warp_transpose32(v[c][k], lane)) << k;
                v[c][k] = 0u;
            }
    };
    const uint32_t groups = (sg.n + 31u) >> 5, stride = nblk * NW;
    constexpr uint32_t U = kLocusBatch;  // groups whose records are loaded before any is added
    uint32_t held = 0;  // records each lane has added since the last flush (the same in the whole warp)
    for (uint32_t q0 = blk * NW + warp; q0 < groups; q0 += U * stride) {
        uint32_t r[U][2 * W];
#pragma unroll
        for (uint32_t u = 0; u < U; ++u) {
            const uint32_t q = q0 + u * stride, i = q * 32u + lane;
            if (q < groups && i < sg.n) {
                load_record<W>(rec + (size_t)i * (2 * W), r[u]);
            } else {
#pragma unroll
                for (int c = 0; c < 2 * W; ++c) r[u][c] = 0u;
            }
        }
        if (held + U > (1u << K) - 1u) {  // the counters hold up to 2^K - 1
            flush();
            held = 0;
        }
#pragma unroll
        for (uint32_t u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < 2 * W; ++c) {  // ripple-carry add of one bit per locus
                uint32_t x = r[u][c];
#pragma unroll
                for (int k = 0; k < K - 1; ++k) {
                    const uint32_t carry = v[c][k] & x;
                    v[c][k] ^= x;
                    x = carry;
                }
                v[c][K - 1] ^= x;
            }
        held += U;
    }
    if (held) flush();
#pragma unroll
    for (int w = 0; w < W; ++w) atomicAdd(&s_cnt[32u * w + lane], acc[w]);
    __syncthreads();
    for (uint32_t i = tid; i < L; i += kLocusBlock)
        if (s_cnt[i]) atomicAdd(la.acc + i, s_cnt[i]);
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(la.done, 1u) == nblk - 1u ? 1u : 0u;
    __syncthreads();
    if (s_last) {  // every block has added its counts
        __threadfence();
        uint32_t *slot = la.ring + (size_t)((g - 1u) % la.cap) * L;
        for (uint32_t i = tid; i < L; i += kLocusBlock) {
            slot[i] = __ldcg(la.acc + i);
            la.acc[i] = 0u;
        }
        if (tid == 0) {
            *la.done = 0u;
            *la.last = g;
        }
    }
}

template <int W>
LocusKernel locus_instance(bool group) {
    return group ? &k_locus_counts<W, true> : &k_locus_counts<W, false>;
}

LocusKernel locus_kernel(uint32_t words, bool group) {
    switch (words) {
        case 1: return locus_instance<1>(group);
        case 2: return locus_instance<2>(group);
        case 4: return locus_instance<4>(group);
        case 8: return locus_instance<8>(group);
        default: return nullptr;
    }
}

int launch_dense_gather(uint32_t words, const uint32_t *geno, const uint32_t *surv, uint32_t S, uint32_t *dense,
                        void *stream) {
    if (S == 0) return SPG_OK;
    const dim3 grid((S + 255) / 256), block(256);
    cudaStream_t s = (cudaStream_t)stream;
    switch (words) {
        case 1: k_dense_gather<1><<<grid, block, 0, s>>>(geno, surv, S, dense); break;
        case 2: k_dense_gather<2><<<grid, block, 0, s>>>(geno, surv, S, dense); break;
        case 4: k_dense_gather<4><<<grid, block, 0, s>>>(geno, surv, S, dense); break;
        case 8: k_dense_gather<8><<<grid, block, 0, s>>>(geno, surv, S, dense); break;
        default: return SPG_ERR_INVALID;
    }
    return cudaGetLastError() == cudaSuccess ? SPG_OK : SPG_ERR_CUDA;
}

OffspringKernel offspring_kernel(uint32_t words, const Shape &shape, bool linked, bool weighted, bool eco, bool dom,
                                 bool staged) {
    staged = staged && kStagedParents && words <= 4 && shape.lanes == 1 && !linked;
    OffspringKernel k;
    switch (words) {
        case 1: k = offspring_kernel_w1(shape, linked, weighted, staged); break;
        case 2: k = offspring_kernel_w2(shape, linked, weighted, staged); break;
        case 4: k = offspring_kernel_w4(shape, linked, weighted, staged); break;
        case 8: k = offspring_kernel_w8(shape, linked, weighted, staged); break;
        default: return OffspringKernel{};
    }
    if (!k.fn) return k;
    // dynamic shared memory: byte tables, thresholds (and attack rates when
    // some population of the launch has an ecology), dominance byte tables
    // (only when some population has dominance)
    const uint32_t lut = words * 4u * (uint32_t)kLutWords * 4u;
    const uint32_t tab = eco ? (uint32_t)kBins * 8u : (uint32_t)kBins * 4u;
    k.words = words;
    k.eco_table = eco ? 1u : 0u;
    k.smem_dlut = dom ? lut + tab : 0u;
    k.smem = lut + tab + (dom ? lut : 0u);
    if (staged) {  // the ring of staged parent records
        k.smem_parents = k.smem;
        k.smem += kParentStages * 2u * k.block * k.items * 8u * words;
    }
    return k;
}

template <int G>
GenKernel cont_instance(bool group) {
    return group ? &k_offspring_cont<G, kContInFlight, true> : &k_offspring_cont<G, kContInFlight, false>;
}

OffspringKernel continuous_kernel(uint32_t n_loci, bool group) {
    OffspringKernel k;
    switch (n_loci) {
        case 32: k.fn = cont_instance<4>(group); break;
        case 64: k.fn = cont_instance<8>(group); break;
        case 128: k.fn = cont_instance<16>(group); break;
        case 256: k.fn = cont_instance<32>(group); break;
        default: return OffspringKernel{};
    }
    k.block = kBlock;
    k.items = 1;
    k.smem = 0;
    k.resident = 0;
    k.persistent = false;  // one block per 256 offspring
    return k;
}

int prepare_offspring(OffspringKernel &k) {
    if (!k.fn) return SPG_ERR_INVALID;
    const void *fn = reinterpret_cast<const void *>(k.fn);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return SPG_ERR_CUDA;
    if (k.persistent) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
        if (e != cudaSuccess) return SPG_ERR_CUDA;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)k.block, k.smem);
    if (e != cudaSuccess || per_sm <= 0) return SPG_ERR_CUDA;
    k.resident = (uint32_t)per_sm * (uint32_t)sms;
    return SPG_OK;
}

void apply_kernel(const OffspringKernel &k, GenArgs &a) {
    a.eco_table = k.eco_table;
    a.smem_dlut = k.smem_dlut;
    a.smem_parents = k.smem_parents;
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