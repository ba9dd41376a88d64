// The offspring kernel of the per-generation update (sm_103a): Fig. 1 A-D
// of the paper for every offspring of every population of a launch.
//
// Persistent: each block forms the tiles of its runs (a run is a contiguous
// range of one population's tiles of BLOCK * ITEMS offspring; a single
// population gives each block one contiguous share).  Per offspring it draws
// both parents from the previous survivors (A), forms the gametes by
// crossover masks and mutation XOR (B), sums the genetic value (C) and decides
// survival (D); it writes the child record, the alive bitmap, per-bucket
// survivor counts and exact integer statistics.
//
// Parents.  The compaction of the previous generation wrote the survivors'
// records in rank order (the population's dense parent buffer), so parent
// rank r = floor(u * S / 2^32) is record r of that buffer: one random record
// read per parent and no survivor-index hop.  (A launch without dense
// buffers -- the allocation-free call -- reads survivor index r first.)
// Each record is fetched with a single vector load (256 bits for L = 128,
// two for L = 256): random reads are bounded by the number of L2 requests, and
// one request per 32-byte sector is the minimum.  The records of tile t+1 are
// loaded into registers while tile t is formed, the draws of tile t+2 made
// before that; or, for parents in HBM, they go through a shared-memory ring
// two tiles ahead (staged parent records, below).  In a launch over many populations a block also prefetches its
// next run's parent records into L2 with one bulk prefetch per 16 KB, so the
// random reads of a population resident in HBM hit L2 (random 32-byte reads
// from DRAM run at a fraction of the sequential bandwidth).
//
// Tables.  Per run the block copies the population's tables into its dynamic
// shared memory with cp.async:
//   * the survival thresholds by phenotype bin, and the attack rates when the
//     launch carries an ecology;
//   * the byte tables of the genetic value: entry (k, v) is the sum of the
//     effects of loci 8k .. 8k+7 whose allele bit is set in v, so a
//     haplotype's additive value is L/8 shared-memory lookups instead of a
//     popcount per effect bit plane and word (a popcount issues at a quarter
//     of the integer rate); dominance deviations likewise on h0 ^ h1.
#pragma once

#include "device_common.cuh"

namespace spg {
namespace {

// Blocks per SM the compiler is asked to fit (a register cap:
// 65536 / (BLOCK * blocks) per thread): 16 warps per SM.
constexpr int offspring_min_blocks(int block) { return block >= 512 ? 1 : 512 / block; }

// Draws of one tile: parents (ranks in the dense parent buffer, or record
// indices through the survivor list) and the survival / mutation-count draws
// of each item.
template <int ITEMS>
struct TileDraws {
    uint32_t mom[ITEMS], dad[ITEMS], u_surv[ITEMS], u_mut[ITEMS];
};

// Parent records of one tile, in registers.
template <int W, int ITEMS>
struct TileRecs {
    uint32_t m[ITEMS][2 * W], f[ITEMS][2 * W];
};

// One run's population as the tile loop sees it.
struct SegCtx {
    const PopParams *P;
    const uint32_t *par;               // parent records: dense buffer (by rank) or all records (by index)
    const uint32_t *sin;               // survivor indices (null: parents by rank in the dense buffer)
    uint32_t *chi;
    uint32_t *alive;
    uint32_t *bucket_now;
    const unsigned long long *survw;   // weighted parents: [2][n] survivor index | role threshold << 32
    uint16_t *obin;                    // weighted parents: bins of the offspring formed
    uint32_t dlut;                     // byte offset of the dominance byte tables (0: none)
    uint32_t n, S, f, g, rep, k0, k1, kmax, shift;
    int32_t bias;
    bool eco;
};

// The dynamic shared memory of the offspring kernel: the byte tables of the
// additive value at 0 (so a lookup's address is its byte value times 4 plus a
// constant), the survival thresholds after them, the attack rates after those
// (eco launches), the dominance byte tables at the offset the launch gives.
extern __shared__ __align__(16) unsigned char s_dyn[];
template <int W>
struct SmemLayout {
    static constexpr uint32_t kThr = 4096u * W;       // 4W byte tables of 256 int32
    static constexpr uint32_t kAtt = kThr + kBins * 4u;
};

__device__ __forceinline__ uint32_t smem_u32(uint32_t byte_off) {
    return *reinterpret_cast<const uint32_t *>(s_dyn + byte_off);
}
__device__ __forceinline__ int32_t smem_i32(uint32_t byte_off) {
    return *reinterpret_cast<const int32_t *>(s_dyn + byte_off);
}

// Weighted parents (pi = 0 mother, 1 father) by bounded rejection sampling:
// proposal k draws a uniform survivor rank and an acceptance value (lanes
// 2(k%2), 2(k%2)+1 of Philox sub pi<<8 | k/2) and is taken when the
// survivor's bin threshold is certain or above the value; the last proposal
// stands if all kMateAttempts are rejected.  Proposals go in pairs (one
// Philox block), both roles together, so four gathers are in flight at once;
// the first accepted proposal in order is the parent, as if they were tried
// one at a time.  A gathered word carries the survivor's threshold for the
// role (looked up once per survivor by the compaction), so a proposal is one
// 8-byte read and a comparison.  The parent is returned as its rank.
static_assert(kMateAttempts % 2 == 0, "whole Philox blocks of proposals");

// Proposals k and k+1 of one role (ranks r0, r1 and their words): whether one
// was taken, and the parent rank (the first taken, else proposal k+1).
__device__ __forceinline__ bool weighted_pair(const uint4 &d, uint32_t r0, uint32_t r1, unsigned long long e0,
                                              unsigned long long e1, uint32_t &parent) {
    const uint32_t t0 = (uint32_t)(e0 >> 32), t1 = (uint32_t)(e1 >> 32);
    const bool a0 = t0 == kCertain || d.y < t0, a1 = t1 == kCertain || d.w < t1;
    parent = a0 ? r0 : r1;
    return a0 || a1;
}

__device__ __forceinline__ void weighted_parents(const SegCtx &c, uint32_t j, uint32_t &mom, uint32_t &dad) {
    bool open_m = true, open_f = true;
    for (uint32_t k = 0; k < kMateAttempts && (open_m || open_f); k += 2) {
        const uint32_t sub = (kMateW << 24) | (k >> 1);
        uint4 dm = make_uint4(0u, 0u, 0u, 0u), df = dm;
        uint32_t rm0 = 0, rm1 = 0, rf0 = 0, rf1 = 0;
        unsigned long long em0 = 0, em1 = 0, ef0 = 0, ef1 = 0;
        if (open_m) {
            dm = philox(make_uint4(j, c.g, c.rep, sub), c.k0, c.k1);
            rm0 = __umulhi(dm.x, c.S);
            rm1 = __umulhi(dm.z, c.S);
            em0 = __ldcg(c.survw + rm0);
            em1 = __ldcg(c.survw + rm1);
        }
        if (open_f) {
            df = philox(make_uint4(j, c.g, c.rep, sub | (1u << 8)), c.k0, c.k1);
            rf0 = __umulhi(df.x, c.S);
            rf1 = __umulhi(df.z, c.S);
            ef0 = __ldcg(c.survw + c.n + rf0);
            ef1 = __ldcg(c.survw + c.n + rf1);
        }
        if (open_m) open_m = !weighted_pair(dm, rm0, rm1, em0, em1, mom);
        if (open_f) open_f = !weighted_pair(df, rf0, rf1, ef0, ef1, dad);
    }
}

template <int ITEMS, int BLOCK, bool WEIGHTED>
__device__ __forceinline__ void draw_parents(const SegCtx &c, uint32_t base, int tid, TileDraws<ITEMS> &d) {
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const uint32_t j = base + (uint32_t)(it * BLOCK + tid);
        d.mom[it] = d.dad[it] = d.u_surv[it] = d.u_mut[it] = 0u;
        if (j < c.n) {
            const uint4 r = philox(make_uint4(j, c.g, c.rep, kMate << 24), c.k0, c.k1);
            if constexpr (WEIGHTED) {
                weighted_parents(c, j, d.mom[it], d.dad[it]);
            } else {
                d.mom[it] = __umulhi(r.x, c.S);
                d.dad[it] = __umulhi(r.y, c.S);
                if (c.sin) {  // survivor indices through L2 only (random 4-byte reads)
                    d.mom[it] = __ldcg(c.sin + d.mom[it]);
                    d.dad[it] = __ldcg(c.sin + d.dad[it]);
                }
            }
            d.u_surv[it] = r.z;
            d.u_mut[it] = r.w;
        }
    }
}

// One parent record (2W words) in a single request per 32-byte sector,
// through L2 only (the parents are read-only for the whole launch).
template <int W>
__device__ __forceinline__ void load_parent(const uint32_t *__restrict__ p, uint32_t (&r)[2 * W]) {
    if constexpr (W == 1) {
        asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "l"(p));
    } else if constexpr (W == 2) {
        asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "l"(p));
    } else {
#pragma unroll
        for (int q = 0; q < W / 4; ++q)
            asm volatile("ld.global.nc.L1::no_allocate.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=r"(r[8 * q]), "=r"(r[8 * q + 1]), "=r"(r[8 * q + 2]), "=r"(r[8 * q + 3]),
                           "=r"(r[8 * q + 4]), "=r"(r[8 * q + 5]), "=r"(r[8 * q + 6]), "=r"(r[8 * q + 7])
                         : "l"(p + 8 * q));
    }
}

template <int W, int ITEMS, int BLOCK>
__device__ __forceinline__ void load_parents(const SegCtx &c, uint32_t base, int tid, const TileDraws<ITEMS> &d,
                                             TileRecs<W, ITEMS> &rec) {
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const uint32_t j = base + (uint32_t)(it * BLOCK + tid);
        if (j < c.n) {
            load_parent<W>(c.par + (size_t)d.mom[it] * (2 * W), rec.m[it]);
            load_parent<W>(c.par + (size_t)d.dad[it] * (2 * W), rec.f[it]);
        }
    }
}

// Prefetch records [r0, r1) of a parent buffer into L2: one bulk prefetch of
// up to 16 KB per thread (the buffer is 256-byte aligned and the prefetched
// length is cut to a multiple of 16 bytes, as the instruction requires).
template <int W, int BLOCK>
__device__ __forceinline__ void prefetch_parents(const uint32_t *par, uint32_t r0, uint32_t r1, int tid) {
    constexpr uint32_t kRec = 8u * W;    // bytes per record
    constexpr uint32_t kChunk = 16384u;  // bytes per prefetch
    if (r1 <= r0) return;
    const size_t a0 = ((size_t)r0 * kRec + 15u) & ~(size_t)15;  // 16-byte aligned start inside the range
    const char *lo = reinterpret_cast<const char *>(par) + a0;
    const size_t end = (size_t)r1 * kRec;
    if (end <= a0) return;
    const size_t n16 = (end - a0) & ~(size_t)15;
    for (size_t off = (size_t)tid * kChunk; off < n16; off += (size_t)BLOCK * kChunk) {
        const uint32_t len = (uint32_t)(n16 - off < kChunk ? n16 - off : kChunk);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo + off), "r"(len) : "memory");
    }
}

// Sum of the byte-table entries of one word x holding loci 32w .. 32w+31 (its
// four bytes): part of a haplotype's genetic value (eq. S2-phenval, per locus
// e_l * allele), exact in int32.  lut: byte offset of the tables (0 for the
// additive ones, a compile-time constant then).
__device__ __forceinline__ int32_t byte_table_word(uint32_t lut, uint32_t w, uint32_t x) {
    constexpr uint32_t T = (uint32_t)kLutWords * 4u;  // bytes per table
    const uint32_t t = lut + 4u * w * T;
    return smem_i32(t + ((x << 2) & 0x3FCu)) + smem_i32(t + T + ((x >> 6) & 0x3FCu)) +
           smem_i32(t + 2u * T + ((x >> 14) & 0x3FCu)) + smem_i32(t + 3u * T + ((x >> 22) & 0x3FCu));
}

// Genetic value (Fig. 1C) of a record from the byte tables: both
// haplotypes' additive values, plus the dominance deviations of the
// heterozygous loci (h0 ^ h1) when dlut is set; allele and heterozygosity
// counts for the statistics.
template <int W, int w = 0>
__device__ __forceinline__ void genetic_value(const uint32_t (&ch)[2 * W], uint32_t dlut, int32_t &raw, uint32_t &allele,
                                              uint32_t &hz) {
    if constexpr (w < W) {
        const uint32_t x = ch[w] ^ ch[W + w];
        raw += byte_table_word(0u, (uint32_t)w, ch[w]) + byte_table_word(0u, (uint32_t)w, ch[W + w]);
        if (dlut) raw += byte_table_word(dlut, (uint32_t)w, x);
        allele += __popc(ch[w]) + __popc(ch[W + w]);
        hz += __popc(x);
        genetic_value<W, w + 1>(ch, dlut, raw, allele, hz);
    }
}

struct ThreadStats {
    long long sum_raw = 0, sum_raw_s = 0;
    unsigned long long sum_raw2 = 0, cons = 0;
    uint32_t het = 0, allele = 0;
    int mn = INT_MAX, mx = INT_MIN;
};

// One tile: gametes (B), genetic value (C), survival (D), bitmap (E, first half).
template <int W, int ITEMS, int BLOCK, bool LINKED, bool WEIGHTED>
__device__ __forceinline__ uint32_t offspring_tile(const SegCtx &c, uint32_t base, int tid, int lane, int warp,
                                                   const TileRecs<W, ITEMS> &rec, const TileDraws<ITEMS> &dr,
                                                   const uint32_t *s_cdf, ThreadStats &ts, const LinkSmem &lk) {
    constexpr int NW = BLOCK / 32;
    uint32_t alive_count = 0;  // the warp's survivors (same in every lane)
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const uint32_t j = base + (uint32_t)(it * BLOCK + tid);
        bool alive = false;
        uint32_t mm[LINKED ? W : 1], mf[LINKED ? W : 1];
        if constexpr (LINKED)  // (B) the linkage-map masks, by the whole warp
            linked_masks_warp<W>(lk, j, j < c.n, c.g, c.rep, c.k0, c.k1, mm, mf);
        if (j < c.n) {
            const uint32_t(&pm)[2 * W] = rec.m[it];
            const uint32_t(&pf)[2 * W] = rec.f[it];
            uint32_t ch[2 * W];
            if constexpr (LINKED) {
                // (B) gametes under the linkage map
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
            const uint32_t u_mut = dr.u_mut[it];
            if (c.kmax != 0u && u_mut >= s_cdf[0]) {
                uint32_t k = 0;
                for (uint32_t i = 0; i < c.kmax; ++i) k += (u_mut >= s_cdf[i]) ? 1u : 0u;
                mutate<W>(ch, k, j, c.g, c.rep, c.k0, c.k1);
            }
            store_record<W>(c.chi + (size_t)j * (2 * W), ch);

            // (C) genetic value from the byte tables
            int32_t raw = 0;
            uint32_t allele = 0, hz = 0;
            genetic_value<W>(ch, c.dlut, raw, allele, hz);
            // (D) survival: the bin's threshold scaled by the resource factor
            const long long v = (long long)raw + (long long)c.bias;
            const uint32_t bin = v < 0 ? 0u : (uint32_t)min(v >> c.shift, (long long)(kBins - 1));
            if constexpr (WEIGHTED) c.obin[j] = (uint16_t)bin;
            uint32_t thr = smem_u32(SmemLayout<W>::kThr + bin * 4u);
            if (c.f != kCertain) thr = __umulhi(thr, c.f);
            alive = (thr == kCertain) || (dr.u_surv[it] < thr);

            ts.sum_raw += raw;
            ts.sum_raw2 += (unsigned long long)((long long)raw * (long long)raw);
            ts.mn = min(ts.mn, raw);
            ts.mx = max(ts.mx, raw);
            ts.het += hz;
            ts.allele += allele;
            if (alive) {
                ts.sum_raw_s += raw;
                if (c.eco) ts.cons += smem_u32(SmemLayout<W>::kAtt + bin * 4u);
            }
        }
        // (E, first half) alive bitmap word (base + it*BLOCK + 32*warp)/32
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, alive);
        if (lane == 0) c.alive[(base >> 5) + (uint32_t)(it * NW + warp)] = bal;
        alive_count += __popc(bal);
    }
    return alive_count;
}

// Copy the run's tables into shared memory (see the file comment): 16-byte
// cp.async chunks spread over the block, committed as one group.  eco: the
// launch has an attack-rate table (zeros for a population without ecology);
// dlut: the population's dominance tables are needed.
template <int W, int BLOCK>
__device__ __forceinline__ void copy_tables(const PopParams *P, bool eco, bool has_eco, uint32_t dyn, uint32_t dlut_off,
                                            bool dlut, int tid) {
    const uint32_t s_lut = dyn, s_thr = dyn + SmemLayout<W>::kThr, s_att = dyn + SmemLayout<W>::kAtt,
                   s_dlut = dyn + dlut_off;
    constexpr uint32_t kTab16 = (uint32_t)kBins * 4u / 16u;         // 16-byte chunks of a bin table
    constexpr uint32_t kLut16 = (uint32_t)W * 4u * kLutWords / 4u;  // of the 4W byte tables
    for (uint32_t i = (uint32_t)tid; i < kTab16; i += BLOCK) cp_async_16(s_thr + 16u * i, P->table + 4u * i);
    if (eco) {
        if (has_eco) {
            for (uint32_t i = (uint32_t)tid; i < kTab16; i += BLOCK) cp_async_16(s_att + 16u * i, P->attack + 4u * i);
        } else {
            for (uint32_t i = (uint32_t)tid; i < kTab16; i += BLOCK)
                asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(s_att + 16u * i), "r"(0u) : "memory");
        }
    }
    for (uint32_t i = (uint32_t)tid; i < kLut16; i += BLOCK) cp_async_16(s_lut + 16u * i, P->lut + 4u * i);
    if (dlut)
        for (uint32_t i = (uint32_t)tid; i < kLut16; i += BLOCK) cp_async_16(s_dlut + 16u * i, P->dlut + 4u * i);
    cp_async_commit();
}

// Tiles [lt0, lt1) of one run (see the file comment for the pipeline).
template <int W, int ITEMS, int BLOCK, bool LINKED, bool WEIGHTED>
__device__ __forceinline__ void offspring_run(const SegCtx &c, uint32_t lt0, uint32_t lt1, uint32_t *bucket_next,
                                              int tid, int lane, int warp, const uint32_t *s_cdf, ThreadStats &ts,
                                              const LinkSmem &lk, uint32_t &warp_alive) {
    constexpr uint32_t TILE = (uint32_t)(BLOCK * ITEMS);
    TileDraws<ITEMS> d0, d1;
    TileRecs<W, ITEMS> ra, rb;
    draw_parents<ITEMS, BLOCK, WEIGHTED>(c, lt0 * TILE, tid, d0);
    if (lt0 + 1 < lt1) draw_parents<ITEMS, BLOCK, WEIGHTED>(c, (lt0 + 1) * TILE, tid, d1);
    load_parents<W, ITEMS, BLOCK>(c, lt0 * TILE, tid, d0, ra);
    cp_async_wait<0>();
    __syncthreads();  // the run's tables (and cdf) are visible to every thread

    uint32_t bucket_alive = 0, bucket_cur = (lt0 * TILE) / kBucket;
    // one tile: prefetch the next tile's records, draw the one after next
    // (before forming this one, so the compiler can interleave its Philox
    // rounds with the tile's; parent ranks need no memory access, so only the
    // records' latency has to be covered), form this one
    auto step = [&](uint32_t lt, const TileRecs<W, ITEMS> &cur, TileRecs<W, ITEMS> &nxt) {
        const uint32_t base = lt * TILE;
        if (lt + 1 < lt1) load_parents<W, ITEMS, BLOCK>(c, base + TILE, tid, d1, nxt);
        if (tid == 0 && base % kBucket == 0u) bucket_next[base / kBucket] = 0u;
        const uint32_t bkt = base / kBucket;
        if (bkt != bucket_cur) {
            if (lane == 0 && bucket_alive) atomicAdd(&c.bucket_now[bucket_cur], bucket_alive);
            bucket_alive = 0;
            bucket_cur = bkt;
        }
        TileDraws<ITEMS> d2;
        draw_parents<ITEMS, BLOCK, WEIGHTED>(c, base + 2 * TILE, tid, d2);  // past the run: unused
        const uint32_t cnt =
            offspring_tile<W, ITEMS, BLOCK, LINKED, WEIGHTED>(c, base, tid, lane, warp, cur, d0, s_cdf, ts, lk);
        bucket_alive += cnt;
        warp_alive += cnt;
        d0 = d1;
        d1 = d2;
    };
    for (uint32_t lt = lt0; lt < lt1; lt += 2) {  // record sets alternate, so no register copies
        step(lt, ra, rb);
        if (lt + 1 < lt1) step(lt + 1, rb, ra);
    }
    if (lane == 0 && bucket_alive) atomicAdd(&c.bucket_now[bucket_cur], bucket_alive);
}

// ------------------------------------------------- staged parent records
// The single-lane kernels for L <= 128 without linkage keep their parents'
// records in a shared-memory ring of kParentStages tiles instead of
// registers: each thread copies its own items' records with cp.async
// kParentStages - 1 tiles ahead and reads them back when it forms the tile,
// so the loads in flight hold no registers and need no block barrier.  Used
// where the parents come from HBM (launch groups, weighted populations,
// populations with more than kStageParentBytes of parents); an L2-resident
// population is faster with the register prefetch.  Slot
// x = it * BLOCK + tid of stage s, parent p: 16-byte planes q (8-byte slots
// for W = 1), plane-major so a warp's accesses are conflict-free.
template <int W, int ITEMS, int BLOCK>
__device__ __forceinline__ uint32_t parent_slot(uint32_t ring, uint32_t s, uint32_t p, uint32_t q, uint32_t x) {
    constexpr uint32_t TILE = (uint32_t)(BLOCK * ITEMS);
    if constexpr (W == 1) return ring + ((s * 2u + p) * TILE + x) * 8u;
    else return ring + (((s * 2u + p) * (uint32_t)(W / 2) + q) * TILE + x) * 16u;
}

template <int W, int ITEMS, int BLOCK>
__device__ __forceinline__ void stage_parents(const SegCtx &c, uint32_t base, int tid, const TileDraws<ITEMS> &d,
                                              uint32_t ring, uint32_t s) {
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const uint32_t j = base + (uint32_t)(it * BLOCK + tid), x = (uint32_t)(it * BLOCK + tid);
        if (j < c.n) {
#pragma unroll
            for (uint32_t p = 0; p < 2u; ++p) {
                const uint32_t *src = c.par + (size_t)(p ? d.dad[it] : d.mom[it]) * (2 * W);
                if constexpr (W == 1) {
                    cp_async_8(parent_slot<W, ITEMS, BLOCK>(ring, s, p, 0u, x), src);
                } else {
#pragma unroll
                    for (uint32_t q = 0; q < (uint32_t)(W / 2); ++q)
                        cp_async_16(parent_slot<W, ITEMS, BLOCK>(ring, s, p, q, x), src + 4u * q);
                }
            }
        }
    }
    cp_async_commit();  // one group per tile (empty past the run's end), so group counts stay uniform
}

template <int W, int ITEMS, int BLOCK>
__device__ __forceinline__ void read_parents(uint32_t ring, uint32_t s, int tid, TileRecs<W, ITEMS> &rec) {
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const uint32_t x = (uint32_t)(it * BLOCK + tid);
#pragma unroll
        for (uint32_t p = 0; p < 2u; ++p) {
            uint32_t(&r)[2 * W] = p ? rec.f[it] : rec.m[it];
            if constexpr (W == 1) {
                asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];"
                             : "=r"(r[0]), "=r"(r[1])
                             : "r"(parent_slot<W, ITEMS, BLOCK>(ring, s, p, 0u, x))
                             : "memory");
            } else {
#pragma unroll
                for (uint32_t q = 0; q < (uint32_t)(W / 2); ++q)
                    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                                 : "=r"(r[4 * q]), "=r"(r[4 * q + 1]), "=r"(r[4 * q + 2]), "=r"(r[4 * q + 3])
                                 : "r"(parent_slot<W, ITEMS, BLOCK>(ring, s, p, q, x))
                                 : "memory");
            }
        }
    }
}

// Tiles [lt0, lt1) of one run with staged parents: at tile t the records of
// tile t+2 are requested, those of tile t (requested two tiles earlier) read
// back, and the draws of tile t+3 made.
template <int W, int ITEMS, int BLOCK, bool WEIGHTED>
__device__ __forceinline__ void offspring_run_staged(const SegCtx &c, uint32_t lt0, uint32_t lt1,
                                                     uint32_t *bucket_next, int tid, int lane, int warp,
                                                     const uint32_t *s_cdf, ThreadStats &ts, const LinkSmem &lk,
                                                     uint32_t &warp_alive, uint32_t ring) {
    static_assert(kParentStages == 3, "the draws rotate through three tiles");
    constexpr uint32_t TILE = (uint32_t)(BLOCK * ITEMS);
    TileDraws<ITEMS> d0, d1, d2;
    draw_parents<ITEMS, BLOCK, WEIGHTED>(c, lt0 * TILE, tid, d0);
    draw_parents<ITEMS, BLOCK, WEIGHTED>(c, (lt0 + 1) * TILE, tid, d1);  // past the run: no effect (j >= n) or unused
    draw_parents<ITEMS, BLOCK, WEIGHTED>(c, (lt0 + 2) * TILE, tid, d2);
    stage_parents<W, ITEMS, BLOCK>(c, lt0 * TILE, tid, d0, ring, 0u);
    if (lt0 + 1 < lt1) stage_parents<W, ITEMS, BLOCK>(c, (lt0 + 1) * TILE, tid, d1, ring, 1u);
    else cp_async_commit();
    cp_async_wait<2>();  // the run's tables (committed before the two parent groups)
    __syncthreads();     // ... and the cdf are visible to every thread

    uint32_t bucket_alive = 0, bucket_cur = (lt0 * TILE) / kBucket;
    uint32_t s = 0;  // ring stage of tile lt
    for (uint32_t lt = lt0; lt < lt1; ++lt) {
        const uint32_t base = lt * TILE;
        const uint32_t s2 = s >= 1u ? s - 1u : 2u;  // stage of tile lt + 2
        if (lt + 2 < lt1) stage_parents<W, ITEMS, BLOCK>(c, base + 2 * TILE, tid, d2, ring, s2);
        else cp_async_commit();
        if (tid == 0 && base % kBucket == 0u) bucket_next[base / kBucket] = 0u;
        const uint32_t bkt = base / kBucket;
        if (bkt != bucket_cur) {
            if (lane == 0 && bucket_alive) atomicAdd(&c.bucket_now[bucket_cur], bucket_alive);
            bucket_alive = 0;
            bucket_cur = bkt;
        }
        cp_async_wait<2>();  // this thread's records of tile lt have landed
        TileRecs<W, ITEMS> rec;
        read_parents<W, ITEMS, BLOCK>(ring, s, tid, rec);
        const uint32_t cnt =
            offspring_tile<W, ITEMS, BLOCK, false, WEIGHTED>(c, base, tid, lane, warp, rec, d0, s_cdf, ts, lk);
        bucket_alive += cnt;
        warp_alive += cnt;
        d0 = d1;
        d1 = d2;
        if (lt + 3 < lt1) draw_parents<ITEMS, BLOCK, WEIGHTED>(c, base + 3 * TILE, tid, d2);
        s = s == 2u ? 0u : s + 1u;
    }
    if (lane == 0 && bucket_alive) atomicAdd(&c.bucket_now[bucket_cur], bucket_alive);
}

// ----------------------------------------------------------- lane pairs
// The second launch shape for L = 128 and 256 ("words per thread"): two lanes
// per offspring.  Lane h of a pair (h = 0 mother, 1 father) draws that
// parent, loads its record (one request per sector) and forms the gamete that
// becomes the child's haplotype h; the pair shares the gamete-mask draws (each
// lane computes half the Philox blocks and hands the other lane its lanes of
// them), the genetic value (each lane sums its gamete's byte tables, and the
// dominance tables over half the heterozygous words) and the survival
// decision.  A lane holds one parent record instead of two, so twice as many
// records can be in flight per register file; the two gametes of a child are
// written by adjacent lanes as one coalesced record.
constexpr int pair_min_blocks(int block) { return block >= 512 ? 1 : 512 / block; }

template <int ITEMS>
struct PairDraws {
    uint32_t par[ITEMS], u_surv[ITEMS], u_mut[ITEMS];  // this lane's parent, the offspring's uniforms
};

template <int W, int ITEMS>
struct PairRecs {
    uint32_t r[ITEMS][2 * W];  // this lane's parent record
};

template <int ITEMS, int BLOCK>
__device__ __forceinline__ void pair_draw(const SegCtx &c, uint32_t base, int tid, uint32_t h, PairDraws<ITEMS> &d) {
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const uint32_t j = base + (uint32_t)(it * (BLOCK / 2) + (tid >> 1));
        d.par[it] = d.u_surv[it] = d.u_mut[it] = 0u;
        if (j < c.n) {
            const uint4 r = philox(make_uint4(j, c.g, c.rep, kMate << 24), c.k0, c.k1);
            uint32_t p = __umulhi(h ? r.y : r.x, c.S);
            if (c.sin) p = __ldcg(c.sin + p);
            d.par[it] = p;
            d.u_surv[it] = r.z;
            d.u_mut[it] = r.w;
        }
    }
}

template <int W, int ITEMS, int BLOCK>
__device__ __forceinline__ void pair_load(const SegCtx &c, uint32_t base, int tid, const PairDraws<ITEMS> &d,
                                          PairRecs<W, ITEMS> &rec) {
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const uint32_t j = base + (uint32_t)(it * (BLOCK / 2) + (tid >> 1));
        if (j < c.n) load_parent<W>(c.par + (size_t)d.par[it] * (2 * W), rec.r[it]);
    }
}

// The gamete-mask words of lane h's parent: the gamete stream q = 2w + h is
// lane q % 4 of Philox sub q / 4 (sub s covers words 2s and 2s+1: lanes x, y
// mother and father of word 2s, z, w of word 2s+1).  Of each pair of subs
// (2t, 2t+1) lane h computes sub 2t + h and receives its lanes of the other
// from the partner lane.  All lanes of the warp take part (shuffles).
template <int W>
__device__ __forceinline__ void pair_masks(const SegCtx &c, uint32_t j, uint32_t h, uint32_t (&m)[W]) {
    static_assert(W % 4 == 0, "lane pairs serve records of 4 or 8 words per haplotype");
#pragma unroll
    for (int t = 0; t < W / 4; ++t) {
        const uint4 d = philox(make_uint4(j, c.g, c.rep, (kRecomb << 24) | (uint32_t)(2 * t) + h), c.k0, c.k1);
        const uint32_t a = __shfl_xor_sync(0xFFFFFFFFu, h ? d.x : d.y, 1);
        const uint32_t b = __shfl_xor_sync(0xFFFFFFFFu, h ? d.z : d.w, 1);
        m[4 * t + 0] = h ? a : d.x;  // word 4t:   sub 2t, lane x (mother) / y (father)
        m[4 * t + 1] = h ? b : d.z;  // word 4t+1: sub 2t, lane z / w
        m[4 * t + 2] = h ? d.y : a;  // word 4t+2: sub 2t+1, lane x / y
        m[4 * t + 3] = h ? d.w : b;  // word 4t+3: sub 2t+1, lane z / w
    }
}

// Per-locus mutation of a pair's child (the draws of mutate(), made by both
// lanes alike): each position belongs to one haplotype, whose lane checks it
// against the positions already chosen there and flips it; the pair agrees
// on every duplicate through a shuffle, so both count the same K distinct
// positions.
template <int W>
__device__ __forceinline__ void pair_mutate(uint32_t (&g)[W], uint32_t k, uint32_t j, uint32_t gen, uint32_t rep,
                                            uint32_t k0, uint32_t k1, uint32_t h, uint32_t pair_mask) {
    constexpr uint32_t L = 32u * W;
    uint32_t seen[W];
#pragma unroll
    for (int w = 0; w < W; ++w) seen[w] = 0u;
    uint32_t chosen = 0;
    for (uint32_t a4 = 0; a4 < kMutDraws / 4 && chosen < k; ++a4) {
        const uint4 d = philox(make_uint4(j, gen, rep, (kMutPos << 24) | a4), k0, k1);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            if (chosen < k) {
                const uint32_t pos = __umulhi(lane_of(d, l), 2u * L);  // [0, 2L)
                const uint32_t owner = pos >= L ? 1u : 0u, loc = pos - owner * L;
                const uint32_t wi = loc >> 5, bit = 1u << (loc & 31u);
                bool mine_dup = false;
#pragma unroll
                for (int w = 0; w < W; ++w)
                    if ((uint32_t)w == wi) mine_dup = (seen[w] & bit) != 0u;
                const bool other_dup = __shfl_xor_sync(pair_mask, mine_dup, 1);
                const bool dup = owner == h ? mine_dup : other_dup;
                if (!dup) {
                    if (owner == h) {
#pragma unroll
                        for (int w = 0; w < W; ++w)
                            if ((uint32_t)w == wi) {
                                seen[w] |= bit;
                                g[w] ^= bit;
                            }
                    }
                    ++chosen;
                }
            }
        }
    }
}

// W words of a gamete at p (16-byte aligned for W = 4, 32-byte for W = 8).
template <int W>
__device__ __forceinline__ void store_gamete(uint32_t *__restrict__ p, const uint32_t (&g)[W]) {
    if constexpr (W == 4) {
        *reinterpret_cast<uint4 *>(p) = make_uint4(g[0], g[1], g[2], g[3]);
    } else {
        asm volatile("st.global.v8.u32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(g[0]), "r"(g[1]),
                     "r"(g[2]), "r"(g[3]), "r"(g[4]), "r"(g[5]), "r"(g[6]), "r"(g[7]));
    }
}

// One tile of a pair kernel (BLOCK / 2 * ITEMS offspring).
template <int W, int ITEMS, int BLOCK>
__device__ __forceinline__ uint32_t pair_tile(const SegCtx &c, uint32_t base, int tid, int lane, int warp,
                                              const PairRecs<W, ITEMS> &rec, const PairDraws<ITEMS> &dr,
                                              const uint32_t *s_cdf, ThreadStats &ts) {
    const uint32_t h = (uint32_t)lane & 1u, pair_mask = 3u << (lane & ~1);
    uint32_t alive_count = 0;  // the warp's survivors (same in every lane)
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const uint32_t j = base + (uint32_t)(it * (BLOCK / 2) + (tid >> 1));
        const bool live = j < c.n;
        // (B) this lane's gamete from its parent: crossover masks, mutation
        uint32_t m[W], g[W];
        pair_masks<W>(c, j, h, m);
        const uint32_t(&pr)[2 * W] = rec.r[it];
#pragma unroll
        for (int w = 0; w < W; ++w) g[w] = (pr[w] & ~m[w]) | (pr[W + w] & m[w]);
        const uint32_t u_mut = dr.u_mut[it];
        if (live && c.kmax != 0u && u_mut >= s_cdf[0]) {  // the same in both lanes of the pair
            uint32_t k = 0;
            for (uint32_t i = 0; i < c.kmax; ++i) k += (u_mut >= s_cdf[i]) ? 1u : 0u;
            pair_mutate<W>(g, k, j, c.g, c.rep, c.k0, c.k1, h, pair_mask);
        }
        if (live) store_gamete<W>(c.chi + (size_t)j * (2 * W) + h * W, g);
        // (C) genetic value: this gamete's additive value; the dominance
        // deviations and heterozygosity of half of the words
        int32_t part = 0;
        uint32_t allele = 0, hz = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            part += byte_table_word(0u, (uint32_t)w, g[w]);
            allele += __popc(g[w]);
        }
#pragma unroll
        for (int i = 0; i < W / 2; ++i) {
            const uint32_t mine = h ? g[W / 2 + i] : g[i];  // words h * W/2 + i
            const uint32_t other = __shfl_xor_sync(0xFFFFFFFFu, h ? g[i] : g[W / 2 + i], 1);
            const uint32_t x = mine ^ other;
            hz += __popc(x);
            if (c.dlut) part += byte_table_word(c.dlut, h * (W / 2) + (uint32_t)i, x);
        }
        const int32_t raw = part + __shfl_xor_sync(0xFFFFFFFFu, part, 1);
        // (D) survival: the bin's threshold scaled by the resource factor
        bool alive = false;
        if (live) {
            const long long v = (long long)raw + (long long)c.bias;
            const uint32_t bin = v < 0 ? 0u : (uint32_t)min(v >> c.shift, (long long)(kBins - 1));
            uint32_t thr = smem_u32(SmemLayout<W>::kThr + bin * 4u);
            if (c.f != kCertain) thr = __umulhi(thr, c.f);
            alive = (thr == kCertain) || (dr.u_surv[it] < thr);
            ts.het += hz;
            ts.allele += allele;
            if (h == 0u) {  // the offspring's sums once per pair
                ts.sum_raw += raw;
                ts.sum_raw2 += (unsigned long long)((long long)raw * (long long)raw);
                ts.mn = min(ts.mn, raw);
                ts.mx = max(ts.mx, raw);
                if (alive) {
                    ts.sum_raw_s += raw;
                    if (c.eco) ts.cons += smem_u32(SmemLayout<W>::kAtt + bin * 4u);
                }
            }
        }
        // (E, first half) the warp's 16 offspring: bit p of the half word is
        // pair p's decision (the even lanes of the ballot)
        uint32_t bal = __ballot_sync(0xFFFFFFFFu, alive) & 0x55555555u;
        bal = (bal | (bal >> 1)) & 0x33333333u;
        bal = (bal | (bal >> 2)) & 0x0F0F0F0Fu;
        bal = (bal | (bal >> 4)) & 0x00FF00FFu;
        bal = (bal | (bal >> 8)) & 0x0000FFFFu;
        const uint32_t j0 = base + (uint32_t)(it * (BLOCK / 2) + warp * 16);
        if (lane == 0) reinterpret_cast<uint16_t *>(c.alive)[j0 >> 4] = (uint16_t)bal;
        alive_count += __popc(bal);
    }
    return alive_count;
}

template <int W, int ITEMS, int BLOCK>
__device__ __forceinline__ void pair_run(const SegCtx &c, uint32_t lt0, uint32_t lt1, uint32_t *bucket_next, int tid,
                                         int lane, int warp, const uint32_t *s_cdf, ThreadStats &ts,
                                         uint32_t &warp_alive) {
    constexpr uint32_t TILE = (uint32_t)(BLOCK / 2 * ITEMS);
    const uint32_t h = (uint32_t)lane & 1u;
    PairDraws<ITEMS> d0, d1;
    PairRecs<W, ITEMS> ra, rb;
    pair_draw<ITEMS, BLOCK>(c, lt0 * TILE, tid, h, d0);
    if (lt0 + 1 < lt1) pair_draw<ITEMS, BLOCK>(c, (lt0 + 1) * TILE, tid, h, d1);
    pair_load<W, ITEMS, BLOCK>(c, lt0 * TILE, tid, d0, ra);
    cp_async_wait<0>();
    __syncthreads();  // the run's tables (and cdf) are visible to every thread

    uint32_t bucket_alive = 0, bucket_cur = (lt0 * TILE) / kBucket;
    auto step = [&](uint32_t lt, const PairRecs<W, ITEMS> &cur, PairRecs<W, ITEMS> &nxt) {
        const uint32_t base = lt * TILE;
        if (lt + 1 < lt1) pair_load<W, ITEMS, BLOCK>(c, base + TILE, tid, d1, nxt);
        if (tid == 0 && base % kBucket == 0u) bucket_next[base / kBucket] = 0u;
        const uint32_t bkt = base / kBucket;
        if (bkt != bucket_cur) {
            if (lane == 0 && bucket_alive) atomicAdd(&c.bucket_now[bucket_cur], bucket_alive);
            bucket_alive = 0;
            bucket_cur = bkt;
        }
        PairDraws<ITEMS> d2;  // drawn before the tile is formed (see offspring_run)
        pair_draw<ITEMS, BLOCK>(c, base + 2 * TILE, tid, h, d2);  // past the run: unused
        const uint32_t cnt = pair_tile<W, ITEMS, BLOCK>(c, base, tid, lane, warp, cur, d0, s_cdf, ts);
        bucket_alive += cnt;
        warp_alive += cnt;
        d0 = d1;
        d1 = d2;
    };
    for (uint32_t lt = lt0; lt < lt1; lt += 2) {
        step(lt, ra, rb);
        if (lt + 1 < lt1) step(lt + 1, rb, ra);
    }
    if (lane == 0 && bucket_alive) atomicAdd(&c.bucket_now[bucket_cur], bucket_alive);
}

template <int W, int ITEMS, int BLOCK, bool LINKED, bool WEIGHTED, bool PAIR, bool STAGED>
__global__ void __launch_bounds__(BLOCK, PAIR ? pair_min_blocks(BLOCK) : offspring_min_blocks(BLOCK))
    k_offspring(const __grid_constant__ GenArgs a) {
    static_assert(!STAGED || (W <= 4 && !LINKED && !PAIR), "staged parents: single-lane kernels without linkage");
    constexpr int NW = BLOCK / 32;
    constexpr uint32_t TILE = (uint32_t)(BLOCK * ITEMS) / (PAIR ? 2u : 1u);
    static_assert(kBucket % TILE == 0, "tiles must not straddle compaction buckets");
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
    __shared__ uint32_t s_ltog[LK * NW * 2 * 32 * (W + 3) + 1];
    LinkSmem lk{s_lcdf, s_lcum, s_lchrom, s_lfirst, s_lclast, s_lguide, 0u, 0u, s_ltog};

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t dyn_addr = (uint32_t)__cvta_generic_to_shared(s_dyn);

    uint32_t r = 0, r_end = 1;
    if (a.nsegs != 1u) {
        r = __ldg(a.block_runs + blockIdx.x);
        r_end = __ldg(a.block_runs + blockIdx.x + 1u);
    }
    bool first = true;  // the first run's tables are copied while the previous kernel finishes
    for (; r < r_end; ++r) {
        uint32_t lt0, lt1;
        const Segment *sgp;
        if (a.nsegs == 1u) {
            const uint32_t T = a.total_tiles, G = gridDim.x;
            lt0 = (uint32_t)(((unsigned long long)T * blockIdx.x) / G);
            lt1 = (uint32_t)(((unsigned long long)T * (blockIdx.x + 1)) / G);
            sgp = &a.one;
        } else {
            const Run run = a.runs[r];
            sgp = a.segs + run.seg;
            lt0 = run.tile0;
            lt1 = run.tile0 + run.count;
        }
        if (lt0 >= lt1) continue;
        const Segment &sg = *sgp;
        // the run's tables (parameters only: nothing the previous kernel writes)
        const PopParams *P = sg.prm;
        const uint32_t dlut = P->has_dom ? a.smem_dlut : 0u;  // 0 also when the launch has no dominance tables
        cp_async_wait<0>();  // a skipped run's copies have landed
        __syncthreads();     // the previous run's tables and statistics scratch are no longer read
        copy_tables<W, BLOCK>(P, a.eco_table != 0u, P->has_eco != 0u, dyn_addr, a.smem_dlut, dlut != 0u, tid);
        if (tid < kMaxKmax) s_cdf[tid] = (uint32_t)tid < P->kmax ? P->cdf[tid] : 0u;
        if constexpr (LINKED) {
            const LinkParams *lp = P->link;
            lk.kmax = lp->kmax;
            lk.nchrom = lp->nchrom;
            for (uint32_t i = tid; i < 32u * W; i += BLOCK) {
                s_lcum[i] = lp->cum[i];
                s_lchrom[i] = lp->chrom[i];
            }
            if (tid < kMaxKmax) s_lcdf[tid] = lp->cdf[tid];
            for (uint32_t i = tid; i < (uint32_t)kLinkGuide; i += BLOCK) s_lguide[i] = lp->guide[i];
            if (tid < kMaxChrom) {
                s_lfirst[tid] = lp->first[tid];
                s_lclast[tid] = lp->clast[tid];
            }
        }
        if (first) {  // from here on: the previous kernel's state, records and counters
            griddep_wait();
            first = false;
            if (a.nsegs != 1u && sg.dense) {  // the first run's parents: this block's share of them, now
                const Run run = a.runs[r];
                prefetch_parents<W, BLOCK>(sg.dense, (uint32_t)(((unsigned long long)sg.n * run.share) / run.shares),
                                           (uint32_t)(((unsigned long long)sg.n * (run.share + 1u)) / run.shares), tid);
            }
        }
        if (a.nsegs != 1u && r + 1u < r_end) {  // the next run's parents into L2 while this run is formed
            const Run nx = a.runs[r + 1u];
            const Segment &sn = a.segs[nx.seg];
            if (sn.dense)
                prefetch_parents<W, BLOCK>(sn.dense, (uint32_t)(((unsigned long long)sn.n * nx.share) / nx.shares),
                                           (uint32_t)(((unsigned long long)sn.n * (nx.share + 1u)) / nx.shares), tid);
        }
        const PopNow now = read_state(sg.state);
        if (!now.active) continue;
        SegCtx c;
        c.P = P;
        c.n = sg.n;
        c.S = min(now.S, sg.n);  // parent ranks stay inside the buffers whatever the state holds
        c.f = now.f;
        c.g = now.gen + 1u;
        c.sin = sg.dense ? nullptr : sg.surv[now.gen & 1u];
        c.par = sg.dense ? sg.dense : sg.geno[now.gen & 1u];
        c.chi = sg.geno[(now.gen + 1u) & 1u];
        c.alive = sg.alive;
        c.survw = sg.survw;
        c.obin = sg.obin;
        c.bucket_now = sg.bucket_sum + (c.g & 1u) * sg.nbuckets;
        uint32_t *bucket_next = sg.bucket_sum + ((c.g + 1u) & 1u) * sg.nbuckets;
        c.rep = c.P->rep;
        c.k0 = c.P->key0;
        c.k1 = c.P->key1;
        c.kmax = c.P->kmax;
        c.shift = c.P->shift;
        c.bias = c.P->bias;
        c.eco = a.eco_table != 0u;
        c.dlut = dlut;

        ThreadStats ts;
        uint32_t warp_alive = 0;
        if constexpr (PAIR)
            pair_run<W, ITEMS, BLOCK>(c, lt0, lt1, bucket_next, tid, lane, warp, s_cdf, ts, warp_alive);
        else if constexpr (STAGED)
            offspring_run_staged<W, ITEMS, BLOCK, WEIGHTED>(c, lt0, lt1, bucket_next, tid, lane, warp, s_cdf, ts, lk,
                                                            warp_alive,
                                                  dyn_addr + a.smem_parents);
        else
            offspring_run<W, ITEMS, BLOCK, LINKED, WEIGHTED>(c, lt0, lt1, bucket_next, tid, lane, warp, s_cdf, ts, lk,
                                                             warp_alive);

        // statistics of this run: exact warp sums, one atomic per field into
        // one of the population's accumulator copies
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
    // the compaction's blocks are launched once every block of this grid is
    // here (released at entry instead, they took SM resources from this
    // grid's tail: 5% slower generations)
    griddep_release();
}

// Host-side description of one instance: entry and shape.
template <int W, int ITEMS, int BLOCK, bool LINKED = false, bool WEIGHTED = false, bool PAIR = false,
          bool STAGED = false>
OffspringKernel offspring_instance() {
    OffspringKernel k;
    k.fn = &k_offspring<W, ITEMS, BLOCK, LINKED, WEIGHTED, PAIR, STAGED>;
    k.block = BLOCK;
    k.items = ITEMS;
    k.lanes = PAIR ? 2u : 1u;
    return k;
}

}  // namespace
}  // namespace spg
