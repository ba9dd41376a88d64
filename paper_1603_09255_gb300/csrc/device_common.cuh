// Device helpers shared by the generation kernels of libspegg_gb300
// (sm_103a): the counter-based Philox generator, packed record access,
// per-locus mutation, linkage-map gamete masks, exact warp sums, population
// state reads and asynchronous global-to-shared copies.  Included by every
// translation unit that defines generation kernels; internal linkage.
#pragma once

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
        // each 32 x 32 -> 64-bit product as one wide multiply (both halves)
        const unsigned long long p0 = (unsigned long long)A * c.x, p1 = (unsigned long long)B * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
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

// Records of 32 bytes or more are written with 256-bit stores: one request
// per whole sector (two 128-bit stores per sector would each touch the
// sector half-written).  Nothing in a generation kernel reads the records it
// writes, so the stores need no ordering against other memory operations.
template <int W>
__device__ __forceinline__ void store_record(uint32_t *__restrict__ p, const uint32_t (&r)[2 * W]) {
    if constexpr (W == 1) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(r[0], r[1]);
    } else if constexpr (W == 2) {
        *reinterpret_cast<uint4 *>(p) = make_uint4(r[0], r[1], r[2], r[3]);
    } else {
#pragma unroll
        for (int q = 0; q < W / 4; ++q)
            asm volatile("st.global.v8.u32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p + 8 * q), "r"(r[8 * q]),
                         "r"(r[8 * q + 1]), "r"(r[8 * q + 2]), "r"(r[8 * q + 3]), "r"(r[8 * q + 4]),
                         "r"(r[8 * q + 5]), "r"(r[8 * q + 6]), "r"(r[8 * q + 7]));
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
    uint32_t *tog;  // warp-cooperative crossovers: per warp, gamete and lane, W toggle words + 3 parity words
};

template <int W>
__device__ __forceinline__ void toggle_bit(uint32_t (&t)[W], uint32_t pos) {
#pragma unroll
    for (int w = 0; w < W; ++w)
        if ((uint32_t)w == (pos >> 5)) t[w] ^= 1u << (pos & 31u);
}

// Origin masks of both gametes of a warp's 32 offspring under the linkage
// map (bit set: the locus comes from the parent's haplotype 1); all lanes
// take part, valid = false gives a lane no crossovers.  Every chromosome
// whose coin is 1 and every crossover flips the loci from its start to the
// chromosome's end.  Each flip is two toggles (at the first flipped locus and
// one past the last); a crossover toggles its start and flips its
// chromosome's parity bit, and the end toggles, which cancel in pairs, are
// applied once per chromosome whose coin and parity differ.  A prefix XOR
// over the L bits turns the toggles into the mask.  The crossovers are dealt
// to the warp's lanes one Philox block (up to four crossovers of one gamete)
// at a time instead of each lane looping over its own, which would run the
// warp to its lanes' largest count; a crossover's toggle and parity flip go
// to the owner's words in shared memory by atomic XOR (flips commute, so the
// order does not matter), and each lane then finishes its own two masks.
template <int W>
__device__ __forceinline__ void linked_masks_warp(const LinkSmem &lk, uint32_t j, bool valid, uint32_t g, uint32_t rep,
                                                  uint32_t k0, uint32_t k1, uint32_t (&mm)[W], uint32_t (&mf)[W]) {
    constexpr uint32_t L = 32u * W, NWD = (uint32_t)W + 3u;  // words per gamete: toggles, parity
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t *tog = lk.tog + warp * (2u * 32u * NWD);        // [gamete][lane][NWD]
    uint4 d0[2];
    uint32_t K[2];
#pragma unroll
    for (uint32_t pi = 0; pi < 2u; ++pi) {
        d0[pi] = philox(make_uint4(j, g, rep, (kLink << 24) | (pi << 8)), k0, k1);
        uint32_t k = 0;
        if (valid && lk.kmax != 0u && d0[pi].x >= lk.cdf[0]) {
            k = 1u;
#pragma unroll
            for (uint32_t step = 16u; step > 0u; step >>= 1)
                if (k + step <= lk.kmax && lk.cdf[k + step - 1u] <= d0[pi].x) k += step;
        }
        K[pi] = k;
#pragma unroll
        for (uint32_t w = 0; w < NWD; ++w) tog[(pi * 32u + lane) * NWD + w] = 0u;
    }
    // this lane's Philox blocks of crossovers, both gametes, and the warp's offsets
    const uint32_t nb0 = (K[0] + 3u) >> 2, nb = nb0 + ((K[1] + 3u) >> 2);
    uint32_t off = nb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, off, o);
        if ((int)lane >= o) off += y;
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, off, 31);
    off -= nb;  // exclusive
    __syncwarp();
    for (uint32_t f0 = 0; f0 < total; f0 += 32u) {
        const uint32_t f = f0 + lane;
        uint32_t o = 0;  // the owner: the last lane whose offset is <= f
#pragma unroll
        for (uint32_t step = 16u; step > 0u; step >>= 1) {
            const uint32_t v = __shfl_sync(0xFFFFFFFFu, off, (int)(o + step));
            if (v <= f) o += step;
        }
        const uint32_t oj = __shfl_sync(0xFFFFFFFFu, j, (int)o), ooff = __shfl_sync(0xFFFFFFFFu, off, (int)o);
        const uint32_t onb0 = __shfl_sync(0xFFFFFFFFu, nb0, (int)o);
        const uint32_t oK0 = __shfl_sync(0xFFFFFFFFu, K[0], (int)o), oK1 = __shfl_sync(0xFFFFFFFFu, K[1], (int)o);
        if (f < total) {
            const uint32_t b = f - ooff, pi = b < onb0 ? 0u : 1u, blk = pi ? b - onb0 : b, Kp = pi ? oK1 : oK0;
            const uint4 d = philox(make_uint4(oj, g, rep, (kLink << 24) | (pi << 8) | (1u + blk)), k0, k1);
            uint32_t *ot = tog + (pi * 32u + o) * NWD;
#pragma unroll
            for (uint32_t l = 0; l < 4u; ++l) {
                if (4u * blk + l < Kp) {
                    const uint32_t u = lane_of(d, (int)l);
                    const uint32_t ge = lk.guide[u >> (32 - kLinkGuideBits)], nbd = ge >> 26;
                    uint32_t I = ge & 0xFFu, ch = (ge >> 8) & 0x7Fu;
                    if (nbd == 1u) {
                        if (lk.cum[I] <= u) {
                            ++I;
                            ch = (ge >> 15) & 0x7Fu;
                        }
                    } else if (nbd > 1u) {
                        while (I + 1u < L && lk.cum[I] <= u) ++I;
                        ch = lk.chrom[I];
                    }
                    atomicXor(ot + (I >> 5), 1u << (I & 31u));
                    atomicXor(ot + W + (ch >> 5), 1u << (ch & 31u));
                }
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (uint32_t pi = 0; pi < 2u; ++pi) {
        const uint32_t *mt = tog + (pi * 32u + lane) * NWD;
        uint32_t t[W];
#pragma unroll
        for (int w = 0; w < W; ++w) t[w] = mt[w];
        const uint32_t par0 = mt[W], par1 = mt[W + 1], par2 = mt[W + 2];
        const uint4 dd = d0[pi];
        for (uint32_t c = 0; c < lk.nchrom; ++c) {
            const uint32_t coin = ((c < 32u ? dd.y : c < 64u ? dd.z : dd.w) >> (c & 31u)) & 1u;
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
            if (pi == 0u) mm[w] = x;
            else mf[w] = x;
            carry = x >> 31;
        }
    }
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

// ------------------------------------- bulk copies and shared barriers
// mbarrier objects (8 bytes of shared memory each) completing when their
// arrivals and expected bytes are in; bulk asynchronous copies (the non-tensor
// TMA path) from global to shared memory completing on one of them.  Every
// wait is bounded.
constexpr uint32_t kMbarTries = 1u << 22;  // try_wait calls before a wait gives up

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// Make initialised barriers visible to the asynchronous (bulk copy) proxy.
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Whether the phase of parity `parity` completed within kMbarTries tries.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < kMbarTries; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
// One thread: `bytes` (a multiple of 16; both addresses 16-byte aligned) from
// global src to shared dst, completing the current phase of barrier bar
// (count 1) once they have landed.  Shared memory that generic loads read
// before is ordered ahead of the copy by the proxy fence.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// ------------------------------------------- programmatic dependent launch
// The generation kernels are launched so that a kernel may start while its
// predecessor in the stream finishes.  griddep_wait() returns once the
// predecessor grid has completed and its memory is visible: every read of a
// predecessor's results comes after it.  griddep_release() lets the next
// kernel's blocks be scheduled as this grid's blocks leave the SMs.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

}  // namespace
}  // namespace spg
