// spg_generation_noalloc: one generation of one population on buffers the
// caller owns, with every piece of working memory taken from a fixed array
// in this file, so the call performs no device allocation at all.
//
// The working memory (parameters, state, statistics accumulators, alive
// bitmap, per-bucket survivor counts) lives in the file-scope array
// g_noalloc_scratch below.  Host code cannot use the array's name as a device
// address, so its address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "spegg.h"
#include "spegg_engine.h"
#include "spegg_internal.h"

namespace spg {
namespace {

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

constexpr uint32_t kMaxBuckets = SPG_NOALLOC_MAX_N / kBucket;
constexpr size_t kOffParams = 0;
constexpr size_t kOffState = kOffParams + align256(sizeof(PopParams));
constexpr size_t kOffAcc = kOffState + align256(sizeof(DevState));
constexpr size_t kOffAlive = kOffAcc + align256(sizeof(StatAcc) * kAccCopies);
constexpr size_t kOffBuckets = kOffAlive + align256((size_t)kMaxBuckets * kBucketWords * 4);
constexpr size_t kScratchBytes = kOffBuckets + align256((size_t)2 * kMaxBuckets * 4);
static_assert(SPG_NOALLOC_MAX_N % kBucket == 0, "the maximum population must be a whole number of buckets");
static_assert(kScratchBytes == SPG_NOALLOC_SCRATCH_BYTES, "spegg.h states the scratch size");

// Shared by every call on a device; it keeps the previous call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on
// the first call made with that device current).
int scratch_address(char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(SPG_ERR_INVALID, "device ordinal %d is not supported", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<char *>(g_scratch_addr[dev]);
    return SPG_OK;
}

}  // namespace
}  // namespace spg

using namespace spg;

extern "C" int spg_generation_noalloc(const spg_noalloc_generation *a, void *stream) {
    if (!a) return fail(SPG_ERR_INVALID, "arguments are NULL");
    if (a->n == 0 || a->n > SPG_NOALLOC_MAX_N)
        return fail(SPG_ERR_INVALID, "n must be in [1, %u] for the allocation-free call (got %u)",
                    (unsigned)SPG_NOALLOC_MAX_N, a->n);
    if (!(a->n_loci == 32 || a->n_loci == 64 || a->n_loci == 128 || a->n_loci == 256))
        return fail(SPG_ERR_INVALID, "n_loci must be 32, 64, 128 or 256 (got %u)", a->n_loci);
    if (a->generation == 0) return fail(SPG_ERR_INVALID, "generation must be >= 1");
    if (a->S == 0 || a->S > a->n) return fail(SPG_ERR_INVALID, "S must be in [1, n] (got %u)", a->S);
    if (!a->effects || !a->surv_table) return fail(SPG_ERR_INVALID, "effects and surv_table are required");
    if (!a->parents || !a->survivors || !a->children || !a->survivors_out || !a->stats)
        return fail(SPG_ERR_INVALID, "device buffers are required");
    if (a->bin_shift > 31) return fail(SPG_ERR_INVALID, "bin_shift must be <= 31");
    if (!(a->mu >= 0.0 && a->mu < 1.0)) return fail(SPG_ERR_INVALID, "mu must be in [0, 1)");

    char *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != SPG_OK) return rc;

    const uint32_t W = a->n_loci / 32, g = a->generation;
    const Shape shape = default_shape(W);
    spg_pop_desc d{};
    d.n = a->n;
    d.n_loci = a->n_loci;
    d.seed = a->seed;
    d.replicate = a->replicate;
    d.effects = a->effects;
    d.surv_table = a->surv_table;
    d.bin_bias = a->bin_bias;
    d.bin_shift = a->bin_shift;
    d.mu = a->mu;
    d.stats_capacity = 1;
    // host staging of the parameters without a per-call host allocation
    static thread_local PopParams prm;
    rc = build_params(&d, prm);
    if (rc != SPG_OK) return rc;
    prm.stats_cap = 1;  // the caller's single statistics record
    prm.has_eco = 0;

    OffspringKernel k = offspring_kernel(W, shape, false, false, false, false, false);
    rc = prepare_offspring(k);
    if (rc != SPG_OK) return fail(rc, "offspring kernel setup failed");
    const uint32_t ntiles = tiles_for(a->n, shape), nbuckets = bucket_count(a->n);

    Segment seg{};
    seg.prm = reinterpret_cast<const PopParams *>(scratch + kOffParams);
    // the kernels pick buffers by the parity of the generation they form
    seg.geno[(g - 1u) & 1u] = const_cast<uint32_t *>(a->parents);
    seg.geno[g & 1u] = a->children;
    seg.surv[(g - 1u) & 1u] = const_cast<uint32_t *>(a->survivors);
    seg.surv[g & 1u] = a->survivors_out;
    seg.alive = reinterpret_cast<uint32_t *>(scratch + kOffAlive);
    seg.bucket_sum = reinterpret_cast<uint32_t *>(scratch + kOffBuckets);
    seg.state = reinterpret_cast<DevState *>(scratch + kOffState);
    seg.acc = reinterpret_cast<StatAcc *>(scratch + kOffAcc);
    seg.ring = a->stats;
    seg.n = a->n;
    seg.tile_begin = 0;
    seg.ntiles = ntiles;
    seg.bucket_begin = 0;
    seg.nbuckets = nbuckets;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // pageable source: the copy is staged before the call returns
    cudaError_t e = cudaMemcpyAsync(scratch + kOffParams, &prm, sizeof prm, cudaMemcpyHostToDevice, s);
    // the per-bucket counts must start at zero; the rest is overwritten
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch + kOffBuckets, 0, (size_t)2 * nbuckets * 4, s);
    if (e != cudaSuccess) return cuda_fail(e, "stage allocation-free generation");
    rc = launch_set_state(reinterpret_cast<DevState *>(scratch + kOffState),
                          reinterpret_cast<StatAcc *>(scratch + kOffAcc), g - 1u, a->S, a->f, 0.0, SPG_OK,
                          0xFFFFFFFFu, s);
    if (rc != SPG_OK) return fail(rc, "reset allocation-free state");

    GenLaunch gl;
    gl.offspring = k;
    gl.compact = compact_kernel(W);  // no dense buffer: parents by survivor index, no record copies
    gl.args.segs = nullptr;  // one segment: the kernels read it from their parameters
    gl.args.nsegs = 1;
    gl.args.one = seg;
    gl.args.total_tiles = ntiles;
    gl.args.total_buckets = nbuckets;
    apply_kernel(k, gl.args);
    gl.blocks = std::min(ntiles, k.resident);
    gl.buckets = nbuckets;
    return launch_generation(gl, s);
}
