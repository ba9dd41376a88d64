// Offspring kernel instances for L = 64 loci (W = 2 words per haplotype):
// every supported launch shape of the plain kernel, and the linkage-map and
// weighted-parent variants (256 threads, one offspring each).
#include "offspring.cuh"

namespace spg {

OffspringKernel offspring_kernel_w2(uint32_t block, uint32_t items, bool linked, bool weighted) {
    if (linked || weighted) {
        if (block != 256 || items != 1) return OffspringKernel{};
        if (linked && weighted) return offspring_instance<2, 1, 256, true, true>();
        return linked ? offspring_instance<2, 1, 256, true, false>() : offspring_instance<2, 1, 256, false, true>();
    }
    if (block == 128 && items == 1) return offspring_instance<2, 1, 128>();
    if (block == 128 && items == 2) return offspring_instance<2, 2, 128>();
    if (block == 256 && items == 1) return offspring_instance<2, 1, 256>();
    if (block == 256 && items == 2) return offspring_instance<2, 2, 256>();
    if (block == 512 && items == 1) return offspring_instance<2, 1, 512>();
    if (block == 512 && items == 2) return offspring_instance<2, 2, 512>();
    return OffspringKernel{};
}

}  // namespace spg
