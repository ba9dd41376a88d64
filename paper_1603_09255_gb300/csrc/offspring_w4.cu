// Offspring kernel instances for L = 128 loci (W = 4 words per haplotype):
// every supported launch shape of the plain kernel, with parents in registers or staged through shared memory,
// and the linkage-map and weighted-parent variants (256 threads, one
// offspring each).
#include "offspring.cuh"

namespace spg {

OffspringKernel offspring_kernel_w4(const Shape &s, bool linked, bool weighted, bool staged) {
    if (linked || weighted) {
        if (s.block != 256 || s.items != 1 || s.lanes != 1) return OffspringKernel{};
        if (linked && weighted) return offspring_instance<4, 1, 256, true, true>();
        if (linked) return offspring_instance<4, 1, 256, true, false>();
        return staged ? offspring_instance<4, 1, 256, false, true, false, true>()
                      : offspring_instance<4, 1, 256, false, true>();
    }
    if (s.block == 128 && s.items == 1 && s.lanes == 1)
        return staged ? offspring_instance<4, 1, 128, false, false, false, true>()
                      : offspring_instance<4, 1, 128, false, false, false, false>();
    if (s.block == 256 && s.items == 1 && s.lanes == 1)
        return staged ? offspring_instance<4, 1, 256, false, false, false, true>()
                      : offspring_instance<4, 1, 256, false, false, false, false>();
    if (s.block == 512 && s.items == 1 && s.lanes == 1)
        return staged ? offspring_instance<4, 1, 512, false, false, false, true>()
                      : offspring_instance<4, 1, 512, false, false, false, false>();
    if (s.block == 128 && s.items == 1 && s.lanes == 2) return offspring_instance<4, 1, 128, false, false, true>();
    if (s.block == 256 && s.items == 1 && s.lanes == 2) return offspring_instance<4, 1, 256, false, false, true>();
    if (s.block == 512 && s.items == 1 && s.lanes == 2) return offspring_instance<4, 1, 512, false, false, true>();
    return OffspringKernel{};
}

}  // namespace spg
