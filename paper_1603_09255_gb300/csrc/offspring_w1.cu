// Offspring kernel instances for L = 32 loci (W = 1 word per haplotype):
// every supported launch shape of the plain kernel, with parents in registers or staged through shared memory,
// and the linkage-map and weighted-parent variants (256 threads, one
// offspring each).
#include "offspring.cuh"

namespace spg {

OffspringKernel offspring_kernel_w1(const Shape &s, bool linked, bool weighted, bool staged) {
    if (linked || weighted) {
        if (s.block != 256 || s.items != 1 || s.lanes != 1) return OffspringKernel{};
        if (linked && weighted) return offspring_instance<1, 1, 256, true, true>();
        if (linked) return offspring_instance<1, 1, 256, true, false>();
        return staged ? offspring_instance<1, 1, 256, false, true, false, true>()
                      : offspring_instance<1, 1, 256, false, true>();
    }
    if (s.block == 128 && s.items == 1 && s.lanes == 1)
        return staged ? offspring_instance<1, 1, 128, false, false, false, true>()
                      : offspring_instance<1, 1, 128, false, false, false, false>();
    if (s.block == 128 && s.items == 2 && s.lanes == 1)
        return staged ? offspring_instance<1, 2, 128, false, false, false, true>()
                      : offspring_instance<1, 2, 128, false, false, false, false>();
    if (s.block == 256 && s.items == 1 && s.lanes == 1)
        return staged ? offspring_instance<1, 1, 256, false, false, false, true>()
                      : offspring_instance<1, 1, 256, false, false, false, false>();
    if (s.block == 256 && s.items == 2 && s.lanes == 1)
        return staged ? offspring_instance<1, 2, 256, false, false, false, true>()
                      : offspring_instance<1, 2, 256, false, false, false, false>();
    if (s.block == 512 && s.items == 1 && s.lanes == 1)
        return staged ? offspring_instance<1, 1, 512, false, false, false, true>()
                      : offspring_instance<1, 1, 512, false, false, false, false>();
    if (s.block == 512 && s.items == 2 && s.lanes == 1)
        return staged ? offspring_instance<1, 2, 512, false, false, false, true>()
                      : offspring_instance<1, 2, 512, false, false, false, false>();
    return OffspringKernel{};
}

}  // namespace spg
