// Instantiations of the tensor-core split kernel for systems with an infinite
// bus (held in the last machine slot): four warps per sample, the 8-disturbance
// bucket, every slot count.
#include "simulate_wide.cuh"

namespace fmc {

cudaError_t wide_tc_bus(int nmt, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    switch (nmt) {
        case 4: return launch_wide_t<4, 8, true, 4, true>(maps, a, st, occ);
        case 5: return launch_wide_t<5, 8, true, 4, true>(maps, a, st, occ);
        case 7: return launch_wide_t<7, 8, true, 4, true>(maps, a, st, occ);
        case 10: return launch_wide_t<10, 8, true, 4, true>(maps, a, st, occ);
        case 13: return launch_wide_t<13, 8, true, 4, true>(maps, a, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fmc
