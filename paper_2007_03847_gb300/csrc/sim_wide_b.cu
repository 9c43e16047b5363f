// Instantiations of the four-warps-per-sample fused kernel: 3 and 4 machine slots per thread.
#include "simulate_wide.cuh"

namespace fmc {

cudaError_t launch_wide_nmt3(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_wide_t<3, 1>(maps, a, st, occ);
        case 2: return launch_wide_t<3, 2>(maps, a, st, occ);
        case 4: return launch_wide_t<3, 4>(maps, a, st, occ);
        case 8: return launch_wide_t<3, 8>(maps, a, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_wide_nmt4(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_wide_t<4, 1>(maps, a, st, occ);
        case 2: return launch_wide_t<4, 2>(maps, a, st, occ);
        case 4: return launch_wide_t<4, 4>(maps, a, st, occ);
        case 8: return launch_wide_t<4, 8>(maps, a, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fmc
