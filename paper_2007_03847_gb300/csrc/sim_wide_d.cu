// Instantiations of the four-warps-per-sample fused kernel: 10 and 13 machine slots per thread.
#include "simulate_wide.cuh"

namespace fmc {

cudaError_t launch_wide_nmt10(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_wide_t<10, 1>(maps, a, st, occ);
        case 2: return launch_wide_t<10, 2>(maps, a, st, occ);
        case 4: return launch_wide_t<10, 4>(maps, a, st, occ);
        case 8: return launch_wide_t<10, 8>(maps, a, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_wide_nmt13(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_wide_t<13, 1>(maps, a, st, occ);
        case 2: return launch_wide_t<13, 2>(maps, a, st, occ);
        case 4: return launch_wide_t<13, 4>(maps, a, st, occ);
        case 8: return launch_wide_t<13, 8>(maps, a, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fmc
