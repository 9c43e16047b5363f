// Instantiations of the four-warps-per-sample fused kernel: 1 and 2 machine slots per thread.
#include "simulate_wide.cuh"

namespace fmc {

cudaError_t launch_wide_nmt1(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_wide_t<1, 1>(maps, a, st, occ);
        case 2: return launch_wide_t<1, 2>(maps, a, st, occ);
        case 4: return launch_wide_t<1, 4>(maps, a, st, occ);
        case 8: return launch_wide_t<1, 8>(maps, a, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_wide_nmt2(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_wide_t<2, 1>(maps, a, st, occ);
        case 2: return launch_wide_t<2, 2>(maps, a, st, occ);
        case 4: return launch_wide_t<2, 4>(maps, a, st, occ);
        case 8: return launch_wide_t<2, 8>(maps, a, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fmc
