// Instantiations of the four-warps-per-sample fused kernel: 5 and 7 machine slots per thread.
#include "simulate_wide.cuh"

namespace fmc {

cudaError_t launch_wide_nmt5(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_wide_t<5, 1>(maps, a, st, occ);
        case 2: return launch_wide_t<5, 2>(maps, a, st, occ);
        case 4: return launch_wide_t<5, 4>(maps, a, st, occ);
        case 8: return launch_wide_t<5, 8>(maps, a, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_wide_nmt7(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_wide_t<7, 1>(maps, a, st, occ);
        case 2: return launch_wide_t<7, 2>(maps, a, st, occ);
        case 4: return launch_wide_t<7, 4>(maps, a, st, occ);
        case 8: return launch_wide_t<7, 8>(maps, a, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fmc
