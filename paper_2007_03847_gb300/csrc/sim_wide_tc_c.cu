// Instantiations of the tensor-core split kernel with two warps per sample (two
// 256-thread CTAs per SM): 10 machine slots per thread (17..20 machines) and 13
// (21..26 machines, up to 4 disturbances).
#include "simulate_wide.cuh"

namespace fmc {

cudaError_t wide_tc_h2_nmt10(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_wide_t<10, 1, true, 2>(maps, a, st, occ);
        case 2: return launch_wide_t<10, 2, true, 2>(maps, a, st, occ);
        case 4: return launch_wide_t<10, 4, true, 2>(maps, a, st, occ);
        case 8: return launch_wide_t<10, 8, true, 2>(maps, a, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t wide_tc_h2_nmt13(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_wide_t<13, 1, true, 2>(maps, a, st, occ);
        case 2: return launch_wide_t<13, 2, true, 2>(maps, a, st, occ);
        case 4: return launch_wide_t<13, 4, true, 2>(maps, a, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fmc
