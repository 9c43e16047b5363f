// Instantiations of the tensor-core split kernel with two warps per sample (two
// 256-thread CTAs per SM): 9 machine slots per thread (17..18 machines), 11
// (21..22) and 12 (23..24), up to 7 disturbances; 14 (27..28), up to 4.
#include "simulate_wide.cuh"

namespace fmc {

cudaError_t wide_tc_h2_nmt9(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_wide_t<9, 1, true, 2>(maps, a, st, occ);
        case 2: return launch_wide_t<9, 2, true, 2>(maps, a, st, occ);
        case 4: return launch_wide_t<9, 4, true, 2>(maps, a, st, occ);
        case 8: return launch_wide_t<9, 8, true, 2>(maps, a, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t wide_tc_h2_nmt11(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_wide_t<11, 1, true, 2>(maps, a, st, occ);
        case 2: return launch_wide_t<11, 2, true, 2>(maps, a, st, occ);
        case 4: return launch_wide_t<11, 4, true, 2>(maps, a, st, occ);
        case 8: return launch_wide_t<11, 8, true, 2>(maps, a, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t wide_tc_h2_nmt12(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_wide_t<12, 1, true, 2>(maps, a, st, occ);
        case 2: return launch_wide_t<12, 2, true, 2>(maps, a, st, occ);
        case 4: return launch_wide_t<12, 4, true, 2>(maps, a, st, occ);
        case 8: return launch_wide_t<12, 8, true, 2>(maps, a, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t wide_tc_h2_nmt14(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_wide_t<14, 1, true, 2>(maps, a, st, occ);
        case 2: return launch_wide_t<14, 2, true, 2>(maps, a, st, occ);
        case 4: return launch_wide_t<14, 4, true, 2>(maps, a, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fmc
