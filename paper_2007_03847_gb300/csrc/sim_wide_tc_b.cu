// Instantiations of the four-warps-per-sample fused kernel with the network sums
// on the tensor cores: 10 and 13 machine slots per thread.
#include "simulate_wide.cuh"

namespace fmc {

#define FMC_WIDE_TC_ND(NMT)                                                    \
    switch (nd) {                                                              \
        case 1: return launch_wide_t<NMT, 1, true>(maps, a, st, occ);          \
        case 2: return launch_wide_t<NMT, 2, true>(maps, a, st, occ);          \
        case 4: return launch_wide_t<NMT, 4, true>(maps, a, st, occ);          \
        case 8: return launch_wide_t<NMT, 8, true>(maps, a, st, occ);          \
        default: return cudaErrorInvalidValue;                                 \
    }

cudaError_t wide_tc_nmt10(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    FMC_WIDE_TC_ND(10)
}

cudaError_t wide_tc_nmt13(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    FMC_WIDE_TC_ND(13)
}

}  // namespace fmc
