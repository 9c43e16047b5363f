// Instantiations of the fused kernel in its SM-owning form (up to 14 warps per
// CTA, one CTA per SM) for 4 machine slot(s).
#include "simulate_fused.cuh"

namespace fmc {

cudaError_t launch_fused_big_nm4(int nd, const void* params, const CUtensorMap* maps, const FusedArgs& a, int smem,
                              int ntiles, int rows, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_fused_t<4, 1, true>(params, maps, a, smem, ntiles, rows, st, occ);
        case 2: return launch_fused_t<4, 2, true>(params, maps, a, smem, ntiles, rows, st, occ);
        case 4: return launch_fused_t<4, 4, true>(params, maps, a, smem, ntiles, rows, st, occ);
        case 8: return launch_fused_t<4, 8, true>(params, maps, a, smem, ntiles, rows, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fmc
