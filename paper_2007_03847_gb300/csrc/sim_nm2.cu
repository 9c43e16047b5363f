// Instantiations of the simulation kernels for 2 machine slot(s).
#include "simulate_fused.cuh"
#include "simulate_plain.cuh"

namespace fmc {

cudaError_t launch_fused_nm2(int nd, const void* params, const CUtensorMap* maps, const FusedArgs& a, int smem,
                              int ntiles, int rows, cudaStream_t st, int* occ)
{
    switch (nd) {
        case 1: return launch_fused_t<2, 1>(params, maps, a, smem, ntiles, rows, st, occ);
        case 2: return launch_fused_t<2, 2>(params, maps, a, smem, ntiles, rows, st, occ);
        case 4: return launch_fused_t<2, 4>(params, maps, a, smem, ntiles, rows, st, occ);
        case 8: return launch_fused_t<2, 8>(params, maps, a, smem, ntiles, rows, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_plain_nm2(int nd, const void* params, const double* eq, const float* dW, int64_t count, int Nt,
                              float* traj, double* rrf, int smooth, cudaStream_t st)
{
    switch (nd) {
        case 1: return launch_plain_t<2, 1>(params, eq, dW, count, Nt, traj, rrf, smooth, st);
        case 2: return launch_plain_t<2, 2>(params, eq, dW, count, Nt, traj, rrf, smooth, st);
        case 4: return launch_plain_t<2, 4>(params, eq, dW, count, Nt, traj, rrf, smooth, st);
        case 8: return launch_plain_t<2, 8>(params, eq, dW, count, Nt, traj, rrf, smooth, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fmc
