// Instantiations of the four-warps-per-sample fused kernel with the network sums
// on the tensor cores: 4, 5 and 7 machine slots per thread, and its dispatch.
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

static cudaError_t wide_tc_nmt4(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    FMC_WIDE_TC_ND(4)
}

static cudaError_t wide_tc_nmt5(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    FMC_WIDE_TC_ND(5)
}

static cudaError_t wide_tc_nmt7(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ)
{
    FMC_WIDE_TC_ND(7)
}

cudaError_t wide_tc_nmt10(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ);
cudaError_t wide_tc_nmt13(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ);
cudaError_t wide_tc_h2_nmt10(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ);
cudaError_t wide_tc_h2_nmt13(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ);
cudaError_t wide_tc_h2_nmt9(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ);
cudaError_t wide_tc_h2_nmt11(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ);
cudaError_t wide_tc_h2_nmt12(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ);
cudaError_t wide_tc_h2_nmt14(int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ);

cudaError_t wide_tc_bus(int nmt, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st, int* occ);

cudaError_t launch_simulate_wide_tc(int nmt, int H, int nd, bool bus, const CUtensorMap* maps, const WideArgs& a,
                                    cudaStream_t st, int* max_ctas_per_sm)
{
    if (a.n > H * nmt || a.d > nd || a.tmem_cols != (H == 2 ? 256u : 512u)) return cudaErrorInvalidValue;
    if (bus) {
        if (H != 4 || nd != 8 || a.n >= H * nmt) return cudaErrorInvalidValue;
        return wide_tc_bus(nmt, maps, a, st, max_ctas_per_sm);
    }
    if (H == 2) {
        if (nmt == 9) return wide_tc_h2_nmt9(nd, maps, a, st, max_ctas_per_sm);
        if (nmt == 10) return wide_tc_h2_nmt10(nd, maps, a, st, max_ctas_per_sm);
        if (nmt == 11) return wide_tc_h2_nmt11(nd, maps, a, st, max_ctas_per_sm);
        if (nmt == 12) return wide_tc_h2_nmt12(nd, maps, a, st, max_ctas_per_sm);
        if (nmt == 13) return wide_tc_h2_nmt13(nd, maps, a, st, max_ctas_per_sm);
        if (nmt == 14) return wide_tc_h2_nmt14(nd, maps, a, st, max_ctas_per_sm);
        return cudaErrorInvalidValue;
    }
    if (H != 4) return cudaErrorInvalidValue;
    switch (nmt) {
        case 4: return wide_tc_nmt4(nd, maps, a, st, max_ctas_per_sm);
        case 5: return wide_tc_nmt5(nd, maps, a, st, max_ctas_per_sm);
        case 7: return wide_tc_nmt7(nd, maps, a, st, max_ctas_per_sm);
        case 10: return wide_tc_nmt10(nd, maps, a, st, max_ctas_per_sm);
        case 13: return wide_tc_nmt13(nd, maps, a, st, max_ctas_per_sm);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fmc
