// Dispatch of the simulation kernels over the (machine, disturbance) slot
// buckets they are instantiated for, and the shared-memory plan of the fused
// kernel.
#include "simulate_fused.cuh"

namespace fmc {

cudaError_t launch_fused_nm1(int, const void*, const CUtensorMap*, const FusedArgs&, int, int, int, cudaStream_t, int*);
cudaError_t launch_plain_nm1(int, const void*, const double*, const float*, int64_t, int, float*, double*, int, cudaStream_t);
cudaError_t launch_fused_nm2(int, const void*, const CUtensorMap*, const FusedArgs&, int, int, int, cudaStream_t, int*);
cudaError_t launch_plain_nm2(int, const void*, const double*, const float*, int64_t, int, float*, double*, int, cudaStream_t);
cudaError_t launch_fused_nm4(int, const void*, const CUtensorMap*, const FusedArgs&, int, int, int, cudaStream_t, int*);
cudaError_t launch_plain_nm4(int, const void*, const double*, const float*, int64_t, int, float*, double*, int, cudaStream_t);
cudaError_t launch_fused_nm8(int, const void*, const CUtensorMap*, const FusedArgs&, int, int, int, cudaStream_t, int*);
cudaError_t launch_plain_nm8(int, const void*, const double*, const float*, int64_t, int, float*, double*, int, cudaStream_t);
cudaError_t launch_fused_nm10(int, const void*, const CUtensorMap*, const FusedArgs&, int, int, int, cudaStream_t, int*);
cudaError_t launch_plain_nm10(int, const void*, const double*, const float*, int64_t, int, float*, double*, int, cudaStream_t);
cudaError_t launch_fused_nm12(int, const void*, const CUtensorMap*, const FusedArgs&, int, int, int, cudaStream_t, int*);
cudaError_t launch_plain_nm12(int, const void*, const double*, const float*, int64_t, int, float*, double*, int, cudaStream_t);
cudaError_t launch_fused_nm16(int, const void*, const CUtensorMap*, const FusedArgs&, int, int, int, cudaStream_t, int*);
cudaError_t launch_plain_nm16(int, const void*, const double*, const float*, int64_t, int, float*, double*, int, cudaStream_t);


cudaError_t launch_wide_nmt1(int, const CUtensorMap*, const WideArgs&, cudaStream_t, int*);
cudaError_t launch_wide_nmt2(int, const CUtensorMap*, const WideArgs&, cudaStream_t, int*);
cudaError_t launch_wide_nmt3(int, const CUtensorMap*, const WideArgs&, cudaStream_t, int*);
cudaError_t launch_wide_nmt4(int, const CUtensorMap*, const WideArgs&, cudaStream_t, int*);
cudaError_t launch_wide_nmt5(int, const CUtensorMap*, const WideArgs&, cudaStream_t, int*);
cudaError_t launch_wide_nmt7(int, const CUtensorMap*, const WideArgs&, cudaStream_t, int*);
cudaError_t launch_wide_nmt10(int, const CUtensorMap*, const WideArgs&, cudaStream_t, int*);
cudaError_t launch_wide_nmt13(int, const CUtensorMap*, const WideArgs&, cudaStream_t, int*);

int wide_nmt_for(int n)
{
    static const int slots[] = {1, 2, 3, 4, 5, 7, 10, 13};
    for (int m : slots)
        if (n <= 4 * m) return m;
    return -1;
}

cudaError_t launch_simulate_wide(int nmt, int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st,
                                 int* max_ctas_per_sm)
{
    if (a.n > 4 * nmt || a.d > nd) return cudaErrorInvalidValue;
    switch (nmt) {
        case 1: return launch_wide_nmt1(nd, maps, a, st, max_ctas_per_sm);
        case 2: return launch_wide_nmt2(nd, maps, a, st, max_ctas_per_sm);
        case 3: return launch_wide_nmt3(nd, maps, a, st, max_ctas_per_sm);
        case 4: return launch_wide_nmt4(nd, maps, a, st, max_ctas_per_sm);
        case 5: return launch_wide_nmt5(nd, maps, a, st, max_ctas_per_sm);
        case 7: return launch_wide_nmt7(nd, maps, a, st, max_ctas_per_sm);
        case 10: return launch_wide_nmt10(nd, maps, a, st, max_ctas_per_sm);
        case 13: return launch_wide_nmt13(nd, maps, a, st, max_ctas_per_sm);
        default: return cudaErrorInvalidValue;
    }
}

// Ring stages of the fused kernel: as many as a CTA's share of the SM's shared
// memory holds (2..TC_MAX_STAGES), so that more of a chunk's loads are in flight.
// A half tile (64 rows) keeps 4 KB after the ring: its M = 128 MMA reads 64 rows
// past the last loaded tile.
int fused_ring_stages(int TC, int split, int max_ctas_per_sm, int rows)
{
    const int stage = (rows * 64 + TC * 64) * (split ? 2 : 1);
    int share = 233472 / max_ctas_per_sm - 2048;  // per CTA: 1 KB reserved, 1 KB static
    if (share > TC_SMEM_DYN_MAX) share = TC_SMEM_DYN_MAX;
    int ns = (share - 1024 - (TC_M - rows) * 64) / stage;
    return ns < 2 ? 2 : (ns > TC_MAX_STAGES ? TC_MAX_STAGES : ns);
}

int fused_smem_bytes(int nm_bucket, int TC, int split, int max_ctas_per_sm, int rows)
{
    const int stage = (rows * 64 + TC * 64) * (split ? 2 : 1);
    const int ring = fused_ring_stages(TC, split, max_ctas_per_sm, rows) * stage + (TC_M - rows) * 64;
    const int warps = rows / 32;
    const int mom = (warps * 32 * (2 * nm_bucket + 1) + fu_ms(nm_bucket) * warps * 6 * nm_bucket) * 4;
    int need = (ring > mom ? ring : mom) + 1024;
    // at most max_ctas_per_sm CTAs per SM (233472 bytes of shared memory per SM,
    // 1 KB reserved per CTA), so that their TMEM columns fit the SM's 512
    const int floor = 233472 / (max_ctas_per_sm + 1) - 1024 + 64;
    return need > floor ? need : floor;
}

cudaError_t launch_simulate_fused(int nm_bucket, int nd_bucket, const void* params, const CUtensorMap* maps,
                                  int64_t count, int Nt, int TC, int d, int Ks, int nkb, int split, uint32_t tmem_cols,
                                  int rows, int max_ctas, const double* eq, float* part, double* S1, double* S2,
                                  float* traj, int* err, const EmSpec& em, double* rrf, const L2Keep& keep,
                                  int smooth, cudaStream_t st, int* max_ctas_per_sm)
{
    if (rows != TC_M && rows != TC_M / 2) return cudaErrorInvalidValue;
    int cap = (int)(512u / tmem_cols) < max_ctas ? (int)(512u / tmem_cols) : max_ctas;
    const int cw = smooth ? 2 * TC : TC;  // basis rows of a chunk (the smooth form's half steps)
    FusedArgs a{count, Nt, TC, d, Ks, nkb, split, fused_ring_stages(cw, split, cap, rows), tmem_cols, eq, part,
                traj, err, S1, S2, em, rrf, static_cast<const uint8_t*>(keep.hi), static_cast<const uint8_t*>(keep.lo),
                keep.row_bytes, keep.tiles, smooth};
    const int smem = fused_smem_bytes(nm_bucket, cw, split, cap, rows);
    const int64_t ntiles = (count + rows - 1) / rows;
    if (ntiles > 2147483647LL) return cudaErrorInvalidValue;
    switch (nm_bucket) {
        case 1: return launch_fused_nm1(nd_bucket, params, maps, a, smem, (int)ntiles, rows, st, max_ctas_per_sm);
        case 2: return launch_fused_nm2(nd_bucket, params, maps, a, smem, (int)ntiles, rows, st, max_ctas_per_sm);
        case 4: return launch_fused_nm4(nd_bucket, params, maps, a, smem, (int)ntiles, rows, st, max_ctas_per_sm);
        case 8: return launch_fused_nm8(nd_bucket, params, maps, a, smem, (int)ntiles, rows, st, max_ctas_per_sm);
        case 10: return launch_fused_nm10(nd_bucket, params, maps, a, smem, (int)ntiles, rows, st, max_ctas_per_sm);
        case 12: return launch_fused_nm12(nd_bucket, params, maps, a, smem, (int)ntiles, rows, st, max_ctas_per_sm);
        case 16: return launch_fused_nm16(nd_bucket, params, maps, a, smem, (int)ntiles, rows, st, max_ctas_per_sm);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_simulate_plain(int nm_bucket, int nd_bucket, const void* params, const double* eq, const float* dW,
                                  int64_t count, int Nt, float* traj, double* rrf, int smooth, cudaStream_t st)
{
    switch (nm_bucket) {
        case 1: return launch_plain_nm1(nd_bucket, params, eq, dW, count, Nt, traj, rrf, smooth, st);
        case 2: return launch_plain_nm2(nd_bucket, params, eq, dW, count, Nt, traj, rrf, smooth, st);
        case 4: return launch_plain_nm4(nd_bucket, params, eq, dW, count, Nt, traj, rrf, smooth, st);
        case 8: return launch_plain_nm8(nd_bucket, params, eq, dW, count, Nt, traj, rrf, smooth, st);
        case 10: return launch_plain_nm10(nd_bucket, params, eq, dW, count, Nt, traj, rrf, smooth, st);
        case 12: return launch_plain_nm12(nd_bucket, params, eq, dW, count, Nt, traj, rrf, smooth, st);
        case 16: return launch_plain_nm16(nd_bucket, params, eq, dW, count, Nt, traj, rrf, smooth, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fmc
