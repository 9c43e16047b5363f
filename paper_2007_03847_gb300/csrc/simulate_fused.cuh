// Algorithm 1 steps 2-4 fused on one SM-resident CTA per 128 samples:
//
// (A CTA may also take 64 samples in two warps -- "half tiles" -- so that a
// grid that would leave SMs with uneven numbers of 4-warp CTAs spreads its
// warps more evenly; the MMA then still has M = 128, its upper 64 rows being
// whatever follows the 64-row tile in shared memory, and lanes 64..127 of the
// accumulator are never read.)
//
//   for each time chunk of TC steps:
//     tensor cores:  dW[128 x TC] per disturbance = Z_tile . Phi_chunk^T into TMEM
//                    (BF16 or split BF16x3 operands streamed by TMA, FP32 accumulate)
//     disturbances:  thread r (= sample r of the tile, = TMEM lane r) turns its
//                    increments into the chunk's disturbance paths by Euler-Maruyama,
//                    in place in TMEM (tcgen05.ld / tcgen05.st, see disturb_chunk.cuh)
//     FP32 pipes:    it reads x(t_{n+1}) with tcgen05.ld and advances the swing
//                    equations by RK4/Heun, step by step
//     moments:       per step, each warp transposes its 32 samples' shifted states
//                    through shared memory and sums them (S1, S2) per state; the
//                    four warps' sums are added in a fixed order and written as
//                    FP32 partials [tile][t][S1 | S2]
//
// Trajectories never go to HBM (unless a debug buffer is given).  A separate
// kernel combines the per-tile partials in FP64 in a fixed order.
#pragma once

#include "fmc_common.cuh"
#include "kernels.cuh"
#include "swing.cuh"
#include "tc_common.cuh"
#include "disturb_chunk.cuh"

namespace fmc {

constexpr int FU_THREADS = 128;  // full tile; a half tile has 64 threads
constexpr int FU_MS = 32;  // steps between flushes of the moment buffer (measured: 8 -> 32 saves 0.8%)

struct FusedArgs {
    int64_t count;
    int Nt, TC, d, Ks, nkb, split;
    int ns;             // ring stages
    uint32_t tmem_cols;
    const double* eq;   // [delta* n][pm n][moment shift 2n] (the shift is used by the reduce)
    float* part;        // [ntiles][Nt+1][4n], or nullptr: add into S1, S2 with FP64 atomics
    float* traj;        // [count][Nt+1][2n] or nullptr
    int* err;
    double* S1;         // [Nt+1][2n] when part == nullptr
    double* S2;
    EmSpec em;          // on: per-step normals instead of the contraction (no tensor cores)
    double* rrf;        // [2]: sums of the response function and its square, or nullptr
};

template <int NM, int ND>
__global__ void __launch_bounds__(FU_THREADS, 4)
    simulate_fused_kernel(const __grid_constant__ SwingParams<NM, ND> p, const __grid_constant__ CUtensorMap mAh,
                          const __grid_constant__ CUtensorMap mAl, const __grid_constant__ CUtensorMap mBh,
                          const __grid_constant__ CUtensorMap mBl, FusedArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1 KB alignment by an offset from the shared array itself (not through an
    // integer round trip), so that every access through these pointers stays a
    // shared-memory access rather than a generic one
    uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ uint64_t bars[2 * TC_MAX_STAGES + 1];  // full[ns], freed[ns], done
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int rows = blockDim.x, warps = rows / 32;  // samples (= threads) and warps of this CTA
    const int n = p.n, d = p.d, S = 2 * n, S4 = 4 * n;
    const int64_t row0 = (int64_t)blockIdx.x * rows;
    const int64_t srow = row0 + tid;
    const bool active = srow < a.count;
    const int TC = a.TC;

    // ring (used only while the tensor cores fill TMEM) aliases the moment buffers
    TcRing r;
    r.a_bytes = rows * 64;
    r.b_bytes = TC * 64;
    r.split = a.split;
    r.base = smem;
    r.ns = (uint32_t)a.ns;
    r.full = &bars[0];
    r.freed = &bars[TC_MAX_STAGES];
    uint64_t* done = &bars[2 * TC_MAX_STAGES];
    const int WROW = 2 * NM + 1;
    float* wbuf = reinterpret_cast<float*>(smem) + warp * 32 * WROW;           // [32][WROW] per warp
    float* msum = reinterpret_cast<float*>(smem) + warps * 32 * WROW;          // [FU_MS][warps][4*NM]

    const bool em = a.em.on != 0;
    if (tid == 0) {
        if (!em) {
            prefetch_tmap(&mAh);
            prefetch_tmap(&mBh);
        }
        for (int b = 0; b < 2 * TC_MAX_STAGES + 1; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    if (warp == 0) tmem_alloc(&tmem_base, a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);

    float del[NM], w[NM], theta = 0.f;   // deviations from the equilibrium (see swing_step)
    float x0[ND];
#pragma unroll
    for (int i = 0; i < NM; ++i) {
        del[i] = 0.f;
        w[i] = 0.f;
    }
#pragma unroll
    for (int q = 0; q < ND; ++q) x0[q] = 0.f;

    const int64_t trow = 2 * (int64_t)n;
    float* traj = (a.traj != nullptr && active) ? a.traj + srow * (int64_t)(a.Nt + 1) * trow : nullptr;
    if (traj) {
#pragma unroll
        for (int i = 0; i < NM; ++i)
            if (i < n) {
                traj[i] = p.dst[i];
                traj[n + i] = 0.f;
            }
    }
    // time 0: every sample sits at the (rounded) shift, so both sums are zero
    float* part_tile = a.part ? a.part + (int64_t)blockIdx.x * (a.Nt + 1) * S4 : nullptr;
    if (part_tile)
        for (int v = tid; v < S4; v += rows) part_tile[v] = 0.f;

    const uint32_t idesc = umma_idesc_bf16(TC_M, TC);
    uint32_t g = 0;  // K blocks issued so far (thread 0)
    float racc = 0.f;  // sum over the grid of the squared centre-of-inertia speed
    const int J = d * a.nkb;

    for (int c = 0, n0 = 0; n0 < a.Nt; ++c, n0 += TC) {
        // ---- tensor cores: dW of this chunk into TMEM ----
        if (!em) {
        tc_fence_before();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            bool ok = ring_load(r, g, &mAh, &mAl, &mBh, &mBl, 0, (int)row0, 0, n0);
            for (int j = 0; j < J && ok; ++j) {
                if (j + 1 < J) {
                    const int w1 = (j + 1) / a.nkb, kb1 = (j + 1) % a.nkb;
                    ok = ring_load(r, g + j + 1, &mAh, &mAl, &mBh, &mBl, w1 * a.Ks + kb1 * TC_BK, (int)row0,
                                   kb1 * TC_BK, n0);
                }
                const int wj = j / a.nkb, kbj = j % a.nkb;
                if (ok) ok = ring_mma(r, g + j, tmem + (uint32_t)(wj * TC), idesc, kbj == 0);
            }
            g += (uint32_t)J;
            if (ok) {
                umma_commit(done);
            } else {
                abort_flag = 1;
                atomicExch(a.err, DEV_TIMEOUT_TMA);
            }
        }
        __syncthreads();
        bool ok = (abort_flag == 0);
        if (ok && !mbar_wait(done, (uint32_t)c & 1u)) {
            ok = false;
            atomicExch(a.err, DEV_TIMEOUT_MMA);
        }
        if (!__syncthreads_and(ok)) break;
        tc_fence_after();
        }

        // ---- disturbance paths of this chunk into TMEM (each warp its own lanes) ----
        const int steps = (a.Nt - n0) < TC ? (a.Nt - n0) : TC;
        disturbance_chunk<ND, ND, true>(lane_addr, TC, steps, n0, d, -1, x0, p.ou_a, p.ou_s, p.ito, p.dt, a.em,
                                  (uint32_t)(a.em.k0 + srow));

        // ---- FP32 pipes: integrate this chunk ----
        for (int s = 0; s < steps; ++s) {
            float x1[ND];
#pragma unroll
            for (int q = 0; q < ND; ++q) x1[q] = 0.f;
#pragma unroll
            for (int q = 0; q < ND; ++q)
                if (q < d) x1[q] = tmem_ld1(lane_addr + (uint32_t)(q * TC + s));
            tmem_ld_wait();
            // the event slot: 0 before the event's grid step, 1 from it
#pragma unroll
            for (int q = 0; q < ND; ++q)
                if (q == p.ev_slot) {
                    x0[q] = (n0 + s >= p.ev_step) ? 1.f : 0.f;
                    x1[q] = x0[q];
                }
            swing_step<NM, ND>(p, del, w, theta, x0, x1);
            if (a.rrf) {
                const float cs = coi_speed<NM, ND>(p, w);
                racc = fmaf(cs, cs, racc);
            }
#pragma unroll
            for (int q = 0; q < ND; ++q) x0[q] = x1[q];

            const int tn = n0 + s + 1;  // grid index of the new state
            if (traj) {
                float* o = traj + (int64_t)tn * trow;
#pragma unroll
                for (int i = 0; i < NM; ++i)
                    if (i < n) {
                        o[i] = (theta + del[i]) + p.dst[i];
                        o[n + i] = w[i];
                    }
            }
            // ---- moments: transpose the warp's states and sum per state ----
            float* myrow = wbuf + lane * WROW;
#pragma unroll
            for (int i = 0; i < NM; ++i)
                if (i < n) {
                    myrow[i] = active ? theta + del[i] : 0.f;
                    myrow[n + i] = active ? w[i] : 0.f;
                }
            __syncwarp();
            const int ms = s % FU_MS;
            if (lane < S) {
                // the warp's sum and squared deviations from its mean, per state
                const int64_t left = a.count - (srow - lane);
                const int na_warp = left <= 0 ? 0 : (left >= 32 ? 32 : (int)left);
                float s1, m2;
                column_sum_m2(wbuf + lane, WROW, na_warp, &s1, &m2);
                msum[(ms * warps + warp) * (4 * NM) + lane] = s1;
                msum[(ms * warps + warp) * (4 * NM) + S + lane] = m2;
            }
            __syncwarp();
            if (ms == FU_MS - 1 || s == steps - 1) {
                asm volatile("bar.sync 1, %0;" ::"r"(rows) : "memory");
                const int nst = ms + 1;
                const int tn0 = tn - ms;
                // samples of this tile (the last tile may be partly empty)
                const int64_t left = a.count - row0;
                const int n_tile = left <= 0 ? 0 : (left >= rows ? rows : (int)left);
                for (int e = tid; e < nst * S4; e += rows) {
                    const int sl = e / S4, v = e - sl * S4;
                    const int j = v < S ? v : v - S;  // state
                    const float* m = msum + sl * warps * (4 * NM) + j;
                    // tile sum; for the second half the tile's squared deviations (parallel combine)
                    const float t1 =
                        warps == 4 ? ((m[0] + m[4 * NM]) + m[2 * 4 * NM]) + m[3 * 4 * NM] : m[0] + m[4 * NM];
                    const float acc = v < S ? t1 : combine_m2(m, m + S, 4 * NM, left, warps);
                    if (part_tile) {
                        part_tile[(int64_t)(tn0 + sl) * S4 + v] = acc;
                    } else {
                        // the tile's S1 and S2 (= M2 + S1^2 / n) about the shift, in FP64
                        const int64_t row = (int64_t)(tn0 + sl) * S;
                        if (v < S)
                            atomicAdd(a.S1 + row + v, (double)acc);
                        else if (n_tile > 0)
                            atomicAdd(a.S2 + row + j, (double)acc + (double)t1 * (double)t1 / (double)n_tile);
                    }
                }
                asm volatile("bar.sync 1, %0;" ::"r"(rows) : "memory");
            }
        }
    }
    if (a.rrf) rrf_accumulate(active ? sqrtf(racc / (float)a.Nt) : 0.f, a.rrf);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, a.tmem_cols);
}

template <int NM, int ND>
cudaError_t launch_fused_t(const void* params, const CUtensorMap* maps, const FusedArgs& a, int smem, int ntiles,
                           int rows, cudaStream_t st, int* max_ctas_per_sm)
{
    const SwingParams<NM, ND>& p = *static_cast<const SwingParams<NM, ND>*>(params);
    auto kern = simulate_fused_kernel<NM, ND>;
    // the attribute is process-wide and launches from several host threads may
    // race on it: always the same (largest) bound, the launch passes its own size
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_DYN_MAX);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, rows, smem);
    if (e != cudaSuccess) return e;
    *max_ctas_per_sm = occ;
    // every resident CTA holds tmem_cols TMEM columns; 512 per SM
    if (occ < 1 || (uint32_t)occ * a.tmem_cols > 512u) return cudaErrorInvalidConfiguration;
    kern<<<ntiles, rows, smem, st>>>(p, maps[0], maps[1], maps[2], maps[3], a);
    return cudaGetLastError();
}

}  // namespace fmc
