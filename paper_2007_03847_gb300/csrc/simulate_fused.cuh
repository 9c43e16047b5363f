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
//                    through shared memory and forms per state a reference value
//                    (its first sample), the sum about it and the squared
//                    deviations (column_sums); every few steps the warps' triples
//                    are combined in a fixed order into the tile's and written as
//                    FP32 partials [tile][t][ref | dev | m2]
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
// Steps between flushes of the moment buffer (measured: 8 -> 32 saves 0.8%; 16
// above 10 machine slots, so that four CTAs' buffers still share an SM)
__host__ __device__ constexpr int fu_ms(int nm) { return nm > 10 ? 16 : 32; }

struct FusedArgs {
    int64_t count;
    int Nt, TC, d, Ks, nkb, split;
    int ns;             // ring stages
    uint32_t tmem_cols;
    const double* eq;   // [delta* n][pm n][moment shift 2n] (the shift is used by the reduce)
    float* part;        // [ntiles][Nt+1][3][2n] (ref | dev | m2), or nullptr: add into S1, S2 with FP64 atomics
    float* traj;        // [count][Nt+1][2n] or nullptr
    int* err;
    double* S1;         // [Nt+1][2n] when part == nullptr
    double* S2;
    EmSpec em;          // on: per-step normals instead of the contraction (no tensor cores)
    double* rrf;        // [2]: sums of the response function and its square, or nullptr
    // L2 residency of the design: tiles below keep_tiles load their rows with an
    // evict_last policy (every chunk re-reads them), the others evict_first; at
    // exit the kept lines return to normal priority.  keep_tiles 0: no hint.
    const uint8_t* zeta_hi;
    const uint8_t* zeta_lo;
    int64_t zeta_row_bytes;
    int keep_tiles;
    // the smooth form (Eq. eqkl as a random ODE): the contraction gives the
    // forcing at the 2 TC half-step times t_n0 + dt/2 .. t_n0+TC of each chunk
    // (2 TC TMEM columns per disturbance; the chunk's first value, at t_n0, is
    // carried from the chunk before, and a first contraction over rows up to 0
    // gives f(0)), and the step loop forms the disturbances' RK stage values
    int smooth;
};

template <int NM, int ND, bool SMOOTH>
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
    const int n = p.n, d = p.d, S = 2 * n, S3 = 3 * S;
    constexpr int FU_MS = fu_ms(NM);
    constexpr int MSLOT = 6 * NM;  // floats per (step, warp) slot: ref | dev | m2 of up to 2 NM states
    const int64_t row0 = (int64_t)blockIdx.x * rows;
    const int64_t srow = row0 + tid;
    const bool active = srow < a.count;
    const int TC = a.TC;
    const int CW = SMOOTH ? 2 * TC : TC;  // TMEM columns per disturbance and chunk

    // ring (used only while the tensor cores fill TMEM) aliases the moment buffers
    TcRing r;
    r.a_bytes = rows * 64;
    r.b_bytes = CW * 64;
    r.split = a.split;
    r.base = smem;
    r.ns = (uint32_t)a.ns;
    r.full = &bars[0];
    r.freed = &bars[TC_MAX_STAGES];
    r.a_policy = 0;
    if (a.keep_tiles > 0) r.a_policy = (int)blockIdx.x < a.keep_tiles ? l2_policy_evict_last() : l2_policy_evict_first();
    uint64_t* done = &bars[2 * TC_MAX_STAGES];
    const int WROW = 2 * NM + 1;
    float* wbuf = reinterpret_cast<float*>(smem) + warp * 32 * WROW;           // [32][WROW] per warp
    float* msum = reinterpret_cast<float*>(smem) + warps * 32 * WROW;          // [FU_MS][warps][MSLOT]

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
    const int J = d * a.nkb;  // K blocks of a chunk
    const uint32_t idesc = umma_idesc_bf16(TC_M, CW);

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
    float* part_tile = a.part ? a.part + (int64_t)blockIdx.x * (a.Nt + 1) * S3 : nullptr;
    if (part_tile)
        for (int v = tid; v < S3; v += rows) part_tile[v] = 0.f;

    uint32_t g = 0;  // K blocks issued so far (thread 0)
    float racc = 0.f;  // sum over the grid of the squared centre-of-inertia speed

    float f0[ND];  // the smooth form's forcing at the chunk's first grid time
#pragma unroll
    for (int q = 0; q < ND; ++q) f0[q] = 0.f;
    for (int c = 0, n0 = SMOOTH ? -TC : 0; n0 < a.Nt; ++c, n0 += TC) {
        // ---- tensor cores: dW of this chunk into TMEM ----
        if (!em) {
        tc_fence_before();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            // item j: disturbance wj, K block kb; loads run up to ns - 1 items ahead
            // of the MMAs (a stage is refilled once its MMAs completed)
            auto load_item = [&](int j) {
                const int wj = j / a.nkb, kb = j - wj * a.nkb;
                return ring_load(r, g + (uint32_t)j, &mAh, &mAl, &mBh, &mBl, wj * a.Ks + kb * TC_BK, (int)row0,
                                 kb * TC_BK, SMOOTH ? 2 * n0 + 1 : n0);
            };
            bool ok = true;
            int issued = 0;
            for (; issued < J && issued + 1 < (int)r.ns && ok; ++issued) ok = load_item(issued);
            for (int j = 0; j < J && ok; ++j) {
                if (issued < J) {
                    ok = load_item(issued);
                    ++issued;
                    if (!ok) break;
                }
                const int wj = j / a.nkb, kb = j - wj * a.nkb;
                ok = ring_mma(r, g + (uint32_t)j, tmem + (uint32_t)(wj * CW), idesc, kb == 0);
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

        if constexpr (SMOOTH) {
            if (n0 < 0) {
                // f(0): the last column of the contraction over the rows up to 0
#pragma unroll
                for (int q = 0; q < ND; ++q)
                    if (q < d) f0[q] = tmem_ld1(lane_addr + (uint32_t)(q * CW + CW - 1));
                tmem_ld_wait();
                continue;
            }
        }
        const int steps = (a.Nt - n0) < TC ? (a.Nt - n0) : TC;
        // ---- disturbance paths of this chunk into TMEM (each warp its own lanes) ----
        if constexpr (!SMOOTH)
            disturbance_chunk<ND, ND, true>(lane_addr, TC, steps, n0, d, -1, x0, p.ou_a, p.ou_s, p.ito, p.dt, a.em,
                                            (uint32_t)(a.em.k0 + srow));

        // ---- FP32 pipes: integrate this chunk ----
        for (int s = 0; s < steps; ++s) {
            if constexpr (SMOOTH) {
                // the forcing at t_n + dt/2 and t_{n+1}; the stage values of the
                // disturbances' random ODE feed the swing stages
                float fh[ND], f1[ND], xst[4][ND];
#pragma unroll
                for (int q = 0; q < ND; ++q) {
                    fh[q] = 0.f;
                    f1[q] = 0.f;
                }
#pragma unroll
                for (int q = 0; q < ND; ++q)
                    if (q < d) {
                        fh[q] = tmem_ld1(lane_addr + (uint32_t)(q * CW + 2 * s));
                        f1[q] = tmem_ld1(lane_addr + (uint32_t)(q * CW + 2 * s + 1));
                    }
                tmem_ld_wait();
                smooth_stages<NM, ND>(p, n0 + s, x0, f0, fh, f1, xst);
#pragma unroll
                for (int q = 0; q < ND; ++q) f0[q] = f1[q];
                swing_step_staged<NM, ND>(p, del, w, theta, xst);
            } else {
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
                swing_step<NM, ND, (NM <= 10)>(p, del, w, theta, x0, x1);
#pragma unroll
                for (int q = 0; q < ND; ++q) x0[q] = x1[q];
            }
            if (a.rrf) {
                const float cs = coi_speed<NM, ND>(p, w);
                racc = fmaf(cs, cs, racc);
            }

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
            // (row r holds lane r's sample: angles in columns 0..NM-1, speeds in
            // NM..2NM-1; rows past the tile's last sample hold whatever those
            // lanes integrated, and column_sums reads only the first na_warp rows)
            float* myrow = wbuf + lane * WROW;
#pragma unroll
            for (int i = 0; i < NM; ++i) {
                myrow[i] = theta + del[i];
                myrow[NM + i] = w[i];
            }
            __syncwarp();
            const int ms = s % FU_MS;
            if (lane < S) {
                // the warp's reference value, sum about it and squared deviations, per
                // state (lane j: state j, its column of the transpose buffer)
                const int mcol = lane < n ? lane : NM + lane - n;
                const int64_t left = a.count - (srow - lane);
                const int na_warp = left <= 0 ? 0 : (left >= 32 ? 32 : (int)left);
                float rf, dv, m2;
                column_sums(wbuf + mcol, WROW, na_warp, &rf, &dv, &m2);
                float* slot = msum + (ms * warps + warp) * MSLOT;
                slot[lane] = rf;
                slot[S + lane] = dv;
                slot[2 * S + lane] = m2;
            }
            __syncwarp();
            if (ms == FU_MS - 1 || s == steps - 1) {
                asm volatile("bar.sync 1, %0;" ::"r"(rows) : "memory");
                const int nst = ms + 1;
                const int tn0 = tn - ms;
                // samples of this tile (the last tile may be partly empty)
                const int64_t left = a.count - row0;
                const int n_tile = left <= 0 ? 0 : (left >= rows ? rows : (int)left);
                for (int e = tid; e < nst * S; e += rows) {
                    const int sl = e / S, j = e - sl * S;  // step slot, state
                    const float* m = msum + sl * warps * MSLOT + j;
                    // the tile's triple: reference (warp 0's), sum about it, squared deviations
                    float c, dv, m2;
                    combine_groups(m, m + S, m + 2 * S, MSLOT, left, warps, &c, &dv, &m2);
                    if (part_tile) {
                        float* o = part_tile + (int64_t)(tn0 + sl) * S3;
                        o[j] = c;
                        o[S + j] = dv;
                        o[2 * S + j] = m2;
                    } else if (n_tile > 0) {
                        // the tile's S1 and S2 (= M2 + S1^2 / n) about the shift, in FP64
                        const int64_t row = (int64_t)(tn0 + sl) * S;
                        const double s1 = fma((double)n_tile, (double)c, (double)dv);
                        atomicAdd(a.S1 + row + j, s1);
                        atomicAdd(a.S2 + row + j, (double)m2 + s1 * s1 / (double)n_tile);
                    }
                }
                asm volatile("bar.sync 1, %0;" ::"r"(rows) : "memory");
            }
        }
    }
    if (a.rrf) rrf_accumulate(active ? sqrtf(racc / (float)a.Nt) : 0.f, a.rrf);
    if (!em && (int)blockIdx.x < a.keep_tiles) {
        // the tile's design rows back to normal L2 priority
        const int64_t left = a.count - row0;
        const int64_t bytes = (left < rows ? left : rows) * a.zeta_row_bytes;
        for (int64_t o = (int64_t)tid * 128; o < bytes; o += (int64_t)rows * 128) {
            l2_priority_normal(a.zeta_hi + row0 * a.zeta_row_bytes + o);
            if (a.split) l2_priority_normal(a.zeta_lo + row0 * a.zeta_row_bytes + o);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, a.tmem_cols);
}

template <int NM, int ND>
cudaError_t launch_fused_t(const void* params, const CUtensorMap* maps, const FusedArgs& a, int smem, int ntiles,
                           int rows, cudaStream_t st, int* max_ctas_per_sm)
{
    const SwingParams<NM, ND>& p = *static_cast<const SwingParams<NM, ND>*>(params);
    auto kern = a.smooth ? simulate_fused_kernel<NM, ND, true> : simulate_fused_kernel<NM, ND, false>;
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
