// Eq. (eqkl) as increments on the tcgen05 tensor cores, materialising dW:
//   dW[s][w][n] = sum_k zeta[s][w*K + k] phi[k][n]
// with BF16 operands (or split hi/lo BF16, three products) and FP32
// accumulation in TMEM.  One CTA per [128 samples x TN steps] block of one
// disturbance; thread 0 streams the K blocks with TMA and issues the MMAs, then
// each of the four warps reads its 32 TMEM lanes (= its 32 samples) and writes
// the rows to HBM.  This standalone form serves fmc_kle_reconstruct; the fused
// simulation consumes the same TMEM tiles without writing them out.
#include <cuda_bf16.h>

#include "fmc_common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace fmc {

struct ContractArgs {
    int64_t count;
    int d, Ks, nkb, Nt, TN;
    int split;
    float* dW;
    int* err;
};

__global__ void __launch_bounds__(128) contract_tc_kernel(const __grid_constant__ CUtensorMap mAh,
                                                          const __grid_constant__ CUtensorMap mAl,
                                                          const __grid_constant__ CUtensorMap mBh,
                                                          const __grid_constant__ CUtensorMap mBl, ContractArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1 KB alignment by an offset from the shared array itself (not through an
    // integer round trip), so that every access through these pointers stays a
    // shared-memory access rather than a generic one
    uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ uint64_t bars[5];  // full[2], freed[2], done
    __shared__ uint32_t tmem_base;
    __shared__ int ok_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int n0 = blockIdx.x * a.TN;
    const int64_t row0 = (int64_t)blockIdx.y * TC_M;
    const int w = blockIdx.z;
    const uint32_t ncols = a.TN < 32 ? 32 : a.TN;

    TcRing r;
    r.a_bytes = TC_M * 64;
    r.b_bytes = a.TN * 64;
    r.split = a.split;
    r.base = smem;
    r.ns = 2;
    r.full = &bars[0];
    r.freed = &bars[2];

    if (threadIdx.x == 0) {
        prefetch_tmap(&mAh);
        prefetch_tmap(&mBh);
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        mbar_init(&bars[3], 1);
        mbar_init(&bars[4], 1);
        fence_mbar_init();
        ok_flag = 1;
    }
    if (warp == 0) tmem_alloc(&tmem_base, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (threadIdx.x == 0) {
        const uint32_t idesc = umma_idesc_bf16(TC_M, a.TN);
        bool ok = true;
        const int ax0 = w * a.Ks;
        ok = ring_load(r, 0, &mAh, &mAl, &mBh, &mBl, ax0, (int)row0, 0, n0);
        for (int kb = 0; kb < a.nkb && ok; ++kb) {
            if (kb + 1 < a.nkb)
                ok = ring_load(r, kb + 1, &mAh, &mAl, &mBh, &mBl, ax0 + (kb + 1) * TC_BK, (int)row0,
                               (kb + 1) * TC_BK, n0);
            if (ok) ok = ring_mma(r, kb, tmem, idesc, kb == 0);
        }
        if (ok) umma_commit(&bars[4]);
        if (!ok) {
            ok_flag = 0;
            atomicExch(a.err, DEV_TIMEOUT_TMA);
        }
    }
    __syncthreads();
    bool ok = ok_flag != 0;
    if (ok && !mbar_wait(&bars[4], 0)) {
        ok = false;
        if (lane == 0) atomicExch(a.err, DEV_TIMEOUT_MMA);
    }
    // warps agree on ok (tcgen05.ld is warp-collective)
    ok = __all_sync(0xffffffffu, ok);
    tc_fence_after();
    if (ok) {
        const int64_t srow = row0 + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c = 0; c < a.TN; c += 4) {
            float v[4];
            tmem_ld4(lane_addr + c, v);
            tmem_ld_wait();
            if (srow < a.count) {
                float* out = a.dW + (srow * a.d + w) * (int64_t)a.Nt + n0 + c;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (n0 + c + e < a.Nt) out[e] = v[e];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

// zeta [count][d*K] FP32 -> hi/lo [count][d][Ks] BF16 with zero padding.
__global__ void split_rows_kernel(const float* __restrict__ z, int64_t count, int d, int K, int Ks,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo)
{
    int64_t row = (int64_t)d * Ks;
    int64_t total = count * row;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = t / row;
        int rem = (int)(t - j * row);
        int w = rem / Ks, kk = rem - w * Ks;
        float v = (kk < K) ? z[j * (int64_t)d * K + (int64_t)w * K + kk] : 0.f;
        __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[t] = h;
        lo[t] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

cudaError_t launch_split_rows(const float* z, int64_t count, int d, int K, int Ks, void* hi, void* lo, cudaStream_t st)
{
    int64_t total = count * (int64_t)d * Ks;
    int64_t g = (total + 255) / 256;
    if (g > 65536) g = 65536;
    split_rows_kernel<<<(unsigned)g, 256, 0, st>>>(z, count, d, K, Ks, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo);
    return cudaGetLastError();
}

cudaError_t launch_contract_tc(const CUtensorMap* maps, int64_t count, int d, int Ks, int nkb, int Nt, int TN,
                               int split, float* dW, int* err, cudaStream_t st)
{
    ContractArgs a{count, d, Ks, nkb, Nt, TN, split, dW, err};
    const int stage_bytes = (TC_M * 64 + TN * 64) * (split ? 2 : 1);
    // at least 47 KB so that no more than four CTAs (4 x 128 TMEM columns) share an SM
    int smem = 2 * stage_bytes + 1024;
    if (smem < 233472 / 5 - 1024 + 64) smem = 233472 / 5 - 1024 + 64;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(contract_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    int64_t gy = (count + TC_M - 1) / TC_M;
    if (gy > 65535) return cudaErrorInvalidValue;
    dim3 grid((Nt + TN - 1) / TN, (unsigned)gy, d);
    contract_tc_kernel<<<grid, 128, smem, st>>>(maps[0], maps[1], maps[2], maps[3], a);
    return cudaGetLastError();
}

}  // namespace fmc
