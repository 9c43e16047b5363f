// Algorithm 1 step 1 / Section IV-B: Latin hypercube sampling of the M = d*K
// KL coefficients on the GPU.  One thread per (sample, dimension); the design is
// stateless (a keyed Feistel permutation per dimension), so any sub-range of the
// N rows is produced bit-identically without sorting or communication.
#include <cuda_bf16.h>

#include "fmc_common.cuh"
#include "kernels.cuh"
#include "lhs_feistel.cuh"

namespace fmc {

__device__ __forceinline__ float lhs_value(uint32_t k, uint32_t dim, uint32_t N, int mode, int h, uint32_t mask,
                                           uint32_t k0, uint32_t k1, uint32_t* s_out)
{
    if (mode == FMC_SRS) {
        uint32_t r = philox4x32_10(U4{k, dim, 0u, 0u}, k0, k1).x;
        *s_out = k;
        return normal_from_fraction(2ull * r + 1ull, 1u);
    }
    uint32_t s = stratum(k, dim, N, h, mask, k0, k1);
    *s_out = s;
    uint64_t num2;
    if (mode == FMC_LHS_MIDPOINT) {
        num2 = ((uint64_t)s << 33) + (1ull << 32);
    } else {
        uint32_t r = philox4x32_10(U4{k, dim, 0u, 0u}, k0, k1).x;
        num2 = ((uint64_t)s << 33) + 2ull * r + 1ull;
    }
    return normal_from_fraction(num2, N);
}

__global__ void lhs_f32_kernel(uint32_t k0s, uint32_t k1s, uint32_t N, int64_t k0, int64_t count, int M, int mode,
                               int h, uint32_t mask, float* __restrict__ zeta, uint32_t* __restrict__ strata)
{
    int64_t total = count * (int64_t)M;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = t / M;
        int i = (int)(t - j * M);
        uint32_t s;
        float z = lhs_value((uint32_t)(k0 + j), (uint32_t)i, N, mode, h, mask, k0s, k1s, &s);
        if (zeta) zeta[t] = z;
        if (strata) strata[(int64_t)i * count + j] = s;
    }
}

// Split-BF16 layout for the tensor-core contraction: [count][d][Ks] with zeros
// in the K..Ks-1 padding of every group.
__global__ void lhs_split_kernel(uint32_t k0s, uint32_t k1s, uint32_t N, int64_t k0, int64_t count, int d, int K,
                                 int Ks, int mode, int h, uint32_t mask, __nv_bfloat16* __restrict__ hi,
                                 __nv_bfloat16* __restrict__ lo)
{
    int64_t row = (int64_t)d * Ks;
    int64_t total = count * row;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = t / row;
        int rem = (int)(t - j * row);
        int w = rem / Ks;
        int kk = rem - w * Ks;
        float z = 0.f;
        if (kk < K) {
            uint32_t s;
            z = lhs_value((uint32_t)(k0 + j), (uint32_t)(w * K + kk), N, mode, h, mask, k0s, k1s, &s);
        }
        __nv_bfloat16 zh = __float2bfloat16_rn(z);
        hi[t] = zh;
        if (lo) lo[t] = __float2bfloat16_rn(z - __bfloat162float(zh));
    }
}

// The paper's traditional Monte Carlo (Section V-B, Eq. distito): increments
// dW[s][w][n] = sqrt(dt) em_normal(seed, k0 + s, w, n) of samples k0..k0+count-1.
__global__ void em_increments_kernel(uint32_t k0s, uint32_t k1s, int64_t k0, int64_t count, int d, int Nt,
                                     float sqdt, float* __restrict__ dW)
{
    int64_t total = count * (int64_t)d * Nt;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t sw = t / Nt;
        int n = (int)(t - sw * Nt);
        int64_t s = sw / d;
        int w = (int)(sw - s * d);
        dW[t] = sqdt * em_normal((uint32_t)(k0 + s), w, n, k0s, k1s);
    }
}

static int grid_for(int64_t total, int block, int sms)
{
    int64_t g = (total + block - 1) / block;
    int64_t cap = (int64_t)sms * 32;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_lhs_f32(uint64_t seed, int64_t N, int64_t k0, int64_t count, int M, int mode, float* zeta,
                           uint32_t* strata, int sms, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    FeistelShape f = feistel_shape(N);
    int64_t total = count * (int64_t)M;
    lhs_f32_kernel<<<grid_for(total, 256, sms), 256, 0, st>>>((uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)N,
                                                              k0, count, M, mode, f.h, f.mask, zeta, strata);
    return cudaGetLastError();
}

cudaError_t launch_lhs_split(uint64_t seed, int64_t N, int64_t k0, int64_t count, int d, int K, int mode,
                             void* hi, void* lo, int sms, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    FeistelShape f = feistel_shape(N);
    int Ks = round_up(K, 8);
    int64_t total = count * (int64_t)d * Ks;
    lhs_split_kernel<<<grid_for(total, 256, sms), 256, 0, st>>>(
        (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)N, k0, count, d, K, Ks, mode, f.h, f.mask,
        (__nv_bfloat16*)hi, (__nv_bfloat16*)lo);
    return cudaGetLastError();
}

cudaError_t launch_em_increments(uint64_t seed, int64_t k0, int64_t count, int d, int Nt, double dt, float* dW,
                                 int sms, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    int64_t total = count * (int64_t)d * Nt;
    em_increments_kernel<<<grid_for(total, 256, sms), 256, 0, st>>>((uint32_t)seed, (uint32_t)(seed >> 32), k0, count,
                                                                    d, Nt, (float)sqrt(dt), dW);
    return cudaGetLastError();
}

}  // namespace fmc
