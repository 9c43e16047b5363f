// Algorithm 1 step 2 (Eqs. kl, kle): increment basis of the truncated KL
// expansion, computed in FP64 on the GPU and rounded for the contraction.
//
// Brownian eigenbasis (FMC_BASIS_SINE):
//   phi[k][n] = c_k (sin(a_k t_{n+1}) - sin(a_k t_n)),  a_k = (k+1/2) pi / T,
//   c_k = sqrt(2T) / ((k+1/2) pi),  t_n = n T / Nt,   k = 0..K-1.
// Written without cancellation as a product,
//   phi[k][n] = 2 c_k cos(pi (2k+1)(2n+1) / (4 Nt)) sin(pi (2k+1) / (4 Nt)),
// with the argument of the cosine reduced exactly in integers modulo its period
// (8 Nt in units of pi / (4 Nt)) and evaluated by cospi / sinpi.
//
// The paper's basis of Eq. (klb2) (FMC_BASIS_COSINE), integrated over a step:
//   k = 0:  dt / sqrt(T)  (the constant mode 1/sqrt(T));
//   k >= 1: c_k (sin(a_k t_{n+1}) - sin(a_k t_n)), a_k = k pi / T, c_k = sqrt(2T)/(k pi)
//         = 2 c_k cos(pi k (2n+1) / (2 Nt)) sin(pi k / (2 Nt)),
// the cosine's argument reduced modulo 4 Nt (units of pi / (2 Nt)).
#include <cuda_bf16.h>

#include "fmc_common.cuh"
#include "kernels.cuh"

namespace fmc {

__device__ __forceinline__ double basis_value(int k, int n, int Nt, double T, int basis)
{
    const double PI = 3.141592653589793238462643;
    if (basis == FMC_BASIS_COSINE) {
        if (k == 0) return sqrt(T) / (double)Nt;
        int64_t m = ((int64_t)k * (int64_t)(2 * n + 1)) % (4LL * Nt);
        double c = sqrt(2.0 * T) / ((double)k * PI);
        return 2.0 * c * cospi((double)m / (2.0 * Nt)) * sinpi((double)k / (2.0 * Nt));
    }
    int64_t m = ((int64_t)(2 * k + 1) * (int64_t)(2 * n + 1)) % (8LL * Nt);
    double c = 2.0 * sqrt(2.0 * T) / ((double)(2 * k + 1) * PI);
    return 2.0 * c * cospi((double)m / (4.0 * Nt)) * sinpi((double)(2 * k + 1) / (4.0 * Nt));
}

// phi32 [K][Nt] FP32
__global__ void basis_f32_kernel(int K, int Nt, double T, int basis, float* __restrict__ phi)
{
    int64_t total = (int64_t)K * Nt;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int k = (int)(t / Nt);
        int n = (int)(t - (int64_t)k * Nt);
        phi[t] = (float)basis_value(k, n, Nt, T, basis);
    }
}

// Time-major split BF16 for the tensor-core B operand: hi/lo [Nt][Kpad],
// zeros for k >= K.
__global__ void basis_split_kernel(int K, int Nt, double T, int basis, int Kpad, __nv_bfloat16* __restrict__ hi,
                                   __nv_bfloat16* __restrict__ lo)
{
    int64_t total = (int64_t)Nt * Kpad;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int n = (int)(t / Kpad);
        int k = (int)(t - (int64_t)n * Kpad);
        float v = 0.f;
        if (k < K) v = (float)basis_value(k, n, Nt, T, basis);
        __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[t] = h;
        if (lo) lo[t] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// The forcing of the smooth form (Eq. eqkl as a random ODE): the time
// derivative of the basis function at the half-step times t = j T / (2 Nt),
// j = 0..2 Nt.  Brownian eigenbasis: sqrt(2/T) cos((k+1/2) pi t / T) =
// sqrt(2/T) cospi((2k+1) j / (4 Nt)), the argument reduced modulo 8 Nt; the
// paper's basis: 1/sqrt(T) (k = 0), sqrt(2/T) cospi(k j / (2 Nt)) (mod 4 Nt).
__device__ __forceinline__ double forcing_value(int k, int j, int Nt, double T, int basis)
{
    if (basis == FMC_BASIS_COSINE) {
        if (k == 0) return 1.0 / sqrt(T);
        int64_t m = ((int64_t)k * (int64_t)j) % (4LL * Nt);
        return sqrt(2.0 / T) * cospi((double)m / (2.0 * Nt));
    }
    int64_t m = ((int64_t)(2 * k + 1) * (int64_t)j) % (8LL * Nt);
    return sqrt(2.0 / T) * cospi((double)m / (4.0 * Nt));
}

// mdot [K][2 Nt + 1] FP32
__global__ void forcing_f32_kernel(int K, int Nt, double T, int basis, float* __restrict__ mdot)
{
    const int J = 2 * Nt + 1;
    int64_t total = (int64_t)K * J;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int k = (int)(t / J);
        int j = (int)(t - (int64_t)k * J);
        mdot[t] = (float)forcing_value(k, j, Nt, T, basis);
    }
}

// The forcing basis in the split-BF16 layout of the fused path: time-major
// [2 Nt + 1][Kpad], the K contiguous (the tensor cores' K-major B operand).
__global__ void forcing_split_kernel(int K, int Nt, double T, int basis, int Kpad, __nv_bfloat16* __restrict__ hi,
                                     __nv_bfloat16* __restrict__ lo)
{
    const int64_t total = (2 * (int64_t)Nt + 1) * Kpad;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / Kpad);
        const int k = (int)(t - (int64_t)j * Kpad);
        const float v = k < K ? (float)forcing_value(k, j, Nt, T, basis) : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[t] = h;
        if (lo) lo[t] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

cudaError_t launch_forcing_split(int K, int Nt, double T, int basis, int Kpad, void* hi, void* lo, int sms,
                                 cudaStream_t st)
{
    int64_t total = (2 * (int64_t)Nt + 1) * Kpad;
    int64_t g = (total + 255) / 256;
    if (g > sms * 16) g = sms * 16;
    forcing_split_kernel<<<(int)g, 256, 0, st>>>(K, Nt, T, basis, Kpad, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo);
    return cudaGetLastError();
}

cudaError_t launch_forcing_f32(int K, int Nt, double T, int basis, float* mdot, int sms, cudaStream_t st)
{
    int64_t total = (int64_t)K * (2 * (int64_t)Nt + 1);
    int64_t g = (total + 255) / 256;
    if (g > sms * 16) g = sms * 16;
    forcing_f32_kernel<<<(int)g, 256, 0, st>>>(K, Nt, T, basis, mdot);
    return cudaGetLastError();
}

cudaError_t launch_basis_f32(int K, int Nt, double T, int basis, float* phi, int sms, cudaStream_t st)
{
    int64_t total = (int64_t)K * Nt;
    int64_t g = (total + 255) / 256;
    if (g > sms * 16) g = sms * 16;
    basis_f32_kernel<<<(int)g, 256, 0, st>>>(K, Nt, T, basis, phi);
    return cudaGetLastError();
}

cudaError_t launch_basis_split(int K, int Nt, double T, int basis, int Kpad, void* hi, void* lo, int sms,
                               cudaStream_t st)
{
    int64_t total = (int64_t)Nt * Kpad;
    int64_t g = (total + 255) / 256;
    if (g > sms * 16) g = sms * 16;
    basis_split_kernel<<<(int)g, 256, 0, st>>>(K, Nt, T, basis, Kpad, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo);
    return cudaGetLastError();
}

}  // namespace fmc
