// Test hook: the integrator's sin/cos evaluated over given angles, so that it
// can be checked against CUDA's sincosf and its error bound.
#include "fmc_common.cuh"
#include "kernels.cuh"
#include "swing.cuh"

namespace fmc {

__global__ void sincos_probe_kernel(const float* __restrict__ x, int64_t n, float* __restrict__ s_cw,
                                    float* __restrict__ c_cw, float* __restrict__ s_ref, float* __restrict__ c_ref)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s, c;
    sincos_cw(x[i], &s, &c);
    s_cw[i] = s;
    c_cw[i] = c;
    float s2, c2;
    sincosf(x[i], &s2, &c2);
    s_ref[i] = s2;
    c_ref[i] = c2;
}

cudaError_t launch_sincos_probe(const float* x, int64_t n, float* s_cw, float* c_cw, float* s_ref, float* c_ref,
                                cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    sincos_probe_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, n, s_cw, c_cw, s_ref, c_ref);
    return cudaGetLastError();
}

}  // namespace fmc
