// Diagnostics: the integrator's sin/cos evaluated over given angles (checked
// against CUDA's sincosf and its error bound), and the self-check of the device
// error path of the bounded mbarrier waits.
#include "fmc_common.cuh"
#include "kernels.cuh"
#include "swing.cuh"
#include "tc_common.cuh"

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

// Failure-detection self-check: one thread waits, with the given poll limit, on
// an mbarrier that nothing arrives at (no bulk copy or MMA is in flight), so the
// bounded wait of the production kernels runs out and the kernel records
// DEV_TIMEOUT_MMA in the status word, as they do, and returns.
__global__ void wait_check_kernel(int* err, uint32_t limit)
{
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (!mbar_wait_n(&bar, 0u, limit)) atomicExch(err, DEV_TIMEOUT_MMA);
}

cudaError_t launch_wait_check(int* err, uint32_t limit, cudaStream_t st)
{
    wait_check_kernel<<<1, 32, 0, st>>>(err, limit);
    return cudaGetLastError();
}

}  // namespace fmc
