// The paper's Appendix on the GPU: identification of a scalar Ito model from a
// record xi_0, xi_h, ..., by minimising (Eq. ident)
//   L'(q) = 1/4 sum_j (dxi_j - h mu_j)^2 / D_j + 1/2 sum_j log D_j,
//   D_j = h sigma(xi_j)^2 / 2,
// with mu(x) = q0 + q1 x + q2 x^2 and sigma(x) = q3 + q4 x + q5 x^2 (kind 1,
// the form of Eq. windito) or sigma(x)^2 = q3 + q4 x + q5 x^2 (kind 2, the forms
// of Table I).  One kernel sums L', its gradient and its Hessian over the record
// (FP64, grid-stride, warp shuffles, one FP64 atomic per value and CTA); one
// single-thread kernel solves the shifted Newton system.
#include "fmc_common.cuh"
#include "kernels.cuh"

namespace fmc {

// out: [0] L', [1..6] gradient, [7..42] Hessian (row-major 6 x 6); bad: set to 1
// if some D_j <= 0 (L' is then +infinity).  out and bad zeroed by the caller.
__global__ void __launch_bounds__(256) ito_objective_kernel(int kind, ItoQ q, const double* __restrict__ xi, int64_t n,
                                                            double h, int derivs, double* __restrict__ out,
                                                            int* __restrict__ bad)
{
    constexpr int NV = 1 + 6 + 21;  // L', gradient, upper triangle of the Hessian
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    int badl = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j + 1 < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double x = xi[j];
        const double phi[3] = {1.0, x, x * x};
        const double mu = fma(fma(q.c[2], x, q.c[1]), x, q.c[0]);
        const double sp = fma(fma(q.c[5], x, q.c[4]), x, q.c[3]);
        const double D = kind == 1 ? 0.5 * h * sp * sp : 0.5 * h * sp;
        if (!(D > 0.0)) {
            badl = 1;
            continue;
        }
        const double r = (xi[j + 1] - x) - h * mu;
        const double iD = 1.0 / D;
        acc[0] += 0.25 * r * r * iD + 0.5 * log(D);
        if (!derivs) continue;
        const double lD = 0.5 * iD - 0.25 * r * r * iD * iD;            // d l / d D
        const double lDD = 0.5 * r * r * iD * iD * iD - 0.5 * iD * iD;  // d2 l / d D2
        double g[6], Dq[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Dq[a] = kind == 1 ? h * sp * phi[a] : 0.5 * h * phi[a];
            g[a] = -0.5 * h * r * phi[a] * iD;
            g[3 + a] = lD * Dq[a];
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) acc[1 + a] += g[a];
        int v = 7;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = a; b < 6; ++b, ++v) {
                double hab;
                if (b < 3)
                    hab = 0.5 * h * h * phi[a] * phi[b] * iD;  // drift-drift
                else if (a < 3)
                    hab = 0.5 * h * r * phi[a] * iD * iD * Dq[b - 3];  // drift-diffusion
                else
                    hab = lDD * Dq[a - 3] * Dq[b - 3] + (kind == 1 ? lD * h * phi[a - 3] * phi[b - 3] : 0.0);
                acc[v] += hab;
            }
    }
    // warp sums, then one atomic per value and warp
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double s = acc[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        acc[v] = s;
    }
    if (__any_sync(0xffffffffu, badl) && (threadIdx.x & 31) == 0) atomicExch(bad, 1);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], acc[0]);
        if (derivs) {
            for (int a = 0; a < 6; ++a) atomicAdd(&out[1 + a], acc[1 + a]);
            int v = 7;
            for (int a = 0; a < 6; ++a)
                for (int b = a; b < 6; ++b, ++v) {
                    atomicAdd(&out[7 + a * 6 + b], acc[v]);
                    if (b != a) atomicAdd(&out[7 + b * 6 + a], acc[v]);
                }
        }
    }
}

// step = -(H + lambda I)^-1 g by Cholesky; ok = 0 if the shifted Hessian is
// not positive definite.  One thread.
__global__ void ito_newton_step_kernel(const double* __restrict__ gH, double lambda, double* __restrict__ step,
                                       int* __restrict__ ok)
{
    double Lm[36], b[6];
    const double* g = gH + 1;
    const double* H = gH + 7;
    for (int a = 0; a < 6; ++a) b[a] = -g[a];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) {
            double v = H[i * 6 + j] + (i == j ? lambda : 0.0);
            for (int k = 0; k < j; ++k) v -= Lm[i * 6 + k] * Lm[j * 6 + k];
            if (i == j) {
                if (!(v > 0.0)) {
                    *ok = 0;
                    return;
                }
                Lm[i * 6 + i] = sqrt(v);
            } else {
                Lm[i * 6 + j] = v / Lm[j * 6 + j];
            }
        }
    for (int i = 0; i < 6; ++i) {
        double v = b[i];
        for (int k = 0; k < i; ++k) v -= Lm[i * 6 + k] * b[k];
        b[i] = v / Lm[i * 6 + i];
    }
    for (int i = 5; i >= 0; --i) {
        double v = b[i];
        for (int k = i + 1; k < 6; ++k) v -= Lm[k * 6 + i] * b[k];
        b[i] = v / Lm[i * 6 + i];
    }
    for (int a = 0; a < 6; ++a) step[a] = b[a];
    *ok = 1;
}

cudaError_t launch_ito_objective(int kind, const double* q, const double* xi, int64_t n, double h, int derivs,
                                 double* out, int* bad, int sms, cudaStream_t st)
{
    ItoQ qq;
    for (int a = 0; a < 6; ++a) qq.c[a] = q[a];
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * 43, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    int64_t g = (n + 255) / 256;
    if (g > (int64_t)sms * 8) g = (int64_t)sms * 8;
    if (g < 1) g = 1;
    ito_objective_kernel<<<(unsigned)g, 256, 0, st>>>(kind, qq, xi, n, h, derivs, out, bad);
    return cudaGetLastError();
}

cudaError_t launch_ito_newton_step(const double* gH, double lambda, double* step, int* ok, cudaStream_t st)
{
    ito_newton_step_kernel<<<1, 1, 0, st>>>(gH, lambda, step, ok);
    return cudaGetLastError();
}

}  // namespace fmc
