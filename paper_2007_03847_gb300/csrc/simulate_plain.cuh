// Algorithm 1 step 3, plain FP32 form: one thread per sample integrates the OU
// disturbances (Euler-Maruyama, Eq. distito) and the swing equations (RK4 or
// Heun) from increments dW [count][d][Nt] already in HBM, and writes the whole
// trajectory traj [count][Nt+1][2n] back to HBM for a separate moment pass.
#pragma once

#include "fmc_common.cuh"
#include "kernels.cuh"
#include "swing.cuh"

namespace fmc {

template <int NM, int ND>
__global__ void __launch_bounds__(128) simulate_plain_kernel(const __grid_constant__ SwingParams<NM, ND> p,
                                                             const double* __restrict__ eq, const float* __restrict__ dW,
                                                             int64_t count, int Nt, float* __restrict__ traj,
                                                             double* __restrict__ rrf)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = s < count;
    if (!active && rrf == nullptr) return;
    if (!active) s = count - 1;  // computes a duplicate that is neither stored nor counted
    const int n = p.n;
    const int d = p.d;
    float del[NM], w[NM], theta = 0.f;   // deviations from the equilibrium (see swing_step)
    float x0[ND], x1[ND], dw[ND];
#pragma unroll
    for (int i = 0; i < NM; ++i) {
        del[i] = 0.f;
        w[i] = 0.f;
    }
#pragma unroll
    for (int q = 0; q < ND; ++q) x0[q] = 0.f;
    const int64_t row = 2 * (int64_t)n;
    float* out = traj + s * (int64_t)(Nt + 1) * row;
#pragma unroll
    for (int i = 0; i < NM; ++i)
        if (i < n && active) {
            out[i] = p.dst[i];
            out[n + i] = 0.f;
        }
    const float* dws = dW + s * (int64_t)d * Nt;
    float racc = 0.f;  // sum over the grid of the squared centre-of-inertia speed
    for (int step = 0; step < Nt; ++step) {
#pragma unroll
        for (int q = 0; q < ND; ++q) dw[q] = (q < d) ? __ldg(dws + (int64_t)q * Nt + step) : 0.f;
        event_state<NM, ND>(p, step, x0);
        ou_step<NM, ND>(p, x0, dw, x1);
        swing_step<NM, ND>(p, del, w, theta, x0, x1);
#pragma unroll
        for (int q = 0; q < ND; ++q) x0[q] = x1[q];
        const float c = coi_speed<NM, ND>(p, w);
        racc = fmaf(c, c, racc);
        if (!active) continue;
        float* o = out + (int64_t)(step + 1) * row;
#pragma unroll
        for (int i = 0; i < NM; ++i)
            if (i < n) {
                o[i] = (theta + del[i]) + p.dst[i];
                o[n + i] = w[i];
            }
    }
    if (rrf) rrf_accumulate(active ? sqrtf(racc / (float)Nt) : 0.f, rrf);
}

// The smooth form (FMC_FORCING_SMOOTH): the disturbances follow the random ODE
// of Eq. (eqkl), dy/dt = rate(y, f(t)) with the forcing F [count][d][2 Nt + 1]
// at the half-step times (the KL coefficients times the basis functions'
// derivatives), stepped by the same RK4 / Heun stages as the swing equations;
// each swing stage sees the disturbance's own stage value.
template <int NM, int ND>
__global__ void __launch_bounds__(128) simulate_plain_smooth_kernel(const __grid_constant__ SwingParams<NM, ND> p,
                                                                    const float* __restrict__ F, int64_t count,
                                                                    int Nt, float* __restrict__ traj,
                                                                    double* __restrict__ rrf)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = s < count;
    if (!active && rrf == nullptr) return;
    if (!active) s = count - 1;  // computes a duplicate that is neither stored nor counted
    const int n = p.n;
    const int d = p.d;
    float del[NM], w[NM], theta = 0.f;   // deviations from the equilibrium (see swing_step)
    float x0[ND], f0[ND];
    const int64_t J = 2 * (int64_t)Nt + 1;
    const float* fs = F + s * (int64_t)d * J;
#pragma unroll
    for (int i = 0; i < NM; ++i) {
        del[i] = 0.f;
        w[i] = 0.f;
    }
#pragma unroll
    for (int q = 0; q < ND; ++q) {
        x0[q] = 0.f;
        f0[q] = (q < d) ? __ldg(fs + (int64_t)q * J) : 0.f;
    }
    const int64_t row = 2 * (int64_t)n;
    float* out = traj + s * (int64_t)(Nt + 1) * row;
#pragma unroll
    for (int i = 0; i < NM; ++i)
        if (i < n && active) {
            out[i] = p.dst[i];
            out[n + i] = 0.f;
        }
    float racc = 0.f;  // sum over the grid of the squared centre-of-inertia speed
    for (int step = 0; step < Nt; ++step) {
        float xst[4][ND], fh[ND], f1[ND];
#pragma unroll
        for (int q = 0; q < ND; ++q) {
            fh[q] = (q < d) ? __ldg(fs + (int64_t)q * J + 2 * (int64_t)step + 1) : 0.f;
            f1[q] = (q < d) ? __ldg(fs + (int64_t)q * J + 2 * (int64_t)step + 2) : 0.f;
        }
        smooth_stages<NM, ND>(p, step, x0, f0, fh, f1, xst);
#pragma unroll
        for (int q = 0; q < ND; ++q) f0[q] = f1[q];
        swing_step_staged<NM, ND>(p, del, w, theta, xst);
        const float c = coi_speed<NM, ND>(p, w);
        racc = fmaf(c, c, racc);
        if (!active) continue;
        float* o = out + (int64_t)(step + 1) * row;
#pragma unroll
        for (int i = 0; i < NM; ++i)
            if (i < n) {
                o[i] = (theta + del[i]) + p.dst[i];
                o[n + i] = w[i];
            }
    }
    if (rrf) rrf_accumulate(active ? sqrtf(racc / (float)Nt) : 0.f, rrf);
}

// dW: the increments [count][d][Nt], or with smooth the forcing [count][d][2 Nt + 1].
template <int NM, int ND>
cudaError_t launch_plain_t(const void* params, const double* eq, const float* dW, int64_t count, int Nt, float* traj,
                           double* rrf, int smooth, cudaStream_t st)
{
    const SwingParams<NM, ND>& p = *static_cast<const SwingParams<NM, ND>*>(params);
    int64_t g = (count + 127) / 128;
    if (smooth)
        simulate_plain_smooth_kernel<NM, ND><<<(unsigned)g, 128, 0, st>>>(p, dW, count, Nt, traj, rrf);
    else
        simulate_plain_kernel<NM, ND><<<(unsigned)g, 128, 0, st>>>(p, eq, dW, count, Nt, traj, rrf);
    return cudaGetLastError();
}

}  // namespace fmc
