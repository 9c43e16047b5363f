// Per-sample dynamics of the fused and plain simulation kernels: Euler-Maruyama
// for the OU disturbances and RK4/Heun for the Kron-reduced classical swing
// equations, one CUDA thread per Monte Carlo sample, FP32.
//
// Model (classical machines, Eqs. state/algebra reduced by eliminating the
// network): d delta_i/dt = omega_s domega_i,
//   2 H_i d domega_i/dt = Pm_i + sum_w inj[i][w] x_w - Pe_i - D_i domega_i,
//   Pe_i = sum_j E_i E_j (G_ij cos(delta_i-delta_j) + B_ij sin(delta_i-delta_j))
//          [+ E_i V (Ginf_i cos delta_i + Binf_i sin delta_i)].
// Evaluated in product form: with c_j = cos delta_j, s_j = sin delta_j,
//   Pe_i = c_i u_i + s_i v_i,  u_i = sum_j GE_ij c_j - BE_ij s_j,
//   v_i = sum_j GE_ij s_j + BE_ij c_j,  GE_ij = E_i E_j G_ij, BE_ij = E_i E_j B_ij,
// so a stage costs NM sincos and 4 NM^2 FMAs.  The matrices live in the kernel
// parameter block: fully unrolled loops address them with immediate offsets,
// so every FMA takes its matrix operand straight from the constant bank.
//
// Register economy: a stage evaluates the right-hand side machine by machine and
// immediately folds k_i into the RK accumulator and into the next stage's input,
// so only state, accumulator, stage input and the stage's cos/sin stay live.
// Padded disturbances (index >= d) have zero sigma and zero injection.
#pragma once

#include "fmc_common.cuh"

namespace fmc {

template <int NM, int ND>
struct SwingParams {
    float GE[NM][NM];
    float BE[NM][NM];
    float GEinf[NM];             // E_i Vinf Ginf_i (0 without infinite bus)
    float BEinf[NM];             // E_i Vinf Binf_i
    float inv2H[NM];
    float D[NM];
    float Pm[NM];                // mechanical powers (machine 0's replaced when it is the slack)
    float inj[NM][ND];
    float ou_a[ND];              // 1 - theta_w dt
    float ou_s[ND];              // sigma_w
    float omega_s;
    float dt;
    int d;                       // real disturbances (<= ND; the rest are zero)
    int n;                       // real machines (<= NM; the rest are inert padding)
    int integrator;              // FMC_RK4 / FMC_HEUN
    int slack;                   // 1: machine 0 balances power; its Pm comes from the equilibrium
};

// One step of the swing equations.  The stages run as a loop that is not
// unrolled, so the right-hand side exists once in the code and its constant
// operands are not held in registers across stages.  The disturbance enters
// stage st at x0 + xw (x1 - x0): RK4 xw = 0, 1/2, 1/2, 1 (the midpoint value is
// the average of the two grid values), Heun xw = 0, 1.
template <int NM, int ND>
__device__ __forceinline__ void swing_step(const SwingParams<NM, ND>& p, float pm0, float (&del)[NM], float (&w)[NM],
                                           const float (&x0)[ND], const float (&x1)[ND])
{
    const float dt = p.dt;
    const bool rk4 = (p.integrator == FMC_RK4);
    const int nst = rk4 ? 4 : 2;
    float ad[NM], aw[NM], yd[NM], yw[NM];
#pragma unroll
    for (int i = 0; i < NM; ++i) {
        yd[i] = del[i];
        yw[i] = w[i];
        ad[i] = 0.f;
        aw[i] = 0.f;
    }
#pragma unroll 1
    for (int st = 0; st < nst; ++st) {
        float b, cn, xw;
        if (rk4) {
            b = (st == 1 || st == 2) ? 2.f : 1.f;
            cn = (st == 2) ? dt : 0.5f * dt;
            xw = (st == 0) ? 0.f : ((st == 3) ? 1.f : 0.5f);
        } else {
            b = 1.f;
            cn = dt;
            xw = (st == 0) ? 0.f : 1.f;
        }
        float xs[ND];
#pragma unroll
        for (int q = 0; q < ND; ++q) xs[q] = fmaf(xw, x1[q] - x0[q], x0[q]);
        float c[NM], s[NM];
#pragma unroll
        for (int j = 0; j < NM; ++j) __sincosf(yd[j], &s[j], &c[j]);
#pragma unroll
        for (int i = 0; i < NM; ++i) {
            float u = p.GEinf[i], v = p.BEinf[i];
#pragma unroll
            for (int j = 0; j < NM; ++j) {
                u = fmaf(p.GE[i][j], c[j], u);
                u = fmaf(-p.BE[i][j], s[j], u);
                v = fmaf(p.GE[i][j], s[j], v);
                v = fmaf(p.BE[i][j], c[j], v);
            }
            const float pe = fmaf(c[i], u, s[i] * v);
            float f = (i == 0 && p.slack) ? pm0 : p.Pm[i];
#pragma unroll
            for (int q = 0; q < ND; ++q) f = fmaf(p.inj[i][q], xs[q], f);
            const float kd = p.omega_s * yw[i];
            const float kw = (f - pe - p.D[i] * yw[i]) * p.inv2H[i];
            ad[i] = fmaf(b, kd, ad[i]);
            aw[i] = fmaf(b, kw, aw[i]);
            yd[i] = fmaf(cn, kd, del[i]);
            yw[i] = fmaf(cn, kw, w[i]);
        }
    }
    const float h = rk4 ? dt * (1.0f / 6.0f) : 0.5f * dt;
#pragma unroll
    for (int i = 0; i < NM; ++i) {
        del[i] = fmaf(h, ad[i], del[i]);
        w[i] = fmaf(h, aw[i], w[i]);
    }
}

// One Euler-Maruyama step of the OU disturbances: x1 = (1 - theta dt) x0 + sigma dW.
template <int NM, int ND>
__device__ __forceinline__ void ou_step(const SwingParams<NM, ND>& p, const float (&x0)[ND], const float (&dw)[ND],
                                        float (&x1)[ND])
{
#pragma unroll
    for (int q = 0; q < ND; ++q) x1[q] = fmaf(p.ou_a[q], x0[q], p.ou_s[q] * dw[q]);
}

}  // namespace fmc
