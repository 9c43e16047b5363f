// Disturbance paths of one time chunk, computed ahead of the integration: the
// disturbances do not depend on the machines, so each sample's path of every
// disturbance over the chunk is formed in one pass and written into TMEM over
// the increments it was made from (column w TC + s: the value at grid index
// n0 + s + 1).  The step loop then reads x_w(t_{n+1}) where it read dW_n, and
// the Euler-Maruyama step of the OU or general Ito disturbance (and, for the
// per-step-normal Monte Carlo, the Philox normals) stay out of the step loop.
// The arithmetic per step is that of ou_step: the same FP32 operations in the
// same order.
#pragma once

#include "fmc_common.cuh"
#include "kernels.cuh"
#include "swing.cuh"
#include "tc_common.cuh"

namespace fmc {

// One disturbance's path over the chunk from its value x at grid index n0, in
// place in its TMEM columns col .. col + steps - 1 (rounded up to 8; TC is a
// multiple of 8, so the rounding stays inside the disturbance's columns).
// Warp-collective.  em.on: the increments are drawn here (sqrt(dt) times the
// normal of (sample k, w, step), em_normal); otherwise they are read from TMEM.
template <int NDI>
__device__ __forceinline__ void disturbance_path_body(uint32_t col, int steps, int n0, int q, float x, float a, float sg,
                                                   const ItoParams<NDI>& it, float dt, const EmSpec& em, uint32_t k)
{
#pragma unroll 1
    for (int s0 = 0; s0 < steps; s0 += 8) {
        float v[8];
        if (em.on) {
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = em.sqdt * em_normal(k, q, n0 + s0 + j, em.key0, em.key1);
        } else {
            tmem_ld8(col + (uint32_t)s0, v);
            tmem_ld_wait();
        }
        if (it.on) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                x = ito_step1<NDI>(it, q, a, sg, x, v[j], dt);
                v[j] = x;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                x = fmaf(a, x, sg * v[j]);
                v[j] = x;
            }
        }
        tmem_st8(col + (uint32_t)s0, v);
    }
}

// The same, not inlined: the caller's registers stay allocated for its step
// loop and the few values live across the call are saved once per chunk (the
// large-system kernel, whose step loop needs every register).
template <int NDI>
__device__ __noinline__ void disturbance_path_call(uint32_t col, int steps, int n0, int q, float x, float a, float sg,
                                                   const ItoParams<NDI>& it, float dt, const EmSpec& em, uint32_t k)
{
    disturbance_path_body<NDI>(col, steps, n0, q, x, a, sg, it, dt, em, k);
}

// The chunk (grid steps n0 .. n0 + steps - 1, TC columns per disturbance) for
// the disturbances w < d with sel < 0 or w mod 4 == sel (warp-uniform), one at
// a time; x0[w]: every disturbance at grid index n0.  Ends with the stores
// complete (tcgen05.wait::st); readers in other warps still need a thread
// barrier between tcgen05 fences.
template <int ND, int NDI, bool INLINE>
__device__ __forceinline__ void disturbance_chunk(uint32_t lane_addr, int TC, int steps, int n0, int d, int sel,
                                                  const float (&x0)[ND], const float* ou_a, const float* ou_s,
                                                  const ItoParams<NDI>& it, float dt, const EmSpec& em, uint32_t k)
{
#pragma unroll 1
    for (int q = sel < 0 ? 0 : sel; q < d && q < ND; q += sel < 0 ? 1 : 4) {
        // the disturbance's value at the chunk start (a select, not an indexed load)
        float x = 0.f;
#pragma unroll
        for (int qq = 0; qq < ND; ++qq)
            if (qq == q) x = x0[qq];
        const uint32_t col = lane_addr + (uint32_t)(q * TC);
        if constexpr (INLINE)
            disturbance_path_body<NDI>(col, steps, n0, q, x, ou_a[q], ou_s[q], it, dt, em, k);
        else
            disturbance_path_call<NDI>(col, steps, n0, q, x, ou_a[q], ou_s[q], it, dt, em, k);
    }
    tmem_st_wait();
}

}  // namespace fmc
