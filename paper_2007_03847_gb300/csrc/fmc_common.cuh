// Shared device/host helpers of the fastmc CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fastmc.h"

namespace fmc {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32
// S-box, multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 /
// 0xBB67AE85.  Written here from that published definition.
// ---------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        uint32_t lo1 = 0xCD9E8D57u * c.z;
#else
        uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        U4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// zeta = Phi^-1(p), p = num2 / (N 2^33) given as the exact integer numerator
// num2 = 2 s 2^32 + 2 r + 1 (LHS), 2 s 2^32 + 2^32 (midpoint), 2 r + 1 (SRS, N=1).
// The argument of the CUDA inverse error functions is formed from exact integer
// differences so that it carries FP32 relative accuracy in both tails and at
// the centre:  Phi^-1(p) = -sqrt2 erfcinv(2p) = sqrt2 erfinv(2p - 1)
//            = sqrt2 erfcinv(2(1-p)).
__device__ __forceinline__ float normal_from_fraction(uint64_t num2, uint32_t N)
{
    const uint64_t half = (uint64_t)N << 32;   // den/2
    const float fhalf = (float)N * 4294967296.0f;
    const float SQRT2 = 1.41421356237309515f;
    if (num2 <= (half >> 1)) {                  // p <= 1/4
        float twop = (float)num2 / fhalf;
        return -SQRT2 * erfcinvf(twop);
    }
    uint64_t den = half << 1;
    if (num2 >= den - (half >> 1)) {            // p >= 3/4
        float twoq = (float)(den - num2) / fhalf;
        return SQRT2 * erfcinvf(twoq);
    }
    int64_t c = (int64_t)(num2 - half);         // 2p - 1 = c / half
    return SQRT2 * erfinvf((float)c / fhalf);
}

// The normal of (sample k, disturbance w, step n) of the per-step-normal Monte
// Carlo: Phi^-1((r + 1/2) 2^-32), r = Philox(key, counter (k, n, 256, w / 4))
// word w mod 4 (the tag 256 keeps these counters apart from the design's).
constexpr uint32_t EM_TAG = 256u;

__device__ __forceinline__ float em_normal(uint32_t k, int w, int n, uint32_t k0, uint32_t k1)
{
    const U4 o = philox4x32_10(U4{k, (uint32_t)n, EM_TAG, (uint32_t)(w >> 2)}, k0, k1);
    const uint32_t r = (w & 3) == 0 ? o.x : ((w & 3) == 1 ? o.y : ((w & 3) == 2 ? o.z : o.w));
    return normal_from_fraction(2ull * r + 1ull, 1u);
}

// Packed FP32 (two lanes per register pair) fused multiply-add of sm_100+:
// d = a * b + c elementwise on (x, y) pairs.
__device__ __forceinline__ unsigned long long f2pack(float x, float y)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}

__device__ __forceinline__ void f2unpack(unsigned long long r, float& x, float& y)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(r));
}

__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// The first na of 32 values column[rr * stride] (the rest are ignored) as a
// reference value, their sum about it and their squared deviations from their
// mean, in one pass over shared memory: ref = x_0 (the column's first value),
// dev = sum (x_r - x_0), m2 = sum (x_r - x_0)^2 - dev^2 / na.  x_0 is itself one
// of the values, so dev and the squares stay on the scale of the spread however
// far the values sit from zero, and the sum of the values, na x_0 + dev, is
// never formed in FP32 (its rounding would be on the scale of the values; the
// combines carry x_0 separately).  Four interleaved partials per sum.
__device__ __forceinline__ void column_sums(const float* column, int stride, int na, float* ref, float* dev, float* m2)
{
    const float x0 = column[0];
    float a = 0.f, b = 0.f, c = 0.f, e = 0.f;
    float qa = 0.f, qb = 0.f, qc = 0.f, qe = 0.f;
    if (na == 32) {
        // packed FP32, rows (r, r + 1) in one register pair: d = x * 1 - x0 (exact
        // product, so the same rounding as the subtraction), then the two sums
        const unsigned long long one = f2pack(1.f, 1.f), nx0 = f2pack(-x0, -x0);
        unsigned long long s01 = 0ull, s23 = 0ull, q01 = 0ull, q23 = 0ull;
#pragma unroll
        for (int rr = 0; rr < 32; rr += 4) {
            const unsigned long long d01 = ffma2(f2pack(column[rr * stride], column[(rr + 1) * stride]), one, nx0);
            const unsigned long long d23 =
                ffma2(f2pack(column[(rr + 2) * stride], column[(rr + 3) * stride]), one, nx0);
            s01 = ffma2(d01, one, s01);
            s23 = ffma2(d23, one, s23);
            q01 = ffma2(d01, d01, q01);
            q23 = ffma2(d23, d23, q23);
        }
        f2unpack(s01, a, b);
        f2unpack(s23, c, e);
        f2unpack(q01, qa, qb);
        f2unpack(q23, qc, qe);
    } else {  // the last warp of the last tile only: kept small (not unrolled)
#pragma unroll 1
        for (int rr = 0; rr < 32; rr += 4) {
            const float d0 = rr < na ? column[rr * stride] - x0 : 0.f;
            const float d1 = rr + 1 < na ? column[(rr + 1) * stride] - x0 : 0.f;
            const float d2 = rr + 2 < na ? column[(rr + 2) * stride] - x0 : 0.f;
            const float d3 = rr + 3 < na ? column[(rr + 3) * stride] - x0 : 0.f;
            a += d0;
            b += d1;
            c += d2;
            e += d3;
            qa = fmaf(d0, d0, qa);
            qb = fmaf(d1, d1, qb);
            qc = fmaf(d2, d2, qc);
            qe = fmaf(d3, d3, qe);
        }
    }
    const float sd = (a + b) + (c + e);
    const float sq = (qa + qb) + (qc + qe);
    if (na > 0) {
        *ref = x0;
        *dev = sd;
        *m2 = fmaxf(sq - sd * (sd / (float)na), 0.f);
    } else {
        *ref = 0.f;
        *dev = 0.f;
        *m2 = 0.f;
    }
}

// Samples in group g of 32 when `left` samples remain from group 0 on.
__device__ __forceinline__ int group_count(int64_t left, int g)
{
    const int64_t r = left - 32 * (int64_t)g;
    return r <= 0 ? 0 : (r >= 32 ? 32 : (int)r);
}

// Combines `groups` groups of 32 samples (`left` samples remaining from group 0
// on) given as column_sums triples ref[g], dev[g], m2[g] (strided by `stride`)
// into one triple about the first group's reference c = ref[0]:
//   dev = sum_g (n_g (ref_g - c) + dev_g),
//   m2  = sum_g m2_g + sum_g n_g (mu_g - mu)^2   (Chan, Golub and LeVeque),
// with mu_g - mu = (ref_g - c) + dev_g / n_g - dev / n: every term is on the
// scale of the spread.  Fixed order.
__device__ __forceinline__ void combine_groups(const float* ref, const float* dev, const float* m2, int stride,
                                               int64_t left, int groups, float* c_out, float* dev_out, float* m2_out)
{
    const float c = ref[0];
    if (left >= 32 * (int64_t)groups) {
        // every group full: n_g = 32, and the divisions by 32 are exact products
        float dt = 0.f;
#pragma unroll 1
        for (int g = 0; g < groups; ++g) dt += fmaf(32.f, ref[g * stride] - c, dev[g * stride]);
        const float mu = dt / (float)(32 * groups);
        float acc = 0.f;
#pragma unroll 1
        for (int g = 0; g < groups; ++g) {
            const float dg = (ref[g * stride] - c) + dev[g * stride] * 0.03125f - mu;
            acc += fmaf(32.f * dg, dg, m2[g * stride]);
        }
        *c_out = c;
        *dev_out = dt;
        *m2_out = acc;
        return;
    }
    float dt = 0.f;
    int nt = 0;
#pragma unroll 1
    for (int g = 0; g < groups; ++g) {
        const int ng = group_count(left, g);
        if (ng > 0) dt += fmaf((float)ng, ref[g * stride] - c, dev[g * stride]);
        nt += ng;
    }
    const float mu = nt > 0 ? dt / (float)nt : 0.f;
    float acc = 0.f;
#pragma unroll 1
    for (int g = 0; g < groups; ++g) {
        const int ng = group_count(left, g);
        if (ng > 0) {
            const float dg = (ref[g * stride] - c) + dev[g * stride] / (float)ng - mu;
            acc += fmaf((float)ng * dg, dg, m2[g * stride]);
        }
    }
    *c_out = c;
    *dev_out = dt;
    *m2_out = acc;
}

// Adds a warp's response-function values and their squares into rrf[0], rrf[1]
// (FP64; called by all 32 lanes, inactive lanes passing 0).
__device__ __forceinline__ void rrf_accumulate(float v, double* rrf)
{
    double s1 = v, s2 = (double)v * (double)v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(rrf, s1);
        atomicAdd(rrf + 1, s2);
    }
}

// Device error word written by bounded waits and internal checks.
enum DeviceError : int {
    DEV_OK = 0,
    DEV_TIMEOUT_MMA = 1,
    DEV_TIMEOUT_TMA = 2,
    DEV_BAD_CONFIG = 3,
};

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }
inline int64_t round_up64(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace fmc
