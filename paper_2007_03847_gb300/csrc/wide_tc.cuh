// The network sums of the large-system kernel on the tensor cores.
//
// In every RK stage each machine i of each sample needs
//   du_i = sum_j GE_ij gamma_j - BE_ij eta_j,   dv_i = sum_j BE_ij gamma_j + GE_ij eta_j
// (Sec. II, the Kron-reduced network in the deviation form about the
// equilibrium; GE = E_i E_j G_ij, BE = E_i E_j B_ij, diagonal excluded).  Over
// the 128 samples of a CTA that is one dense product
//   D[128][2n] = A[128][2n] . Net^T,   A = (gamma_j, eta_j) per sample,
// which tcgen05.mma kind::tf32 computes with A in TMEM (one lane per sample,
// written by the threads that own the machines) and Net in shared memory.
// FP32 accuracy comes from the three-term split x = hi + lo of both operands
// (hi = TF32(x), lo = TF32(x - hi)): A_hi Net_hi + A_hi Net_lo + A_lo Net_hi,
// whose dropped terms are below 2^-21 of each product.
//
// Column layout (both the K index of A and the N index of D): slot
// c = h KH + 2 k + {0: gamma / du, 1: eta / dv} for machine i = h + H k (H warps
// per sample: 4, or 2 for two CTAs per SM), with KH = 2 NMT rounded up to a
// multiple of 4, so that every warp (q, h) reads and writes whole 16-byte groups
// of its own columns.  NN = H KH columns rounded up to a multiple of 16 (the
// MMA's N and K granularity); the padding columns of A are zero.
#pragma once

#include <cuda.h>
#include <cstdint>

#include "kernels.cuh"
#include "tc_common.cuh"

namespace fmc {

__host__ __device__ constexpr int wide_kh(int nmt) { return (2 * nmt + 3) & ~3; }
__host__ __device__ constexpr int wide_nn(int nmt, int H = 4) { return (H * wide_kh(nmt) + 15) & ~15; }

// Machine-slot buckets the tensor-core network sum is built for (13 .. 52 machines).
__host__ __device__ constexpr bool wide_tc_built(int nmt)
{
    return nmt == 4 || nmt == 5 || nmt == 7 || nmt == 10 || nmt == 13;
}

// Up to 7 slots (28 machines) the stage inputs alternate between two A buffers,
// so that the angle half of a stage (which needs no network sum) can publish the
// next input while the tensor cores still read the current one.
__host__ __device__ constexpr bool wide_tc_abuf2(int nmt, int H = 4) { return H == 4 && nmt <= 7; }

// TMEM columns the network sum takes past the disturbance columns: A_hi, A_lo, D
// (then A_hi, A_lo of the second buffer).
__host__ __device__ constexpr int wide_tc_cols(int nmt, int H = 4)
{
    return (wide_tc_abuf2(nmt, H) ? 5 : 3) * wide_nn(nmt, H);
}

// Shared-memory bytes of Net_hi and Net_lo: per matrix NN / 16 K blocks of NN
// rows x 64 bytes (16 TF32 values), 64-byte swizzle, as one TMA box each.
__host__ __device__ constexpr int wide_tc_net_bytes(int nmt, int H = 4)
{
    return 2 * wide_nn(nmt, H) * wide_nn(nmt, H) * 4;
}

// Instruction descriptor of tcgen05.mma kind::tf32: D FP32, A and B TF32 (FP32
// bit patterns), both K-major, shape M x N.
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N)
{
    return (1u << 4)                      // D format: F32
           | (2u << 7)                    // A format: TF32
           | (2u << 10)                   // B format: TF32
           | ((uint32_t)(N >> 3) << 17)   // N / 8
           | ((uint32_t)(M >> 4) << 24);  // M / 16
}

#ifdef __CUDACC__
// D (+)= A B^T over K = 8: A is 128 x 8 TF32 in TMEM (lane = row, one 32-bit
// column per k, from column a_tmem), B is N x 8 from a shared-memory descriptor.
__device__ __forceinline__ void umma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                             uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// FP32 rounded to TF32 (nearest, ties away from zero), as an FP32 bit pattern.
__device__ __forceinline__ uint32_t tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Warp-collective: four consecutive 32-bit columns of the warp's 32 lanes.
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v0), "r"(v1),
                 "r"(v2), "r"(v3)
                 : "memory");
}

// One stage's network product, issued by a single thread:
//   D = A_lo Net_hi^T + A_hi Net_lo^T + A_hi Net_hi^T   (K = NN, 8 per MMA).
// The two small correction terms go first, while the accumulator is small, so
// that only the last NN / 8 MMAs add to a full-size accumulator.
// net: shared address of Net_hi's first K block; Net_lo follows after NN/16 blocks.
template <int NMT, int H>
__device__ __forceinline__ void net_mma(uint32_t d_tmem, uint32_t ahi_tmem, uint32_t alo_tmem, uint32_t net)
{
    constexpr int NN = wide_nn(NMT, H);
    constexpr uint32_t KB_BYTES = NN * 64;  // one K block: NN rows of 64 bytes
    constexpr uint32_t LO = (NN / 16) * KB_BYTES;
    constexpr uint32_t idesc = umma_idesc_tf32(TC_M, NN);
#pragma unroll
    for (int ks = 0; ks < NN / 8; ++ks) {
        const uint32_t off = (uint32_t)(ks >> 1) * KB_BYTES + (uint32_t)(ks & 1) * 32u;
        umma_tf32_ts(d_tmem, alo_tmem + 8u * ks, umma_desc_sw64(net + off), idesc, ks > 0 ? 1u : 0u);
    }
#pragma unroll
    for (int ks = 0; ks < NN / 8; ++ks) {
        const uint32_t off = (uint32_t)(ks >> 1) * KB_BYTES + (uint32_t)(ks & 1) * 32u;
        umma_tf32_ts(d_tmem, ahi_tmem + 8u * ks, umma_desc_sw64(net + LO + off), idesc, 1u);
    }
#pragma unroll
    for (int ks = 0; ks < NN / 8; ++ks) {
        const uint32_t off = (uint32_t)(ks >> 1) * KB_BYTES + (uint32_t)(ks & 1) * 32u;
        umma_tf32_ts(d_tmem, ahi_tmem + 8u * ks, umma_desc_sw64(net + off), idesc, 1u);
    }
}

// Bounded wait for a stage's product: polls without sleeping first (the product
// takes well under a microsecond, and a sleep would delay the wake-up), then with
// the production limit and its sleeps.
__device__ __forceinline__ bool net_wait(uint64_t* bar, uint32_t parity)
{
    for (int it = 0; it < 4096; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return mbar_wait(bar, parity);
}

// Warp-collective: four (gamma, eta) values of a pair of machines, split into
// TF32 hi and lo, to columns col .. col + 3 of A_hi and A_lo (the caller waits
// for the stores with tmem_st_wait before the next product).
__device__ __forceinline__ void net_store4(uint32_t hi_addr, uint32_t lo_addr, int col, float v0, float v1, float v2,
                                           float v3)
{
    const float v[4] = {v0, v1, v2, v3};
    uint32_t hv[4], lv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        hv[c] = tf32_rna(v[c]);
        lv[c] = tf32_rna(v[c] - __uint_as_float(hv[c]));
    }
    tmem_st4(hi_addr + (uint32_t)col, hv[0], hv[1], hv[2], hv[3]);
    tmem_st4(lo_addr + (uint32_t)col, lv[0], lv[1], lv[2], lv[3]);
}

// Warp-collective: columns c0 .. c0 + W - 1 (W a multiple of 4) of the warp's
// D, A_hi and A_lo columns: du, dv of machines c0 / 2 .. and the (gamma, eta)
// hi and lo parts the product was formed from.
template <int W>
__device__ __forceinline__ void net_read(uint32_t d_addr, uint32_t hi_addr, uint32_t lo_addr, int c0, float (&dd)[W],
                                         float (&ah)[W], float (&al)[W])
{
#pragma unroll
    for (int c = 0; c < W; c += 4) {
        float v[4];
        tmem_ld4(d_addr + (uint32_t)(c0 + c), v);
        dd[c] = v[0];
        dd[c + 1] = v[1];
        dd[c + 2] = v[2];
        dd[c + 3] = v[3];
        tmem_ld4(hi_addr + (uint32_t)(c0 + c), v);
        ah[c] = v[0];
        ah[c + 1] = v[1];
        ah[c + 2] = v[2];
        ah[c + 3] = v[3];
        tmem_ld4(lo_addr + (uint32_t)(c0 + c), v);
        al[c] = v[0];
        al[c + 1] = v[1];
        al[c + 2] = v[2];
        al[c + 3] = v[3];
    }
    tmem_ld_wait();
}
#endif

// The large-system kernel with the tensor-core network sum.  nmt: machine slots
// per thread for H warps per sample (4: one 512-thread CTA per SM; 2: two
// 256-thread CTAs per SM, each with half the SM's TMEM).  maps: the four
// contraction maps, then the map of Net (FP32 [2 NN][NN]: Net_hi rows, then
// Net_lo rows; box 16 x NN, 64-byte swizzle).  a.tmem_cols must be 512 / (4 / H)
// and hold the disturbance columns d TC (rounded up to 16) plus
// wide_tc_cols(nmt, H).
// bus: the system has an infinite bus (then H = 4 and nd = 8, and the last
// machine slot must be free: n < 4 nmt).
cudaError_t launch_simulate_wide_tc(int nmt, int H, int nd, bool bus, const CUtensorMap* maps, const WideArgs& a,
                                    cudaStream_t st, int* max_ctas_per_sm);

}  // namespace fmc
