// sm_103a building blocks for the tensor-core KL contraction: mbarriers, TMA
// tile loads, tcgen05 (UMMA) descriptors, MMA issue/commit, TMEM allocation and
// loads.  Inline PTX, written for cta_group::1 with BF16 operands in
// 64-byte-swizzled K-major shared-memory tiles and an FP32 accumulator in TMEM.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "fmc_common.cuh"

namespace fmc {

// Rows of a K block are 32 BF16 = 64 bytes: one row of the 64B swizzle atom
// (8 rows x 64 bytes = 512 bytes).  One MMA consumes K = 16 (32 bytes).
constexpr int TC_BK = 32;
constexpr int TC_M = 128;
constexpr uint32_t TC_ATOM_BYTES = 512;

// Iteration limit of every spin on an mbarrier (each poll sleeps ~64 ns, so
// this is on the order of a second); past it the kernel records a timeout.
constexpr uint32_t TC_WAIT_LIMIT = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.  Returns false
// after `limit` polls.
__device__ __forceinline__ bool mbar_wait_n(uint64_t* bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        __nanosleep(64);
    }
    return false;
}

// The same with the production limit, TC_WAIT_LIMIT polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    return mbar_wait_n(bar, parity, TC_WAIT_LIMIT);
}

// 2-D tiled TMA load of box {x: inner elements, y: rows} into shared memory,
// completing on `bar` with the box's byte count.
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// The same with an L2 cache policy (createpolicy) on the loaded lines.
__device__ __forceinline__ void tma_load_2d_hint(void* smem_dst, const CUtensorMap* map, int x, int y, uint64_t* bar,
                                                 uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, "
        "%3}], [%4], %5;" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// L2 policies: lines kept in preference to others (evict_last), or given up
// first (evict_first).
__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Returns the 128-byte L2 line holding global address a to normal priority.
__device__ __forceinline__ void l2_priority_normal(const void* a)
{
    asm volatile("applypriority.global.L2::evict_normal [%0], 128;" ::"l"(__cvta_generic_to_global(a)) : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Shared-memory matrix descriptor (tcgen05): K-major tile whose rows are 64
// bytes, 64B swizzle, 8-row groups 512 bytes apart.
//   [0,14) start address >> 4, [16,30) leading byte offset >> 4 (unused for a
//   swizzled K-major tile whose MMA K fits in the atom; 1), [32,46) stride byte
//   offset >> 4 (512 B between 8-row groups), [46,49) fixed 0b001,
//   [49,52) base offset 0 (atoms are 512-byte aligned), [61,64) swizzle mode
//   4 = 64-byte swizzle.
__device__ __forceinline__ uint64_t umma_desc_sw64(uint32_t smem_addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(TC_ATOM_BYTES >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B BF16, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4)                      // D format: F32
           | (1u << 7)                    // A format: BF16
           | (1u << 10)                   // B format: BF16
           | ((uint32_t)(N >> 3) << 17)   // N / 8
           | ((uint32_t)(M >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once all previously issued tcgen05.mma of this thread finish.
__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM allocation by one full warp; the base address is written to *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Warp-collective: lane l of the warp receives TMEM lane (base lane + l),
// one 32-bit column.
__device__ __forceinline__ float tmem_ld1(uint32_t taddr)
{
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr) : "memory");
    return __uint_as_float(r);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4])
{
    uint32_t r0, r1, r2, r3;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(taddr)
                 : "memory");
    v[0] = __uint_as_float(r0);
    v[1] = __uint_as_float(r1);
    v[2] = __uint_as_float(r2);
    v[3] = __uint_as_float(r3);
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Warp-collective: eight consecutive 32-bit columns of the warp's 32 lanes,
// loaded into / stored from registers.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------------------
// One [128 x TN] block of dW for disturbance w accumulated into TMEM:
//   D[r][c] = sum_k Z[row0 + r][w*Ks + k] * Phi[col0 + c][k],   k < nkb*32,
// streamed through an ns-stage shared-memory ring in K blocks of 32 (ns - 1
// loads in flight while the tensor cores consume one).  Issued by a single
// thread.  `g` counts K blocks over the kernel's lifetime and selects the ring
// stage (g mod ns) and the mbarrier parities.  Returns false if a bounded wait
// gave up.
// ---------------------------------------------------------------------------
constexpr int TC_MAX_STAGES = 8;

// Dynamic shared memory a fused kernel may request: the opt-in maximum per
// block (227 KB) less the kernels' static shared memory (1 KB with the
// alignment of the dynamic array) and a margin.
constexpr int TC_SMEM_DYN_MAX = 227 * 1024 - 2048;

struct TcRing {
    uint8_t* base;          // ns stages, each: A_hi | A_lo | B_hi | B_lo
    uint64_t* full;         // [ns]
    uint64_t* freed;        // [ns]
    uint32_t a_bytes;       // 128 rows x 64 B
    uint32_t b_bytes;       // TN rows x 64 B
    uint32_t ns;            // stages, 2..TC_MAX_STAGES
    int split;              // 1 for BF16x3 (hi/lo operands present)
    uint64_t a_policy = 0;  // L2 policy of the A (design) loads, or 0: none
};

__device__ __forceinline__ uint32_t ring_stage_bytes(const TcRing& r)
{
    return (r.a_bytes + r.b_bytes) * (r.split ? 2u : 1u);
}

__device__ __forceinline__ bool ring_load(const TcRing& r, uint32_t g, const CUtensorMap* mAh, const CUtensorMap* mAl,
                                          const CUtensorMap* mBh, const CUtensorMap* mBl, int ax, int ay, int bx,
                                          int by)
{
    const uint32_t st = g % r.ns;
    const uint32_t fill = g / r.ns;
    if (fill >= 1) {
        if (!mbar_wait(&r.freed[st], (fill - 1) & 1u)) return false;
    }
    uint8_t* base = r.base + st * ring_stage_bytes(r);
    mbar_arrive_expect_tx(&r.full[st], ring_stage_bytes(r));
    if (r.a_policy)
        tma_load_2d_hint(base, mAh, ax, ay, &r.full[st], r.a_policy);
    else
        tma_load_2d(base, mAh, ax, ay, &r.full[st]);
    tma_load_2d(base + r.a_bytes * (r.split ? 2 : 1), mBh, bx, by, &r.full[st]);
    if (r.split) {
        if (r.a_policy)
            tma_load_2d_hint(base + r.a_bytes, mAl, ax, ay, &r.full[st], r.a_policy);
        else
            tma_load_2d(base + r.a_bytes, mAl, ax, ay, &r.full[st]);
        tma_load_2d(base + r.a_bytes * 2 + r.b_bytes, mBl, bx, by, &r.full[st]);
    }
    return true;
}

__device__ __forceinline__ bool ring_mma(const TcRing& r, uint32_t g, uint32_t d_tmem, uint32_t idesc, bool first)
{
    const uint32_t st = g % r.ns;
    const uint32_t fill = g / r.ns;
    if (!mbar_wait(&r.full[st], fill & 1u)) return false;
    tc_fence_after();
    uint8_t* base = r.base + st * ring_stage_bytes(r);
    const uint32_t a_hi = smem_u32(base);
    const uint32_t b_hi = smem_u32(base + r.a_bytes * (r.split ? 2 : 1));
    const uint32_t a_lo = a_hi + r.a_bytes;
    const uint32_t b_lo = b_hi + r.b_bytes;
#pragma unroll
    for (int ks = 0; ks < TC_BK / 16; ++ks) {
        const uint32_t off = ks * 32;  // 16 BF16 along K inside the 64-byte swizzled row
        uint32_t acc = (first && ks == 0) ? 0u : 1u;
        umma_bf16(d_tmem, umma_desc_sw64(a_hi + off), umma_desc_sw64(b_hi + off), idesc, acc);
        if (r.split) {
            umma_bf16(d_tmem, umma_desc_sw64(a_hi + off), umma_desc_sw64(b_lo + off), idesc, 1u);
            umma_bf16(d_tmem, umma_desc_sw64(a_lo + off), umma_desc_sw64(b_hi + off), idesc, 1u);
        }
    }
    umma_commit(&r.freed[st]);
    return true;
}

}  // namespace fmc
