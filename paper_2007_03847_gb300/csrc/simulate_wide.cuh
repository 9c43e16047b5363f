// Algorithm 1 steps 2-4 fused for systems too large to keep one sample's whole
// state in one thread (17..52 machines); smaller systems on request.
//
// One CTA = 128 samples = 128 TMEM lanes, 4 H warps (H = 4, or 2 with two CTAs
// per SM).  Warp (q, h) = (w mod 4, w / 4) integrates the machines i = h + H k
// (k < NMT) of the 32 samples whose TMEM lanes it may read (subpartition q), so
// H warps share every sample and each thread holds 1/H of its sample's state.
// The KL contraction into TMEM is the fused kernel's (one thread issues TMA
// loads and tcgen05.mma per time chunk); the warps of a sample group then turn
// the increments into the chunk's disturbance paths in place in TMEM (warp h
// the disturbances w = h mod 4, and h + 2 mod 4 when H = 2), and all of them
// read every path.
//
// The network sums of an RK stage need, for every machine j, the deviations
//   gamma_j = cos(D*_j + Delta_j) - cos D*_j,  eta_j = sin(D*_j + Delta_j) - sin D*_j
// of the stage input.  FP32 form (TCN false): every thread publishes its
// machines' (gamma, eta) to shared memory (double-buffered, so one named barrier
// of the 128 threads of a sample group per stage suffices), then accumulates the
// sums of its machines over all j, the network matrices laid out [j][h][k] in
// shared memory (k padded to a multiple of 4) so that a warp reads its column
// slice with broadcast 16-byte loads.  Tensor-core form (TCN, wide_tc.cuh): the
// (gamma, eta) go to TMEM and one tcgen05 TF32x3 product per stage forms the sums
// of all 128 samples; the deviations are taken less their per-sample mean, and
// an infinite bus (BUS) is a network node in the last machine slot.  The
// arithmetic per machine is that of swing_step (deviation form around the FP64
// equilibrium, diagonal excluded).
#pragma once

#include "fmc_common.cuh"
#include "kernels.cuh"
#include "swing.cuh"
#include "tc_common.cuh"
#include "disturb_chunk.cuh"
#include "wide_tc.cuh"

namespace fmc {

constexpr int WI_THREADS = 512;
constexpr int WI_MS = 4;  // steps between flushes of the moment buffer

// Moment buffers of a CTA of H warps per sample (4 H warps): per-warp transposes,
// the (step, sample group, h) triples, the per-step centre-of-inertia partials.
template <int NMT, int H = 4>
__host__ __device__ inline int wide_mom_floats()
{
    return 4 * H * 32 * (2 * NMT + 1) + WI_MS * 4 * H * 6 * NMT + WI_MS * H * 128;
}

// sin and cos - 1 of a deviation, rotated into (gamma, eta) about the equilibrium.
__device__ __forceinline__ float2 wide_gamma_eta(float x, float cs, float ss, bool big)
{
    float sn, cm1;
    if (big)
        sin_cosm1_any(x, &sn, &cm1);
    else
        sin_cosm1_small(x, &sn, &cm1);
    return make_float2(fmaf(cs, cm1, -ss * sn), fmaf(ss, cm1, cs * sn));
}

// Warp-collective: the same with the series degree chosen from the warp's
// largest |x| over the lanes where `use` holds (the tiers and their truncation
// bounds of swing.cuh: 3/4 up to 0.05, 5/6 up to 0.25, 9/10 up to 0.8, then the
// reduced-argument form).  Magnitudes compare as their FP32 bit patterns.
__device__ __forceinline__ float2 wide_gamma_eta_tier(float x, float cs, float ss, bool use)
{
    const uint32_t m = __reduce_max_sync(0xffffffffu, use ? __float_as_uint(fabsf(x)) : 0u);
    float sn, cm1;
    if (m <= __float_as_uint(0.05f))
        sin_cosm1_tiny(x, &sn, &cm1);
    else if (m <= __float_as_uint(0.25f))
        sin_cosm1_mid(x, &sn, &cm1);
    else if (m <= __float_as_uint(0.8f))
        sin_cosm1_small(x, &sn, &cm1);
    else
        sin_cosm1_any(x, &sn, &cm1);
    return make_float2(fmaf(cs, cm1, -ss * sn), fmaf(ss, cm1, cs * sn));
}

// cos c - 1 and sin c of an infinite bus's shift (a call, not inlined: only the
// warp that holds the bus's slot of a system with an infinite bus takes it, and
// the hot loops keep their registers).
static __device__ __noinline__ void bus_deviation(float c, float* cm1, float* sn) { sin_cosm1_any(c, sn, cm1); }

// Warp-collective (tensor-core network sum): (gamma, eta) of the deviations
// x[k] - csh of the warp's machines by the series of tier TIER, split and stored
// pairwise to the warp's A_hi, A_lo columns; waits for the stores.  Slot nb (an
// infinite bus, or -1) takes the bus's (bcm, -bsn) = (cos csh - 1, -sin csh).
template <int NMT, int TIER, int CST, int H>
__device__ __forceinline__ void publish_tier(uint32_t hi, uint32_t lo, const float (&x)[NMT], float csh,
                                             const float* cst_s, int h, int n, int nb, float bcm, float bsn)
{
    float pg = 0.f, pe = 0.f;
#pragma unroll
    for (int k = 0; k < NMT; ++k) {
        const int i = h + H * k;
        const float2 csn = *reinterpret_cast<const float2*>(cst_s + i * CST);
        float sn, cm1;
        deviation_trig1<TIER>(x[k] - csh, &sn, &cm1);
        const bool bus = k == NMT - 1 && i == nb;  // (the bus holds a warp's last slot)
        const float gx = i < n ? fmaf(csn.x, cm1, -csn.y * sn) : (bus ? bcm : 0.f);
        const float ex = i < n ? fmaf(csn.y, cm1, csn.x * sn) : (bus ? -bsn : 0.f);
        if (k & 1)
            net_store4(hi, lo, 2 * (k - 1), pg, pe, gx, ex);
        else if (k == NMT - 1)
            net_store4(hi, lo, 2 * k, gx, ex, 0.f, 0.f);
        pg = gx;
        pe = ex;
    }
    tmem_st_wait();
}

// The same with one tier for all of the warp's machines, from their largest
// shifted deviation (the tiers of wide_gamma_eta_tier).
template <int NMT, int CST, int H>
__device__ __forceinline__ void publish_angles(uint32_t hi, uint32_t lo, const float (&x)[NMT], float csh,
                                               const float* cst_s, int h, int n, int nb)
{
    float bcm = 0.f, bsn = 0.f;
    if (nb >= 0 && nb % H == h) bus_deviation(csh, &bcm, &bsn);
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < NMT; ++k)
        if (h + H * k < n) m = fmaxf(m, fabsf(x[k] - csh));
    const uint32_t mm = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
    if (mm <= __float_as_uint(0.05f))
        publish_tier<NMT, 0, CST, H>(hi, lo, x, csh, cst_s, h, n, nb, bcm, bsn);
    else if (mm <= __float_as_uint(0.25f))
        publish_tier<NMT, 1, CST, H>(hi, lo, x, csh, cst_s, h, n, nb, bcm, bsn);
    else if (mm <= __float_as_uint(0.8f))
        publish_tier<NMT, 2, CST, H>(hi, lo, x, csh, cst_s, h, n, nb, bcm, bsn);
    else
        publish_tier<NMT, 3, CST, H>(hi, lo, x, csh, cst_s, h, n, nb, bcm, bsn);
}

// TCN: the network sums on the tensor cores (wide_tc.cuh) instead of the FP32
// pipes; the per-machine arithmetic around them is the same.  H: warps per sample
// (4; or 2 with TCN: two CTAs of 256 threads per SM), machine i = h + H k.
// BUS (with TCN): the system has an infinite bus, held in the last machine slot.
template <int NMT, int ND, bool TCN, int H = 4, bool BUS = false>
__global__ void __launch_bounds__(H * 128, 4 / H)
    simulate_wide_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                         const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                         const __grid_constant__ CUtensorMap mN, const __grid_constant__ WideArgs a)
{
    constexpr int NMTP = wide_nmtp(NMT);
    constexpr int KP = NMT > 10 ? 8 : NMT;  // machine slots per pass over the network sum
    constexpr int JU = NMT > 5 ? 2 : 4;  // unrolling of the loop over j (measured; registers)
    // every pass starts its 16-byte loads of the matrix rows at slot k0, a multiple of KP
    static_assert(KP >= NMT || KP % 4 == 0, "network passes must start on 16-byte boundaries");
    constexpr bool PACK = wide_packed(NMT);  // the BE rows hold -BE when packed, BE otherwise
    constexpr int G4 = 4 * NMT;
    constexpr int WROW = 2 * NMT + 1;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1 KB alignment by an offset from the shared array itself (not through an
    // integer round trip), so that every access through these pointers stays a
    // shared-memory access rather than a generic one
    uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ uint64_t bars[2 * TC_MAX_STAGES + 3];  // full[ns], freed[ns], done, net, net load
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int q = warp & 3, h = warp >> 2;
    const int n = a.n, d = a.d, S = 2 * n, S3 = 3 * S;
    constexpr int GS = 6 * NMT;  // floats per (step, sample group, h) slot: ref | dev | m2 of 2 NMT states
    const int r = 32 * q + lane;  // sample row within the tile = TMEM lane
    const int64_t row0 = (int64_t)blockIdx.x * TC_M;
    const int64_t srow = row0 + r;
    const bool active = srow < a.count;
    const int TC = a.TC;
    static_assert(H == 4 || (H == 2 && TCN), "two warps per sample with the tensor-core network sum only");
    constexpr int NTHR = H * 128;
    constexpr int NN = wide_nn(NMT, H);
    // TCN: TMEM columns of A_hi, A_lo and D past the disturbance columns
    const uint32_t net0 = (uint32_t)((d * TC + 15) & ~15);
    if (TCN && net0 + (uint32_t)wide_tc_cols(NMT, H) > a.tmem_cols) {
        if (tid == 0) atomicExch(a.err, DEV_BAD_CONFIG);
        return;
    }

    // shared memory: [ring | moment buffers] [gamma/eta x2] [w0 x2] [constants]
    TcRing ring;
    ring.a_bytes = TC_M * 64;
    ring.b_bytes = TC * 64;
    ring.split = a.split;
    const uint32_t stage_bytes = (ring.a_bytes + ring.b_bytes) * (a.split ? 2 : 1);
    ring.base = smem;
    ring.ns = (uint32_t)a.ns;
    ring.full = &bars[0];
    ring.freed = &bars[TC_MAX_STAGES];
    uint64_t* done = &bars[2 * TC_MAX_STAGES];
    const uint32_t mom_bytes = (uint32_t)wide_mom_floats<NMT, H>() * 4u;
    const uint32_t ring_bytes = (uint32_t)a.ns * stage_bytes;
    const uint32_t u_bytes = ((ring_bytes > mom_bytes ? ring_bytes : mom_bytes) + 1023u) & ~1023u;
    float* wbuf = reinterpret_cast<float*>(smem) + warp * 32 * WROW;   // [32][WROW] per warp
    float* msum = reinterpret_cast<float*>(smem) + 4 * H * 32 * WROW;  // [WI_MS][q][h][GS]
    // TCN: Net_hi | Net_lo (1 KB aligned); else the (gamma, eta) exchange [2][n][128]
    uint8_t* net_s = smem + u_bytes;
    float2* gh = reinterpret_cast<float2*>(smem + u_bytes);
    float* w0buf = TCN ? reinterpret_cast<float*>(net_s + wide_tc_net_bytes(NMT, H))
                       : reinterpret_cast<float*>(gh + 2 * n * 128);  // [2][128]
    float* racc_s = w0buf + 256;                                        // [128] (warps h = 0)
    // TCN: [2][4 (h)][128] partial sums of a stage input's deviations over the warp's machines
    float* cpart = w0buf + 384;
    float* cst_s = w0buf + 384 + (TCN ? 1024 : 0);
    const int dx = a.dx;
    // TCN keeps only the per-machine rows (the network is in net_s), transposed to
    // [4 NMT][CST] so that a machine's constants are a few 16-byte loads:
    // (cos D*, sin D*, u*, v*), (delta*, 1/(2H), D, H / sum H), injection row
    constexpr int CST = (8 + ND + 3) & ~3;
    const int nskip = TCN ? 2 * n * 4 * NMTP : 0;
    const int nconst = wide_const_floats(n, NMT, ND) - nskip;
    for (int e = tid; e < nconst; e += NTHR) {
        if (TCN) {
            const int row = e / G4, i = e - row * G4;
            cst_s[i * CST + row] = a.consts[nskip + e];
        } else {
            cst_s[e] = a.consts[nskip + e];
        }
    }
    // [j][h][GE row of NMTP | BE row of NMTP]: one address serves both rows
    const float* GB = cst_s;
    const float* pm = cst_s + 2 * n * 4 * NMTP - nskip;
    const float* c_cst = pm;
    const float* c_sst = pm + G4;
    const float* c_ust = pm + 2 * G4;
    const float* c_vst = pm + 3 * G4;
    const float* c_i2h = pm + 5 * G4;
    const float* c_D = pm + 6 * G4;
    const float* c_inj = pm + 8 * G4;  // [dx][4 NMT]
    // constant `row` (0 cos D*, 1 sin D*, 2 u*, 3 v*, 4 delta*, 5 1/(2H), 6 D, 7 H / sum H,
    // 8.. injection) of machine slot i, in either layout
    auto cst = [&](int row, int i) -> float { return TCN ? cst_s[i * CST + row] : pm[row * G4 + i]; };
    // per step and warp, the partial centre-of-inertia speed of the warp's machines
    float* coi_part = msum + WI_MS * 4 * H * GS;  // [WI_MS][H (h)][128]

    const bool em = a.em.on != 0;
    uint64_t* netbar = &bars[2 * TC_MAX_STAGES + 1];
    uint64_t* netld = &bars[2 * TC_MAX_STAGES + 2];
    if (tid == 0) {
        if (!em) {
            prefetch_tmap(&mAh);
            prefetch_tmap(&mBh);
        }
        for (int b = 0; b < 2 * TC_MAX_STAGES + 3; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init();
        abort_flag = 0;
        if (TCN) {
            // Net_hi and Net_lo, one box of NN rows per K block of 16 values
            mbar_arrive_expect_tx(netld, (uint32_t)wide_tc_net_bytes(NMT, H));
            for (int kb = 0; kb < NN / 16; ++kb) {
                tma_load_2d(net_s + kb * NN * 64, &mN, kb * 16, 0, netld);
                tma_load_2d(net_s + (NN / 16 + kb) * NN * 64, &mN, kb * 16, NN, netld);
            }
        }
    }
    if (warp == 0) tmem_alloc(&tmem_base, a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
    // TCN: this warp's columns of A_hi, A_lo (buffer 0; AB2: buffer 1 at +3 NN) and D
    constexpr bool AB2 = TCN && wide_tc_abuf2(NMT, H);
    const uint32_t a_hi = lane_addr + net0 + (uint32_t)(h * wide_kh(NMT));
    const uint32_t a_lo = a_hi + NN, a_d = a_hi + 2 * NN;
    int bad = 0;          // TCN: a bounded wait of this thread gave up
    bool failed = false;  // TCN: the CTA stops (uniform)
    uint32_t nph = 0;     // TCN: parity of the network product's barrier
    if (TCN && tid == 0 && !mbar_wait(netld, 0)) {
        bad = 1;
        atomicExch(a.err, DEV_TIMEOUT_TMA);
    }

    float del[NMT], w[NMT], theta = 0.f;  // deviations from the equilibrium
    float x0[ND];
#pragma unroll
    for (int k = 0; k < NMT; ++k) {
        del[k] = 0.f;
        w[k] = 0.f;
    }
#pragma unroll
    for (int e = 0; e < ND; ++e) x0[e] = 0.f;

    const int64_t trow = 2 * (int64_t)n;
    float* traj = (a.traj != nullptr && active) ? a.traj + srow * (int64_t)(a.Nt + 1) * trow : nullptr;
    if (traj) {
#pragma unroll
        for (int k = 0; k < NMT; ++k) {
            const int i = h + H * k;
            if (i < n) {
                traj[i] = cst(4, i);
                traj[n + i] = 0.f;
            }
        }
    }
    float* part_tile = a.part ? a.part + (int64_t)blockIdx.x * (a.Nt + 1) * S3 : nullptr;
    if (part_tile)
        for (int v = tid; v < S3; v += NTHR) part_tile[v] = 0.f;

    // stage-0 input of the first step: every deviation is zero
    int gb = 0;
    // TCN: the deviations enter the trigonometric terms less their per-sample mean
    // (of the previous stage input; the electrical power depends on angle
    // differences alone, so any common shift is exact), which keeps the product's
    // inputs, and so its rounding, at the size of the machines' relative motion.
    // An infinite bus is one more node at angle 0, so at -csh in the shifted
    // frame: the last machine slot nb = H NMT - 1 (unused: the host takes this
    // layout only when n < H NMT) carries its (cos csh - 1, -sin csh), and the
    // network matrix its column.
    float csh = 0.f;
    const float inv_n = 1.0f / (float)n;
    const int nb = BUS ? H * NMT - 1 : -1;  // (BUS: built for systems with an infinite bus)
    if constexpr (TCN) {
#pragma unroll
        for (int k = 0; k < NMT; k += 2) net_store4(a_hi, a_lo, 2 * k, 0.f, 0.f, 0.f, 0.f);
        // A's columns past the H KH in use (NN is a multiple of 16) stay zero
        if (h == H - 1)
            for (int c = H * wide_kh(NMT); c < NN; c += 4)
                net_store4(lane_addr + net0, lane_addr + net0 + NN, c, 0.f, 0.f, 0.f, 0.f);
        tmem_st_wait();
        cpart[h * 128 + r] = 0.f;
    } else {
#pragma unroll
        for (int k = 0; k < NMT; ++k) {
            const int i = h + H * k;
            if (i < n) gh[i * 128 + r] = make_float2(0.f, 0.f);
        }
    }
    if (h == 0) w0buf[r] = 0.f;

    const uint32_t idesc = umma_idesc_bf16(TC_M, TC);
    uint32_t g = 0;
    const int J = d * a.nkb;
    const float dt = a.dt;
    const bool rk4 = (a.integrator == FMC_RK4);
    const int nst = rk4 ? 4 : 2;
    const float ref = a.rel ? 1.f : 0.f;
    const float hh = rk4 ? dt * (1.0f / 6.0f) : 0.5f * dt;
    // (warps h = 0) sum over the grid of the squared centre-of-inertia speed, kept
    // in shared memory: it is touched only at the flushes, and a register held
    // across the step loop costs the network sums more than the round trips
    if (h == 0) racc_s[r] = 0.f;

    for (int c = 0, n0 = 0; n0 < a.Nt; ++c, n0 += TC) {
        // ---- tensor cores: dW of this chunk into TMEM ----
        if (!em) {
        tc_fence_before();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            bool ok = ring_load(ring, g, &mAh, &mAl, &mBh, &mBl, 0, (int)row0, 0, n0);
            for (int j = 0; j < J && ok; ++j) {
                if (j + 1 < J) {
                    const int w1 = (j + 1) / a.nkb, kb1 = (j + 1) % a.nkb;
                    ok = ring_load(ring, g + j + 1, &mAh, &mAl, &mBh, &mBl, w1 * a.Ks + kb1 * TC_BK, (int)row0,
                                   kb1 * TC_BK, n0);
                }
                const int wj = j / a.nkb, kbj = j % a.nkb;
                if (ok) ok = ring_mma(ring, g + j, tmem + (uint32_t)(wj * TC), idesc, kbj == 0);
            }
            g += (uint32_t)J;
            if (ok) {
                umma_commit(done);
            } else {
                abort_flag = 1;
                atomicExch(a.err, DEV_TIMEOUT_TMA);
            }
        }
        __syncthreads();
        bool ok = (abort_flag == 0);
        if (ok && !mbar_wait(done, (uint32_t)c & 1u)) {
            ok = false;
            atomicExch(a.err, DEV_TIMEOUT_MMA);
        }
        if (!__syncthreads_and(ok)) break;
        tc_fence_after();
        }

        // ---- disturbance paths of this chunk into TMEM ----
        // the four warps of a sample group share its lanes: warp h forms the
        // disturbances w = h mod 4, then all of them read all of them
        const int steps = (a.Nt - n0) < TC ? (a.Nt - n0) : TC;
        if (em) {  // (with the contraction, the barrier above already separates the chunks)
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        }
        // (warp h forms the disturbances w = h mod 4; with two warps per sample,
        // also w = h + 2 mod 4)
        disturbance_chunk<ND, 8, false>(lane_addr, TC, steps, n0, d, h, x0, a.ou_a, a.ou_s, a.ito, dt, a.em,
                                 (uint32_t)(a.em.k0 + srow));
        if (H == 2)
            disturbance_chunk<ND, 8, false>(lane_addr, TC, steps, n0, d, h + 2, x0, a.ou_a, a.ou_s, a.ito, dt, a.em,
                                            (uint32_t)(a.em.k0 + srow));
        tc_fence_before();
        __syncthreads();
        tc_fence_after();

        // ---- FP32 pipes: integrate this chunk ----
        for (int s = 0; s < steps; ++s) {
            float x1[ND];
#pragma unroll
            for (int e = 0; e < ND; ++e) x1[e] = 0.f;
#pragma unroll
            for (int e = 0; e < ND; ++e)
                if (e < d) x1[e] = tmem_ld1(lane_addr + (uint32_t)(e * TC + s));
            tmem_ld_wait();
#pragma unroll
            for (int e = 0; e < ND; ++e)  // the event slot (index d) is 0 before the event, 1 from it
                if (e == d && dx > d) {
                    x0[e] = (n0 + s >= a.ev_step) ? 1.f : 0.f;
                    x1[e] = x0[e];
                }

            float ad[NMT], aw[NMT], yw[NMT];
            float ath = 0.f;
#pragma unroll
            for (int k = 0; k < NMT; ++k) {
                yw[k] = w[k];
                ad[k] = 0.f;
                aw[k] = 0.f;
            }
if constexpr (TCN) {
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
                // A buffers of this stage's input and of the next
                const uint32_t ab = AB2 && gb ? 3u * NN : 0u, an = AB2 && !gb ? 3u * NN : 0u;
                // every warp's A columns of this stage's input are written and
                // every read of the previous product is done
                tc_fence_before();
                if (__syncthreads_or(bad)) {
                    failed = true;
                    break;
                }
                if (tid == 0) {
                    tc_fence_after();
                    net_mma<NMT, H>(tmem + net0 + 2 * NN, tmem + net0 + ab, tmem + net0 + ab + NN,
                                    smem_u32(net_s));
                    umma_commit(netbar);
                }
                {
                    const float* cp = cpart + gb * (H * 128) + r;
                    float sum = cp[0];
#pragma unroll
                    for (int hh2 = 1; hh2 < H; ++hh2) sum += cp[hh2 * 128];
                    csh = sum * inv_n;
                }
                const float w0 = w0buf[gb * 128 + r] * ref;
                const bool pub = (st + 1 < nst);
                float pg = 0.f, pe = 0.f;  // (gamma, eta) of the pair's first machine
                float ps = 0.f;            // sum of the next input's deviations
                if constexpr (AB2) {
                    // the angle half while the product runs: delta' depends on omega
                    // alone, so the next stage's angle input (after the last stage:
                    // the step's new angles, the next step's first input) and its
                    // (gamma, eta) are known before the network sums
                    float yn[NMT];
#pragma unroll
                    for (int k = 0; k < NMT; ++k) {
                        const float kd = a.omega_s * (yw[k] - w0);
                        ad[k] = fmaf(b, kd, ad[k]);
                        yn[k] = pub ? fmaf(cn, kd, del[k]) : fmaf(hh, ad[k], del[k]);
                        ps += h + H * k < n ? yn[k] : 0.f;
                    }
                    publish_angles<NMT, CST, H>(a_hi + an, a_lo + an, yn, csh, cst_s, h, n, nb);
                    cpart[(gb ^ 1) * (H * 128) + h * 128 + r] = ps;
                }
                float xs[ND];
#pragma unroll
                for (int e = 0; e < ND; ++e) xs[e] = fmaf(xw, x1[e] - x0[e], x0[e]);
                if (!net_wait(netbar, nph)) {
                    bad = 1;
                    atomicExch(a.err, DEV_TIMEOUT_MMA);
                }
                nph ^= 1u;
                tc_fence_after();
                // D with the (gamma, eta) it was formed from, in pieces of RP machines
                // (2 RP columns; 2 from 7 slots on, where registers are scarcest),
                // so that few values are live at once; with one A buffer the next
                // stage's input goes out in pairs of machines as soon as they are
                // computed
                constexpr int RP = NMT >= 7 ? 2 : 4;
                float dd[2 * RP], ah[2 * RP], al[2 * RP];
                // (one A buffer: the infinite bus's slot of the next input, from csh)
                float bcm = 0.f, bsn = 0.f;
                if (!AB2 && pub && nb >= 0 && nb % H == h) bus_deviation(csh, &bcm, &bsn);
#pragma unroll
                for (int k = 0; k < NMT; ++k) {
                    if (k % RP == 0) {
                        // columns of a last, partial piece
                        constexpr int WT = NMT % RP == 0 ? 2 * RP : (2 * (NMT % RP) + 3) & ~3;
                        if (NMT - k >= RP)
                            net_read<2 * RP>(a_d, a_hi + ab, a_lo + ab, 2 * k, dd, ah, al);
                        else
                            net_read<WT>(a_d, a_hi + ab, a_lo + ab, 2 * k, reinterpret_cast<float(&)[WT]>(dd),
                                         reinterpret_cast<float(&)[WT]>(ah), reinterpret_cast<float(&)[WT]>(al));
                    }
                    const int i = h + H * k;
                    const int c = 2 * (k % RP);
                    const float du = dd[c], dv = dd[c + 1];
                    const float gi = ah[c] + al[c], ei = ah[c + 1] + al[c + 1];
                    const float4 ca = *reinterpret_cast<const float4*>(cst_s + i * CST);
                    const float cs = ca.x, ss = ca.y;
                    float dpe = fmaf(cs, du, ss * dv);
                    dpe = fmaf(gi, ca.z + du, dpe);
                    dpe = fmaf(ei, ca.w + dv, dpe);
                    float f = 0.f;
#pragma unroll
                    for (int e4 = 0; e4 < ND; e4 += 4) {
                        // rows past the slots in use are zero
                        const float4 cj = *reinterpret_cast<const float4*>(cst_s + i * CST + 8 + e4);
                        const float cjv[4] = {cj.x, cj.y, cj.z, cj.w};
#pragma unroll
                        for (int e = e4; e < ND && e < e4 + 4; ++e) f = fmaf(cjv[e - e4], xs[e], f);
                    }
                    const float2 cb = *reinterpret_cast<const float2*>(cst_s + i * CST + 5);
                    const float kw = (f - dpe - cb.y * yw[k]) * cb.x;
                    if constexpr (!AB2) {
                        const float kd = a.omega_s * (yw[k] - w0);
                        ad[k] = fmaf(b, kd, ad[k]);
                        const float yd = fmaf(cn, kd, del[k]);
                        if (pub) {
                            // the next stage's input of machine i (its columns were read above)
                            const float2 g = wide_gamma_eta_tier(yd - csh, cs, ss, i < n);
                            const bool bus = k == NMT - 1 && i == nb;
                            const float gx = i < n ? g.x : (bus ? bcm : 0.f);
                            const float ex = i < n ? g.y : (bus ? -bsn : 0.f);
                            ps += i < n ? yd : 0.f;
                            if (k & 1)
                                net_store4(a_hi, a_lo, 2 * (k - 1), pg, pe, gx, ex);
                            else if (k == NMT - 1)
                                net_store4(a_hi, a_lo, 2 * k, gx, ex, 0.f, 0.f);
                            pg = gx;
                            pe = ex;
                        }
                    }
                    aw[k] = fmaf(b, kw, aw[k]);
                    yw[k] = fmaf(cn, kw, w[k]);
                }
                if (!AB2 && pub) {
                    tmem_st_wait();
                    cpart[(gb ^ 1) * (H * 128) + h * 128 + r] = ps;
                }
                if (pub && h == 0) w0buf[(gb ^ 1) * 128 + r] = yw[0];
                ath = fmaf(b, a.omega_s * w0, ath);
                if (pub) gb ^= 1;
            }
            if (failed) break;
} else {
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
                // the group's (gamma, eta) of this stage's input are complete
                asm volatile("bar.sync %0, 128;" ::"r"(1 + q) : "memory");
                const float2* ghc = gh + gb * n * 128 + r;
                const float w0 = w0buf[gb * 128 + r] * ref;
                float xs[ND];
#pragma unroll
                for (int e = 0; e < ND; ++e) xs[e] = fmaf(xw, x1[e] - x0[e], x0[e]);
                const bool pub = (st + 1 < nst);
                float2* ghn = gh + (gb ^ 1) * n * 128 + r;
                // KP machine slots per pass over j: one pass up to 10 slots; two
                // passes above, so that fewer network sums are live at once
#pragma unroll
                for (int k0 = 0; k0 < NMT; k0 += KP) {
                    float du[KP + 1], dv[KP + 1];
                    if constexpr (PACK) {
                        // packed FP32 over pairs of machine slots: (du_k, du_k+1) +=
                        // (GE_k, GE_k+1)(gamma_j, gamma_j) + (NBE_k, NBE_k+1)(eta_j, eta_j) and
                        // (dv_k, dv_k+1) += (GE_k, GE_k+1)(eta_j, eta_j) + (NBE_k, NBE_k+1)(-gamma_j, -gamma_j):
                        // the same roundings as the scalar form, half the instructions
                        constexpr int KP2 = (KP + 1) / 2;
                        unsigned long long du2[KP2], dv2[KP2];
#pragma unroll
                        for (int k = 0; k < KP2; ++k) {
                            du2[k] = 0ull;
                            dv2[k] = 0ull;
                        }
#pragma unroll JU
                        for (int j = 0; j < n; ++j) {
                            const float2 gej = ghc[j * 128];
                            const unsigned long long gg2 = f2pack(gej.x, gej.x), ee2 = f2pack(gej.y, gej.y);
                            const unsigned long long ng2 = f2pack(-gej.x, -gej.x);
                            const ulonglong2* g4 = reinterpret_cast<const ulonglong2*>(GB + (j * 4 + h) * 2 * NMTP + k0);
                            const ulonglong2* b4 = g4 + NMTP / 4;
#pragma unroll
                            for (int k4 = 0; k4 < (KP + 3) / 4; ++k4) {
                                if (k0 + 4 * k4 < NMT) {
                                    const ulonglong2 gv = g4[k4], bv = b4[k4];
#pragma unroll
                                    for (int kk = 0; kk < 2; ++kk) {
                                        const int k2 = 2 * k4 + kk;  // pair index
                                        if (k2 < KP2 && k0 + 2 * k2 < NMT) {
                                            const unsigned long long ge = kk ? gv.y : gv.x, nb = kk ? bv.y : bv.x;
                                            du2[k2] = ffma2(ge, gg2, du2[k2]);
                                            du2[k2] = ffma2(nb, ee2, du2[k2]);
                                            dv2[k2] = ffma2(ge, ee2, dv2[k2]);
                                            dv2[k2] = ffma2(nb, ng2, dv2[k2]);
                                        }
                                    }
                                }
                            }
                        }
#pragma unroll
                        for (int k2 = 0; k2 < KP2; ++k2) {
                            f2unpack(du2[k2], du[2 * k2], du[2 * k2 + 1]);
                            f2unpack(dv2[k2], dv[2 * k2], dv[2 * k2 + 1]);
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < KP; ++k) {
                            du[k] = 0.f;
                            dv[k] = 0.f;
                    }
#pragma unroll JU
                    for (int j = 0; j < n; ++j) {
                        const float2 gej = ghc[j * 128];
                        const float4* g4 = reinterpret_cast<const float4*>(GB + (j * 4 + h) * 2 * NMTP + k0);
                        const float4* b4 = g4 + NMTP / 4;
#pragma unroll
                        for (int k4 = 0; k4 < (KP + 3) / 4; ++k4) {
                            if (k0 + 4 * k4 < NMT) {
                                const float4 gv = g4[k4], bv = b4[k4];
                                const float gg[4] = {gv.x, gv.y, gv.z, gv.w};
                                const float bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                                for (int kk = 0; kk < 4; ++kk) {
                                    const int k = 4 * k4 + kk;
                                    if (k < KP && k0 + k < NMT) {
                                        du[k] = fmaf(gg[kk], gej.x, du[k]);
                                        du[k] = fmaf(-bb[kk], gej.y, du[k]);
                                        dv[k] = fmaf(gg[kk], gej.y, dv[k]);
                                        dv[k] = fmaf(bb[kk], gej.x, dv[k]);
                                    }
                                }
                            }
                        }
                    }
                    }
#pragma unroll
                    for (int kq = 0; kq < KP; ++kq) {
                        const int k = k0 + kq;
                        if (k < NMT) {
                            const int i = h + H * k;
                            const float2 ge = ghc[(i < n ? i : 0) * 128];
                            const float cs = c_cst[i], ss = c_sst[i];
                            float dpe = fmaf(cs, du[kq], ss * dv[kq]);
                            dpe = fmaf(ge.x, c_ust[i] + du[kq], dpe);
                            dpe = fmaf(ge.y, c_vst[i] + dv[kq], dpe);
                            float f = 0.f;
#pragma unroll
                            for (int e = 0; e < ND; ++e)
                                f = fmaf(c_inj[e * G4 + i], xs[e], f);  // rows past the slots in use are zero
                            const float kd = a.omega_s * (yw[k] - w0);
                            const float kw = (f - dpe - c_D[i] * yw[k]) * c_i2h[i];
                            ad[k] = fmaf(b, kd, ad[k]);
                            aw[k] = fmaf(b, kw, aw[k]);
                            const float yd = fmaf(cn, kd, del[k]);
                            yw[k] = fmaf(cn, kw, w[k]);
                            if (pub) {
                                // the next stage's input of machine i
                                const bool big = __any_sync(0xffffffffu, i < n && fabsf(yd) > 0.8f);
                                if (i < n) ghn[i * 128] = wide_gamma_eta(yd, cs, ss, big);
                            }
                        }
                    }
                }
                if (pub && h == 0) w0buf[(gb ^ 1) * 128 + r] = yw[0];
                ath = fmaf(b, a.omega_s * w0, ath);
                if (pub) gb ^= 1;
            }
}
#pragma unroll
            for (int k = 0; k < NMT; ++k) {
                del[k] = fmaf(hh, ad[k], del[k]);
                w[k] = fmaf(hh, aw[k], w[k]);
            }
            theta = fmaf(hh, ath, theta);
#pragma unroll
            for (int e = 0; e < ND; ++e) x0[e] = x1[e];
            // stage-0 input of the next step (AB2: already published by the last stage)
            if constexpr (AB2) {
                if (h == 0) w0buf[(gb ^ 1) * 128 + r] = w[0];
                gb ^= 1;
            } else if constexpr (TCN) {
                float ps = 0.f;
#pragma unroll
                for (int k = 0; k < NMT; ++k) ps += h + H * k < n ? del[k] : 0.f;
                publish_angles<NMT, CST, H>(a_hi, a_lo, del, csh, cst_s, h, n, nb);
                cpart[(gb ^ 1) * (H * 128) + h * 128 + r] = ps;
                if (h == 0) w0buf[(gb ^ 1) * 128 + r] = w[0];
                gb ^= 1;
            } else {
                float2* ghn = gh + (gb ^ 1) * n * 128 + r;
#pragma unroll
                for (int k = 0; k < NMT; ++k) {
                    const int i = h + H * k;
                    const bool big = __any_sync(0xffffffffu, i < n && fabsf(del[k]) > 0.8f);
                    if (i < n) ghn[i * 128] = wide_gamma_eta(del[k], c_cst[i], c_sst[i], big);
                }
                if (h == 0) w0buf[(gb ^ 1) * 128 + r] = w[0];
                gb ^= 1;
            }

            const int tn = n0 + s + 1;  // grid index of the new state
            if (traj) {
                float* o = traj + (int64_t)tn * trow;
#pragma unroll
                for (int k = 0; k < NMT; ++k) {
                    const int i = h + H * k;
                    if (i < n) {
                        o[i] = (theta + del[k]) + cst(4, i);
                        o[n + i] = w[k];
                    }
                }
            }
            // ---- moments: per warp, 32 samples x own machines ----
            float* myrow = wbuf + lane * WROW;
#pragma unroll
            for (int k = 0; k < NMT; ++k) {
                myrow[k] = active ? theta + del[k] : 0.f;
                myrow[NMT + k] = active ? w[k] : 0.f;
            }
            __syncwarp();
            const int ms = s % WI_MS;
            if (lane < 2 * NMT) {
                // the sample group's reference value, sum about it and squared deviations
                const int64_t left = a.count - (srow - lane);
                const int na = left <= 0 ? 0 : (left >= 32 ? 32 : (int)left);
                float rf, dv, m2;
                column_sums(wbuf + lane, WROW, na, &rf, &dv, &m2);
                float* slot = msum + ((ms * 4 + q) * H + h) * GS;
                slot[lane] = rf;
                slot[2 * NMT + lane] = dv;
                slot[4 * NMT + lane] = m2;
            }
            if (a.rrf) {
                float cp = 0.f;
#pragma unroll
                for (int k = 0; k < NMT; ++k) cp = fmaf(cst(7, h + H * k), w[k], cp);
                coi_part[(ms * H + h) * 128 + r] = cp;
            }
            __syncwarp();
            if (ms == WI_MS - 1 || s == steps - 1) {
                __syncthreads();
                if (a.rrf && h == 0) {
                    for (int sl = 0; sl <= ms; ++sl) {
                        const float* cq = coi_part + sl * H * 128 + r;
                        float c = cq[0];
#pragma unroll
                        for (int hh2 = 1; hh2 < H; ++hh2) c += cq[hh2 * 128];
                        racc_s[r] = fmaf(c, c, racc_s[r]);
                    }
                }
                const int nsl = ms + 1;
                const int tn0 = tn - ms;
                // samples of this tile (the last tile may be partly empty)
                const int64_t left = a.count - row0;
                const int n_tile = left <= 0 ? 0 : (left >= 128 ? 128 : (int)left);
                for (int e = tid; e < nsl * S; e += NTHR) {
                    const int sl = e / S, stt = e - sl * S;
                    // state stt < n is delta_i, else omega_(stt - n)
                    const int isw = stt >= n ? 1 : 0;
                    const int i = stt - isw * n;
                    const float* m = msum + (sl * 4 * H + (i % H)) * GS + isw * NMT + (i / H);
                    // the tile's triple over its four sample groups
                    float c, dv, m2;
                    combine_groups(m, m + 2 * NMT, m + 4 * NMT, H * GS, left, 4, &c, &dv, &m2);
                    if (part_tile) {
                        float* o = part_tile + (int64_t)(tn0 + sl) * S3;
                        o[stt] = c;
                        o[S + stt] = dv;
                        o[2 * S + stt] = m2;
                    } else if (n_tile > 0) {
                        // the tile's S1 and S2 (= M2 + S1^2 / n) about the shift, in FP64
                        const int64_t rowt = (int64_t)(tn0 + sl) * S;
                        const double s1 = fma((double)n_tile, (double)c, (double)dv);
                        atomicAdd(a.S1 + rowt + stt, s1);
                        atomicAdd(a.S2 + rowt + stt, (double)m2 + s1 * s1 / (double)n_tile);
                    }
                }
                __syncthreads();
            }
        }
        if (failed) break;
    }
    if (a.rrf && h == 0) rrf_accumulate(active ? sqrtf(racc_s[r] / (float)a.Nt) : 0.f, a.rrf);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, a.tmem_cols);
}

// Dynamic shared memory of the kernel (bytes), alignment slack included.
template <int NMT, int ND, bool TCN, int H = 4>
inline int wide_smem_bytes(int TC, int split, int n, int ns)
{
    const int stage = (TC_M * 64 + TC * 64) * (split ? 2 : 1);
    const int mom = wide_mom_floats<NMT, H>() * 4;
    const int u = ((ns * stage > mom ? ns * stage : mom) + 1023) & ~1023;
    if (TCN)
        return 1024 + u + wide_tc_net_bytes(NMT, H) + (384 + 1024) * 4 + 4 * NMT * ((8 + ND + 3) & ~3) * 4;
    return 1024 + u + 2 * n * 128 * 8 + 384 * 4 + wide_const_floats(n, NMT, ND) * 4;
}

// maps: the four contraction maps, then (TCN) the map of the network matrix.
// H = 2: two CTAs per SM, each with at most half of the SM's shared memory.
template <int NMT, int ND, bool TCN = false, int H = 4, bool BUS = false>
cudaError_t launch_wide_t(const CUtensorMap* maps, const WideArgs& args, cudaStream_t st, int* occ_out)
{
    static_assert(!BUS || (TCN && H == 4), "the infinite-bus form is built for four warps per sample");
    // (the tensor-core form shifts the angles: exact with a network alone, or with
    // the infinite bus held in its slot)
    if (TCN && BUS == (args.rel != 0)) return cudaErrorInvalidValue;
    auto kern = simulate_wide_kernel<NMT, ND, TCN, H, BUS>;
    const int cap = H == 4 ? TC_SMEM_DYN_MAX : 233472 / 2 - 2048;
    // as many ring stages as the shared memory left by the other buffers holds
    WideArgs a = args;
    a.ns = 2;
    while (a.ns < TC_MAX_STAGES && wide_smem_bytes<NMT, ND, TCN, H>(a.TC, a.split, a.n, a.ns + 1) <= cap) ++a.ns;
    const int smem = wide_smem_bytes<NMT, ND, TCN, H>(a.TC, a.split, a.n, a.ns);
    if (smem > cap) return cudaErrorInvalidValue;
    if (smem > TC_SMEM_DYN_MAX) return cudaErrorInvalidValue;
    // the attribute is process-wide and launches from several host threads may
    // race on it: always the same (largest) bound, the launch passes its own size
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_DYN_MAX);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, H * 128, smem);
    if (e != cudaSuccess) return e;
    *occ_out = occ;
    if (occ < 1 || (uint32_t)occ * a.tmem_cols > 512u) return cudaErrorInvalidConfiguration;
    const int64_t ntiles = (a.count + TC_M - 1) / TC_M;
    if (ntiles > 2147483647LL) return cudaErrorInvalidValue;
    kern<<<(unsigned)ntiles, H * 128, smem, st>>>(maps[0], maps[1], maps[2], maps[3], maps[TCN ? 4 : 0], a);
    return cudaGetLastError();
}

}  // namespace fmc
