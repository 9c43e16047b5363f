// Per-sample dynamics of the fused and plain simulation kernels: Euler-Maruyama
// for the OU disturbances and RK4/Heun for the Kron-reduced classical swing
// equations, one CUDA thread per Monte Carlo sample, FP32.
//
// Model (classical machines, Eqs. state/algebra reduced by eliminating the
// network): d delta_i/dt = omega_s domega_i,
//   2 H_i d domega_i/dt = Pm_i + sum_w inj[i][w] x_w - Pe_i - D_i domega_i,
//   Pe_i = sum_j E_i E_j (G_ij cos(delta_i-delta_j) + B_ij sin(delta_i-delta_j))
//          [+ E_i V (Ginf_i cos delta_i + Binf_i sin delta_i)].
// Evaluated in product form around the equilibrium (see swing_step), so a stage
// costs NM small-angle sin/cos pairs and 4 NM (NM - 1) FMAs.  The matrices and
// the equilibrium constants live in the kernel parameter block: fully unrolled
// loops address them with immediate offsets, so every FMA takes its constant
// operand straight from the constant bank.
//
// Register economy: a stage evaluates the right-hand side machine by machine and
// immediately folds k_i into the RK accumulator and into the next stage's input,
// so only state, accumulator, stage input and the stage's deviations stay live.
// Padded disturbances (index >= d) have zero sigma and zero injection; padded
// machines have zero network rows and stay at rest.
#pragma once

#include "fmc_common.cuh"
#include "kernels.cuh"


namespace fmc {

// sin and cos of an FP32 angle to a few ulps, on the FP32 pipe (no MUFU):
// Cody-Waite reduction x = k pi/2 + r with pi/2 split into its FP32 rounding
// and the remainder (both products exact inside the FMAs), then the Taylor
// series of sin r to degree 9 and of cos r to degree 10, whose truncation is
// below 2e-9 on |r| <= pi/4, then the quadrant k mod 4.  The hardware
// approximations (__sinf, __cosf) carry absolute errors near 4e-7, which the
// stiff network terms (|B_ij| E_i E_j up to ~10 p.u.) turn into power errors
// that dominate the speed deviation; this keeps the evaluation at FP32
// rounding level.  Accurate for |x| < 2^20.
__device__ __forceinline__ void sincos_cw(float x, float* s_out, float* c_out)
{
    const float TWO_OVER_PI = 0.636619772367581343f;
    const float PIO2_HI = 1.57079637050628662109375f;   // pi/2 rounded to FP32
    const float PIO2_LO = -4.37113900018624283e-8f;     // pi/2 - PIO2_HI
    const float k = rintf(x * TWO_OVER_PI);
    float r = fmaf(-k, PIO2_HI, x);
    r = fmaf(-k, PIO2_LO, r);
    const float r2 = r * r;
    // sin r = r - r^3/3! + r^5/5! - r^7/7! + r^9/9!
    float ps = fmaf(r2, 2.7557319223985891e-6f, -1.9841269841269841e-4f);
    ps = fmaf(ps, r2, 8.3333333333333333e-3f);
    ps = fmaf(ps, r2, -1.6666666666666667e-1f);
    const float sr = fmaf(ps * r2, r, r);
    // cos r = 1 - r^2/2! + r^4/4! - r^6/6! + r^8/8! - r^10/10!
    float pc = fmaf(r2, -2.7557319223985891e-7f, 2.4801587301587302e-5f);
    pc = fmaf(pc, r2, -1.3888888888888889e-3f);
    pc = fmaf(pc, r2, 4.1666666666666667e-2f);
    pc = fmaf(pc, r2, -0.5f);
    const float cr = fmaf(pc, r2, 1.0f);
    const int q = (int)k;
    const bool odd = (q & 1) != 0;
    const float a = odd ? cr : sr;
    const float b = odd ? sr : cr;
    *s_out = __int_as_float(__float_as_int(a) ^ ((q & 2) << 30));
    *c_out = __int_as_float(__float_as_int(b) ^ (((q + 1) & 2) << 30));
}

template <int NM, int ND>
struct SwingParams {
    // The network in the rotated deviation form (see swing_step_impl), each row i
    // divided by 2 H_i; zero diagonal.  With delta*_ij = delta*_i - delta*_j,
    //   A_ij  = E_i E_j (G_ij cos delta*_ij + B_ij sin delta*_ij),
    //   Bm_ij = E_i E_j (B_ij cos delta*_ij - G_ij sin delta*_ij).
    float2 P1[NM][NM];           // (A_ij, -Bm_ij) / 2H_i: packed multiplier of (cos D_j - 1, sin D_j) -> U
    float2 P2[NM][NM];           // (Bm_ij, A_ij) / 2H_i: packed multiplier of (cos D_j - 1, sin D_j) -> V
    float Ah[NM][NM];            // A_ij / 2H_i (scalar network sum)
    float Bh[NM][NM];            // Bm_ij / 2H_i
    float pst[NM];               // P*_i / 2H_i = (c*_i u*_i + s*_i v*_i) / 2H_i
    float qst[NM];               // Q*_i / 2H_i = (c*_i v*_i - s*_i u*_i) / 2H_i
    float dst[NM];               // equilibrium angles delta*_i (absolute)
    float Dh[NM];                // D_i / 2H_i
    float injh[NM][ND];          // inj[i][w] / 2H_i
    float ou_a[ND];              // 1 - theta_w dt (1 in the event slot)
    float ou_s[ND];              // sigma_w (0 in the event slot)
    float hw[NM];                // H_i / sum H: centre-of-inertia weights of the response function
    float omega_s;
    float dt;
    int d;                       // real disturbances (<= ND; the rest are zero)
    int n;                       // real machines (<= NM; the rest are inert padding)
    int integrator;              // FMC_RK4 / FMC_HEUN
    int rel;                     // 1: angles relative to machine 0 (no infinite bus)
    // An event (a step in one machine's mechanical power from grid step ev_step
    // on) rides in a spare disturbance slot ev_slot >= d: its "disturbance" is 0
    // before the event and 1 from it, its injection the power step; -1: none.
    int ev_slot;
    int ev_step;
    ItoParams<ND> ito;           // general disturbances (ito.on == 0: all OU)
    float th[ND];                // theta_w, the OU rate (the smooth form's drift; 0 in padding and the event slot)
};

// The event slot's value for the step that starts at grid index `step`.
template <int NM, int ND>
__device__ __forceinline__ void event_state(const SwingParams<NM, ND>& p, int step, float (&x0)[ND])
{
#pragma unroll
    for (int q = 0; q < ND; ++q)
        if (q == p.ev_slot) x0[q] = (step >= p.ev_step) ? 1.f : 0.f;
}

// The centre-of-inertia speed deviation of one sample.
template <int NM, int ND>
__device__ __forceinline__ float coi_speed(const SwingParams<NM, ND>& p, const float (&w)[NM])
{
    float c = 0.f;
#pragma unroll
    for (int i = 0; i < NM; ++i) c = fmaf(p.hw[i], w[i], c);
    return c;
}

// sin(a) and cos(a) - 1 of a deviation angle below 0.05 in magnitude: a - a^3/6
// and -a^2/2 + a^4/24, whose truncation, a^4/120 and a^4/360 relative, stays
// below 2^-24 for |a| <= 0.052 (half an FP32 ulp of the result).
__device__ __forceinline__ void sin_cosm1_tiny(float a, float* sn, float* cm1)
{
    const float a2 = a * a;
    *sn = fmaf(a2 * a, -1.6666666666666667e-1f, a);
    *cm1 = fmaf(a2, 4.1666666666666667e-2f, -0.5f) * a2;
}

// The same to degree 5 and 6 for |a| <= 0.25: truncation a^6/5040 and a^6/20160
// relative, below 5e-8.
__device__ __forceinline__ void sin_cosm1_mid(float a, float* sn, float* cm1)
{
    const float a2 = a * a;
    float ps = fmaf(a2, 8.3333333333333333e-3f, -1.6666666666666667e-1f);
    *sn = fmaf(ps * a2, a, a);
    float pc = fmaf(a2, -1.3888888888888889e-3f, 4.1666666666666667e-2f);
    pc = fmaf(pc, a2, -0.5f);
    *cm1 = pc * a2;
}

// sin(a) and cos(a) - 1 of a small deviation angle, without cancellation: the
// Taylor series to degree 9 and 10 (truncation < 3e-9 for |a| <= 0.8).
__device__ __forceinline__ void sin_cosm1_small(float a, float* sn, float* cm1)
{
    const float a2 = a * a;
    float ps = fmaf(a2, 2.7557319223985891e-6f, -1.9841269841269841e-4f);
    ps = fmaf(ps, a2, 8.3333333333333333e-3f);
    ps = fmaf(ps, a2, -1.6666666666666667e-1f);
    *sn = fmaf(ps * a2, a, a);
    float pc = fmaf(a2, -2.7557319223985891e-7f, 2.4801587301587302e-5f);
    pc = fmaf(pc, a2, -1.3888888888888889e-3f);
    pc = fmaf(pc, a2, 4.1666666666666667e-2f);
    pc = fmaf(pc, a2, -0.5f);
    *cm1 = pc * a2;
}

// Any deviation: the reduced-argument evaluation, cos - 1 = -2 sin^2(a/2).
__device__ __forceinline__ void sin_cosm1_any(float a, float* sn, float* cm1)
{
    float c, sh, ch;
    sincos_cw(a, sn, &c);
    sincos_cw(0.5f * a, &sh, &ch);
    *cm1 = -2.0f * sh * sh;
}

// The angle tier of a stage: 0 when every machine of every lane of the warp
// deviates by at most 0.05 rad, 1 up to 0.25, 2 up to 0.8, 3 beyond
// (warp-uniform, so the series below never diverge inside a warp).
// SHORT false: only tiers 2 and 3 (kernels where code size and compile time
// matter more than the shorter series).
template <int NM, bool SHORT>
__device__ __forceinline__ int angle_tier(const float (&yd)[NM])
{
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < NM; ++j) m = fmaxf(m, fabsf(yd[j]));
    const unsigned mask = __activemask();
    if (SHORT && __all_sync(mask, m <= 0.05f)) return 0;
    if (SHORT && __all_sync(mask, m <= 0.25f)) return 1;
    if (__all_sync(mask, m <= 0.8f)) return 2;
    return 3;
}

// sin and cos - 1 of one deviation angle by the series of the warp's tier.
template <int TIER>
__device__ __forceinline__ void deviation_trig1(float a, float* sn, float* cm1)
{
    if constexpr (TIER == 0)
        sin_cosm1_tiny(a, sn, cm1);
    else if constexpr (TIER == 1)
        sin_cosm1_mid(a, sn, cm1);
    else if constexpr (TIER == 2)
        sin_cosm1_small(a, sn, cm1);
    else
        sin_cosm1_any(a, sn, cm1);
}

// The pair (cos Delta_j - 1, sin Delta_j) of every machine for one RK stage.
template <int TIER, int NM>
__device__ __forceinline__ void stage_trig(const float (&yd)[NM], unsigned long long (&cs2)[NM])
{
#pragma unroll
    for (int j = 0; j < NM; ++j) {
        float c, sj;
        deviation_trig1<TIER>(yd[j], &sj, &c);
        cs2[j] = f2pack(c, sj);
    }
}

// Row i's network sums (U_i, V_i) (see swing_step_impl) over the pairs cs2:
// packed, as two partial sums (A cm, -Bm sn) and (Bm cm, A sn) whose halves
// add to U and V.
template <int NM, int ND>
__device__ __forceinline__ void row_network(const SwingParams<NM, ND>& p, int i, const unsigned long long (&cs2)[NM],
                                            float& U, float& V)
{
#if FMC_PACKED_FP32
    unsigned long long au = 0ull, av = 0ull;
#pragma unroll
    for (int j = 0; j < NM; ++j) {
        if (j == i) continue;
        au = ffma2(*reinterpret_cast<const unsigned long long*>(&p.P1[i][j]), cs2[j], au);
        av = ffma2(*reinterpret_cast<const unsigned long long*>(&p.P2[i][j]), cs2[j], av);
    }
    float u0, u1, v0, v1;
    f2unpack(au, u0, u1);
    f2unpack(av, v0, v1);
    U = u0 + u1;
    V = v0 + v1;
#else
    U = 0.f;
    V = 0.f;
#pragma unroll
    for (int j = 0; j < NM; ++j) {
        if (j == i) continue;
        float c, sj;
        f2unpack(cs2[j], c, sj);
        U = fmaf(p.Ah[i][j], c, U);
        U = fmaf(-p.Bh[i][j], sj, U);
        V = fmaf(p.Bh[i][j], c, V);
        V = fmaf(p.Ah[i][j], sj, V);
    }
#endif
}

// The angle derivative omega_s (domega_i - domega_0) enters through cnw = cn
// omega_s, and ad accumulates the speed differences themselves (the caller
// multiplies by omega_s once per step).
// TIER < 0: the tier is the run-time rtier (2 or 3), branching only around the
// sines and cosines.
template <int TIER, int NM, int ND>
__device__ __forceinline__ void stage_rhs(const SwingParams<NM, ND>& p, const float (&xs)[ND], float w0, float b,
                                          float cn, float cnw, const float (&del)[NM], const float (&w)[NM],
                                          float (&ad)[NM], float (&aw)[NM], float (&yd)[NM], float (&yw)[NM],
                                          int rtier = 0)
{
    unsigned long long cs2[NM];
    if constexpr (TIER >= 0) {
        stage_trig<TIER, NM>(yd, cs2);
    } else {
        if (rtier == 2)
            stage_trig<2, NM>(yd, cs2);
        else
            stage_trig<3, NM>(yd, cs2);
    }
#pragma unroll
    for (int i = 0; i < NM; ++i) {
        float U, V, cmi, sni;
        row_network<NM, ND>(p, i, cs2, U, V);
        f2unpack(cs2[i], cmi, sni);
        V += p.qst[i];
        // (forcing - D domega - dPe) / 2H, the rows already scaled
        float dpe = fmaf(cmi, U + p.pst[i], U);
        dpe = fmaf(sni, V, dpe);
        float f = 0.f;
#pragma unroll
        for (int q = 0; q < ND; ++q) f = fmaf(p.injh[i][q], xs[q], f);
        const float kw = fmaf(-p.Dh[i], yw[i], f - dpe);
        const float kv = yw[i] - w0;   // the angle's rate over omega_s
        ad[i] = fmaf(b, kv, ad[i]);
        aw[i] = fmaf(b, kw, aw[i]);
        yd[i] = fmaf(cnw, kv, del[i]);
        yw[i] = fmaf(cn, kw, w[i]);
    }
}

// One step of the swing equations, integrated in deviation variables
//   Delta_i = delta_i - delta*_i - theta   (theta: angle of machine 0 when the
//   system has no infinite bus, so that the common drift of all angles, which
//   the network does not see, never enters the FP32 network terms; 0 otherwise)
// With cm_j = cos Delta_j - 1 and sn_j = sin Delta_j, the angle-difference
// identities give the electrical power's deviation from equilibrium exactly as
//   dPe_i = U_i + cm_i (U_i + P*_i) + sn_i (V_i + Q*_i),
//   U_i = sum_{j!=i} A_ij cm_j - Bm_ij sn_j,   V_i = sum_{j!=i} Bm_ij cm_j + A_ij sn_j,
// with A, Bm the network coupling at the equilibrium angles and P*_i, Q*_i the
// machine's off-diagonal equilibrium power and its quadrature (the infinite bus
// included); the diagonal E_i^2 G_ii is constant.  Every quantity is on the
// scale of the deviations, so FP32 keeps its relative precision, and since
// Pm = Pe(delta*) at the equilibrium,
//   d(domega_i)/dt = (sum_w inj[i][w] x_w - dPe_i - D_i domega_i) / 2H_i,
// with every row already divided by 2H_i on the host.  The state follows the
// same RK4 trajectory as in absolute angles (RK4 commutes with the linear change
// of variables).
// The stages run as a loop that is not unrolled, so the right-hand side exists
// once in the code and its constant operands are not held in registers across
// stages.  The disturbance enters stage st at x0 + xw (x1 - x0): RK4 xw = 0,
// 1/2, 1/2, 1 (the midpoint value is the average of the two grid values), Heun
// xw = 0, 1.
template <int NM, int ND, bool STAGED, bool SHORT>
__device__ __forceinline__ void swing_step_impl(const SwingParams<NM, ND>& p, float (&del)[NM], float (&w)[NM],
                                                float& theta, const float (&x0)[ND], const float (&x1)[ND],
                                                const float (&xst)[4][ND])
{
    const float dt = p.dt;
    const bool rk4 = (p.integrator == FMC_RK4);
    const int nst = rk4 ? 4 : 2;
    const float ref = p.rel ? 1.f : 0.f;
    float ad[NM], aw[NM], yd[NM], yw[NM];
    float ath = 0.f;
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
        if constexpr (STAGED) {
            // the smooth form: the disturbances' own stage values (a select, the
            // stage loop is not unrolled)
#pragma unroll
            for (int q = 0; q < ND; ++q)
                xs[q] = st == 0 ? xst[0][q] : (st == 1 ? xst[1][q] : (st == 2 ? xst[2][q] : xst[3][q]));
        } else {
#pragma unroll
            for (int q = 0; q < ND; ++q) xs[q] = fmaf(xw, x1[q] - x0[q], x0[q]);
        }
        const float w0 = yw[0] * ref;
        ath = fmaf(b, w0, ath);
        const float cnw = cn * p.omega_s;
        // the whole stage per angle tier, so that only the state arrays meet
        // where the branches join
        const int tier = angle_tier<NM, SHORT>(yd);
        if constexpr (SHORT) {
            if (tier == 0)
                stage_rhs<0, NM, ND>(p, xs, w0, b, cn, cnw, del, w, ad, aw, yd, yw);
            else if (tier == 1)
                stage_rhs<1, NM, ND>(p, xs, w0, b, cn, cnw, del, w, ad, aw, yd, yw);
            else if (tier == 2)
                stage_rhs<2, NM, ND>(p, xs, w0, b, cn, cnw, del, w, ad, aw, yd, yw);
            else
                stage_rhs<3, NM, ND>(p, xs, w0, b, cn, cnw, del, w, ad, aw, yd, yw);
        } else {
            // one copy of the stage: only the sines and cosines branch
            stage_rhs<-1, NM, ND>(p, xs, w0, b, cn, cnw, del, w, ad, aw, yd, yw, tier);
        }
    }
    const float h = rk4 ? dt * (1.0f / 6.0f) : 0.5f * dt;
    const float hw = h * p.omega_s;
#pragma unroll
    for (int i = 0; i < NM; ++i) {
        del[i] = fmaf(hw, ad[i], del[i]);
        w[i] = fmaf(h, aw[i], w[i]);
    }
    theta = fmaf(hw, ath, theta);
}

// The disturbance entering stage st at x0 + xw (x1 - x0) (see swing_step_impl).
// SHORT: the short series for small angle deviations are compiled in.
template <int NM, int ND, bool SHORT = false>
__device__ __forceinline__ void swing_step(const SwingParams<NM, ND>& p, float (&del)[NM], float (&w)[NM],
                                           float& theta, const float (&x0)[ND], const float (&x1)[ND])
{
    const float unused[4][ND] = {};
    swing_step_impl<NM, ND, false, SHORT>(p, del, w, theta, x0, x1, unused);
}

// The smooth form: the disturbance's value at RK stage st is xst[st] (Heun: st < 2).
template <int NM, int ND>
__device__ __forceinline__ void swing_step_staged(const SwingParams<NM, ND>& p, float (&del)[NM], float (&w)[NM],
                                                  float& theta, const float (&xst)[4][ND])
{
    swing_step_impl<NM, ND, true, false>(p, del, w, theta, xst[0], xst[3], xst);
}

// One step of a general disturbance (see ItoParams) in the deviation y.
template <int ND>
__device__ __forceinline__ float ito_step1(const ItoParams<ND>& it, int q, float ou_a, float ou_s, float y, float dw,
                                           float dt)
{
    if (it.kind[q] == FMC_ITO_OU) return fmaf(ou_a, y, ou_s * dw);
    const float mu = fmaf(fmaf(it.c2[q], y, it.c1[q]), y, it.c0[q]);
    float sg, corr;
    if (it.kind[q] == FMC_ITO_POLY) {
        sg = fmaf(fmaf(it.e2[q], y, it.e1[q]), y, it.e0[q]);
        corr = sg * fmaf(2.f * it.e2[q], y, it.e1[q]);
    } else {
        const float dy = y - it.ap[q];
        const float v = fmaf(it.e3[q], fabsf(dy), fmaf(fmaf(it.e2[q], y, it.e1[q]), y, it.e0[q]));
        sg = v > 0.f ? sqrtf(v) : 0.f;
        const float sgn = dy > 0.f ? 1.f : (dy < 0.f ? -1.f : 0.f);
        corr = v > 0.f ? 0.5f * fmaf(it.e3[q], sgn, fmaf(2.f * it.e2[q], y, it.e1[q])) : 0.f;
    }
    const float drift = fmaf(-0.5f * it.strat, corr, mu);
    return fmaf(sg, dw, fmaf(drift, dt, y));
}

// The smooth form's rate of disturbance q at deviation y under forcing f:
// dy/dt = -theta y + sigma f (OU), or the general model's drift with the
// Stratonovich correction (its limit on a smooth path) plus sigma(y) f.
template <int NM, int ND>
__device__ __forceinline__ float smooth_rate(const SwingParams<NM, ND>& p, int q, float y, float f)
{
    const ItoParams<ND>& it = p.ito;
    if (!it.on || it.kind[q] == FMC_ITO_OU) return fmaf(-p.th[q], y, p.ou_s[q] * f);
    const float mu = fmaf(fmaf(it.c2[q], y, it.c1[q]), y, it.c0[q]);
    float sg, corr;
    if (it.kind[q] == FMC_ITO_POLY) {
        sg = fmaf(fmaf(it.e2[q], y, it.e1[q]), y, it.e0[q]);
        corr = sg * fmaf(2.f * it.e2[q], y, it.e1[q]);
    } else {
        const float dy = y - it.ap[q];
        const float v = fmaf(it.e3[q], fabsf(dy), fmaf(fmaf(it.e2[q], y, it.e1[q]), y, it.e0[q]));
        sg = v > 0.f ? sqrtf(v) : 0.f;
        const float sgn = dy > 0.f ? 1.f : (dy < 0.f ? -1.f : 0.f);
        corr = v > 0.f ? 0.5f * fmaf(it.e3[q], sgn, fmaf(2.f * it.e2[q], y, it.e1[q])) : 0.f;
    }
    return fmaf(sg, f, fmaf(-0.5f, corr, mu));
}

// The smooth form's step of every disturbance from grid step `step`: the random
// ODE dy/dt = smooth_rate(y, f(t)) by the RK4 (or Heun) stages with the forcing
// f0 at t_n, fh at t_n + dt/2 and f1 at t_{n+1}; xst[st] receives the stage
// values the swing stages see, x0 the value at t_{n+1}.  Slots q >= d: padding
// (0), or the event slot (0 before its grid step, 1 from it).
template <int NM, int ND>
__device__ __forceinline__ void smooth_stages(const SwingParams<NM, ND>& p, int step, float (&x0)[ND],
                                              const float (&f0)[ND], const float (&fh)[ND], const float (&f1)[ND],
                                              float (&xst)[4][ND])
{
    const float dt = p.dt;
    const bool rk4 = (p.integrator == FMC_RK4);
#pragma unroll
    for (int q = 0; q < ND; ++q) {
        float xn;
        if (q < p.d) {
            const float x = x0[q];
            const float k1 = smooth_rate<NM, ND>(p, q, x, f0[q]);
            if (rk4) {
                const float X2 = fmaf(0.5f * dt, k1, x);
                const float k2 = smooth_rate<NM, ND>(p, q, X2, fh[q]);
                const float X3 = fmaf(0.5f * dt, k2, x);
                const float k3 = smooth_rate<NM, ND>(p, q, X3, fh[q]);
                const float X4 = fmaf(dt, k3, x);
                const float k4 = smooth_rate<NM, ND>(p, q, X4, f1[q]);
                xst[0][q] = x;
                xst[1][q] = X2;
                xst[2][q] = X3;
                xst[3][q] = X4;
                xn = fmaf(dt * (1.0f / 6.0f), (k1 + 2.f * k2) + (2.f * k3 + k4), x);
            } else {
                const float X2 = fmaf(dt, k1, x);
                const float k2 = smooth_rate<NM, ND>(p, q, X2, f1[q]);
                xst[0][q] = x;
                xst[1][q] = X2;
                xst[2][q] = X2;
                xst[3][q] = X2;
                xn = fmaf(0.5f * dt, k1 + k2, x);
            }
        } else {
            const float ev = (q == p.ev_slot && step >= p.ev_step) ? 1.f : 0.f;
            xst[0][q] = xst[1][q] = xst[2][q] = xst[3][q] = ev;
            xn = ev;
        }
        x0[q] = xn;
    }
}

// One Euler-Maruyama step of the OU disturbances: x1 = (1 - theta dt) x0 + sigma dW.
template <int NM, int ND>
__device__ __forceinline__ void ou_step(const SwingParams<NM, ND>& p, const float (&x0)[ND], const float (&dw)[ND],
                                        float (&x1)[ND])
{
    if (p.ito.on) {
#pragma unroll
        for (int q = 0; q < ND; ++q) x1[q] = ito_step1<ND>(p.ito, q, p.ou_a[q], p.ou_s[q], x0[q], dw[q], p.dt);
        return;
    }
#pragma unroll
    for (int q = 0; q < ND; ++q) x1[q] = fmaf(p.ou_a[q], x0[q], p.ou_s[q] * dw[q]);
}

}  // namespace fmc
