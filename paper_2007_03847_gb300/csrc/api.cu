// C ABI of the fastmc library: argument validation, workspace, tensor maps and
// the sequencing of the kernels of Algorithm 1 on the caller's stream.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "fmc_common.cuh"
#include "kernels.cuh"
#include "swing.cuh"
#include "tc_common.cuh"
#include "wide_tc.cuh"
#include "api_internal.h"
#include "../../include/fastmc_diag.h"

using namespace fmc;

namespace {

// Grow-only device buffer owned by a context.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

enum Phase {
    PH_LHS = 0, PH_BASIS, PH_EQ, PH_FUSED, PH_REDUCE, PH_CONTRACT, PH_INTEGRATE, PH_MOMENTS, PH_BATCH, PH_COUNT
};

struct ProfRec {
    int phase;
    cudaEvent_t a, b;
};

}  // namespace

// Device buffers of one simulation: design, basis, partial sums, equilibrium,
// status word; the plain path's FP32 design, increments and trajectories.
struct Workspace {
    DevBuf zeta_hi, zeta_lo, phi_hi, phi_lo, phi32, dW, traj, part, eq, scen, status, zeta32;
    DevBuf wconst;  // constant block of the large-system kernel
    DevBuf rrf;     // [4] FP64: sums of the response function and its square, a zero shift
    DevBuf ic, ic_strata;  // the correlation-reducing permutation: working memory, new strata [M][N]
    DevBuf ident;          // identification sums [43], flag, Newton step [6], flag
};

struct fmc_ctx {
    int device = 0;
    int sms = 0;
    int64_t l2_bytes = 0;   // the device's L2 cache
    char name[256] = {0};
    size_t budget = 0;
    size_t used = 0;
    std::string err;
    Workspace ws;                     // workspace of the single-scenario calls
    DevBuf& zeta_hi = ws.zeta_hi;
    DevBuf& zeta_lo = ws.zeta_lo;
    DevBuf& phi_hi = ws.phi_hi;
    DevBuf& phi_lo = ws.phi_lo;
    DevBuf& phi32 = ws.phi32;
    DevBuf& dW = ws.dW;
    DevBuf& traj = ws.traj;
    DevBuf& part = ws.part;
    DevBuf& eq = ws.eq;
    DevBuf& scen = ws.scen;
    DevBuf& status = ws.status;
    DevBuf& zeta32 = ws.zeta32;
    DevBuf& wconst = ws.wconst;
    DevBuf& rrfbuf = ws.rrf;
    // profiling of kernel phases (CUDA events on the launching stream)
    bool prof = false;
    std::vector<ProfRec> recs;
    size_t prof_cap = 0;
    int last_fused_ctas_per_sm = 0;
    int kernel_policy = FMC_KERNEL_AUTO;
    std::vector<fmc_launch_rule> rules;  // measured launch shapes (fmc_set_launch_rules)
    // Contexts used on one stream only (the server's) grow their workspace in
    // stream order on that stream (cudaFreeAsync / cudaMallocAsync) instead of
    // synchronising the whole device, which would stall every other request.
    bool stream_ordered = false;
    cudaStream_t ws_stream = nullptr;
};

static thread_local std::string g_create_err;

typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode()
{
    static PFN_encodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_encodeTiled)p;
    }
    return fn;
}

static int fail(fmc_ctx* ctx, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return code;
}

static int cuda_fail(fmc_ctx* ctx, cudaError_t e, const char* what)
{
    return fail(ctx, FMC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define FMC_CUDA(ctx, expr, what)                         \
    do {                                                  \
        cudaError_t _e = (expr);                          \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, what); \
    } while (0)

static int ensure(fmc_ctx* ctx, DevBuf& b, size_t bytes)
{
    if (b.bytes >= bytes) return FMC_OK;
    size_t want = bytes + bytes / 8;
    if (ctx->budget && ctx->used - b.bytes + want > ctx->budget) {
        want = bytes;
        if (ctx->used - b.bytes + want > ctx->budget)
            return fail(ctx, FMC_ENOMEM, "workspace of %zu bytes exceeds the budget of %zu", bytes, ctx->budget);
    }
    const bool ordered = ctx->stream_ordered && ctx->ws_stream != nullptr;
    if (b.ptr) {
        if (ordered) {
            cudaFreeAsync(b.ptr, ctx->ws_stream);
        } else {
            cudaDeviceSynchronize();
            cudaFree(b.ptr);
        }
        ctx->used -= b.bytes;
        b.ptr = nullptr;
        b.bytes = 0;
    }
    cudaError_t e = ordered ? cudaMallocAsync(&b.ptr, want, ctx->ws_stream) : cudaMalloc(&b.ptr, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, FMC_ENOMEM, "cudaMalloc(%zu): %s", want, cudaGetErrorString(e));
    }
    b.bytes = want;
    ctx->used += want;
    return FMC_OK;
}

// ---- profiling --------------------------------------------------------------

static void prof_begin(fmc_ctx* ctx, int phase, cudaStream_t st, ProfRec** out)
{
    *out = nullptr;
    if (!ctx->prof || ctx->recs.size() >= ctx->prof_cap) return;
    ProfRec r;
    r.phase = phase;
    if (cudaEventCreate(&r.a) != cudaSuccess) return;
    if (cudaEventCreate(&r.b) != cudaSuccess) {
        cudaEventDestroy(r.a);
        return;
    }
    cudaEventRecord(r.a, st);
    ctx->recs.push_back(r);
    *out = &ctx->recs.back();
}

static void prof_end(ProfRec* r, cudaStream_t st)
{
    if (r) cudaEventRecord(r->b, st);
}

static void prof_clear(fmc_ctx* ctx)
{
    for (auto& r : ctx->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    ctx->recs.clear();
}

// ---- scenario checks --------------------------------------------------------

static int nm_bucket_for(int n)
{
    static const int buckets[] = {1, 2, 4, 8, 10, 12, 16};
    for (int b : buckets)
        if (n <= b) return b;
    return -1;
}

static int steps_of(fmc_ctx* ctx, double T, double dt, int* Nt)
{
    if (!(T > 0.0) || !(dt > 0.0) || !std::isfinite(T) || !std::isfinite(dt))
        return fail(ctx, FMC_EINVAL, "T and dt must be positive and finite (T=%g, dt=%g)", T, dt);
    double r = T / dt;
    double k = std::round(r);
    if (k < 1 || k > 2147483647.0 || std::fabs(k * dt - T) > 1e-9 * T)
        return fail(ctx, FMC_EINVAL, "T/dt = %.12g is not an integer number of steps", r);
    *Nt = (int)k;
    return FMC_OK;
}

static int check_scenario(fmc_ctx* ctx, const fmc_scenario* s, int* Nt)
{
    if (!s) return fail(ctx, FMC_EINVAL, "scenario is NULL");
    if (s->n < 1) return fail(ctx, FMC_EINVAL, "n = %d < 1", s->n);
    if (s->n > FMC_MAX_MACHINES) return fail(ctx, FMC_EUNSUPPORTED, "n = %d above %d", s->n, FMC_MAX_MACHINES);
    if (s->d < 1) return fail(ctx, FMC_EINVAL, "d = %d < 1", s->d);
    if (s->d > FMC_MAX_DISTURBANCES)
        return fail(ctx, FMC_EUNSUPPORTED, "d = %d above %d", s->d, FMC_MAX_DISTURBANCES);
    if (s->K < 1) return fail(ctx, FMC_EINVAL, "K = %d < 1", s->K);
    if ((int64_t)s->d * s->K > (1 << 24)) return fail(ctx, FMC_EINVAL, "d*K too large");
    if (s->N < 1 || s->N > (int64_t(1) << 30)) return fail(ctx, FMC_EINVAL, "N = %lld outside [1, 2^30]", (long long)s->N);
    if (s->sampling < 0 || s->sampling > 3) return fail(ctx, FMC_EINVAL, "sampling mode %d", s->sampling);
    if (s->correlation != FMC_CORR_NONE && s->correlation != FMC_CORR_RANK)
        return fail(ctx, FMC_EINVAL, "correlation option %d", s->correlation);
    if (s->correlation == FMC_CORR_RANK) {
        const int64_t M = (int64_t)s->d * s->K;
        if (s->sampling != FMC_LHS && s->sampling != FMC_LHS_MIDPOINT)
            return fail(ctx, FMC_EINVAL, "the correlation-reducing permutation needs an LHS design");
        if (s->N <= M || M > 4096 || s->N * M >= (int64_t(1) << 31))
            return fail(ctx, FMC_EINVAL, "the correlation-reducing permutation needs d K < N, d K <= 4096, N d K < 2^31");
    }
    if (s->precision < 0 || s->precision > 2) return fail(ctx, FMC_EINVAL, "precision %d", s->precision);
    if (s->integrator != FMC_RK4 && s->integrator != FMC_HEUN)
        return fail(ctx, FMC_EINVAL, "integrator %d", s->integrator);
    if (s->basis != FMC_BASIS_SINE && s->basis != FMC_BASIS_COSINE) return fail(ctx, FMC_EINVAL, "basis %d", s->basis);
    if (s->event_machine >= s->n) return fail(ctx, FMC_EINVAL, "event machine %d of %d", s->event_machine, s->n);
    if (s->forcing != FMC_FORCING_INCREMENTS && s->forcing != FMC_FORCING_SMOOTH)
        return fail(ctx, FMC_EINVAL, "forcing %d", s->forcing);
    if (s->forcing == FMC_FORCING_SMOOTH && s->sampling == FMC_SRS_EM)
        return fail(ctx, FMC_EINVAL, "per-step normals have no smooth forcing");
    if (s->ito) {
        for (int q = 0; q < s->d; ++q) {
            const fmc_ito& m = s->ito[q];
            if (m.kind != FMC_ITO_OU && m.kind != FMC_ITO_POLY && m.kind != FMC_ITO_SQRT)
                return fail(ctx, FMC_EINVAL, "disturbance %d: model kind %d", q, m.kind);
            bool fin = std::isfinite(m.a) && std::isfinite(m.x0);
            for (double c : m.m) fin = fin && std::isfinite(c);
            for (double c : m.s) fin = fin && std::isfinite(c);
            for (double c : m.v) fin = fin && std::isfinite(c);
            if (!fin) return fail(ctx, FMC_EINVAL, "disturbance %d: coefficients must be finite", q);
        }
    }
    if (s->event_machine >= 0) {
        if (!(s->event_time >= 0.0) || !std::isfinite(s->event_time) || !std::isfinite(s->event_dpm))
            return fail(ctx, FMC_EINVAL, "event time and power step must be finite, time >= 0");
        if (s->d + 1 > FMC_MAX_DISTURBANCES)
            return fail(ctx, FMC_EUNSUPPORTED, "an event takes a disturbance slot: d <= %d", FMC_MAX_DISTURBANCES - 1);
    }
    if (!s->G || !s->B || !s->H || !s->D || !s->E || !s->Pm || !s->theta || !s->sigma || !s->inject)
        return fail(ctx, FMC_EINVAL, "a scenario array is NULL");
    if (s->has_inf_bus && (!s->Ginf || !s->Binf)) return fail(ctx, FMC_EINVAL, "infinite bus arrays are NULL");
    for (int i = 0; i < s->n; ++i)
        if (!(s->H[i] > 0.0)) return fail(ctx, FMC_EINVAL, "H[%d] must be > 0", i);
    if (!(s->omega_s > 0.0)) return fail(ctx, FMC_EINVAL, "omega_s must be > 0");
    return steps_of(ctx, s->T, s->dt, Nt);
}

// General disturbances in the kernels' form (see ItoParams): the polynomials of
// fmc_ito re-expanded about x0 in FP64 and rounded; the Stratonovich correction
// applies to KL-driven paths.
template <int ND>
static void build_ito(const fmc_scenario* s, ItoParams<ND>& it)
{
    memset(&it, 0, sizeof it);
    if (!s->ito) return;
    it.strat = (s->sampling == FMC_SRS_EM) ? 0.f : 1.f;
    for (int q = 0; q < s->d && q < ND; ++q) {
        const fmc_ito& m = s->ito[q];
        it.kind[q] = m.kind;
        if (m.kind == FMC_ITO_OU) continue;
        it.on = 1;
        const double x0 = m.x0;
        it.c0[q] = (float)(m.m[0] + m.m[1] * x0 + m.m[2] * x0 * x0);
        it.c1[q] = (float)(m.m[1] + 2.0 * m.m[2] * x0);
        it.c2[q] = (float)m.m[2];
        if (m.kind == FMC_ITO_POLY) {
            it.e0[q] = (float)(m.s[0] + m.s[1] * x0 + m.s[2] * x0 * x0);
            it.e1[q] = (float)(m.s[1] + 2.0 * m.s[2] * x0);
            it.e2[q] = (float)m.s[2];
        } else {
            it.e0[q] = (float)(m.v[0] + m.v[1] * x0 + m.v[2] * x0 * x0);
            it.e1[q] = (float)(m.v[1] + 2.0 * m.v[2] * x0);
            it.e2[q] = (float)m.v[2];
            it.e3[q] = (float)m.v[3];
            it.ap[q] = (float)(m.a - x0);
        }
    }
}

// Grid step at which an event takes effect.
static int event_step_of(const fmc_scenario* s) { return (int)std::llround(s->event_time / s->dt); }

static int nd_bucket_for(int d)
{
    static const int buckets[] = {1, 2, 4, 8};
    for (int b : buckets)
        if (d <= b) return b;
    return -1;
}


// Integrator constants in the rotated deviation form (see swing_step_impl), all
// from the FP64 equilibrium and rounded once: the network coupling at the
// equilibrium angles A_ij = E_iE_j(G_ij cos d*_ij + B_ij sin d*_ij), Bm_ij =
// E_iE_j(B_ij cos d*_ij - G_ij sin d*_ij) without the diagonal, the machine's
// off-diagonal equilibrium power P*_i = c*_i u*_i + s*_i v*_i and its quadrature
// Q*_i = c*_i v*_i - s*_i u*_i (u*, v* the product-form sums, the infinite bus
// included), every row divided by 2 H_i.
template <int NM, int ND>
static void build_params(const fmc_scenario* s, const double* delta0, std::vector<unsigned char>& out)
{
    out.assign(sizeof(SwingParams<NM, ND>), 0);
    SwingParams<NM, ND>& p = *reinterpret_cast<SwingParams<NM, ND>*>(out.data());
    const int n = s->n, d = s->d;
    const bool rel = !s->has_inf_bus;
    std::vector<double> c(n), sn(n);
    for (int j = 0; j < n; ++j) {
        double a = rel ? delta0[j] - delta0[0] : delta0[j];
        c[j] = std::cos(a);
        sn[j] = std::sin(a);
    }
    for (int i = 0; i < n; ++i) {
        const double h = 1.0 / (2.0 * s->H[i]);
        double u = 0.0, v = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            const double ge = s->E[i] * s->E[j] * s->G[i * n + j];
            const double be = s->E[i] * s->E[j] * s->B[i * n + j];
            const double cij = c[i] * c[j] + sn[i] * sn[j];   // cos(d*_i - d*_j)
            const double sij = sn[i] * c[j] - c[i] * sn[j];   // sin(d*_i - d*_j)
            const double A = (ge * cij + be * sij) * h;
            const double Bm = (be * cij - ge * sij) * h;
            p.Ah[i][j] = (float)A;
            p.Bh[i][j] = (float)Bm;
            p.P1[i][j] = make_float2((float)A, (float)-Bm);
            p.P2[i][j] = make_float2((float)Bm, (float)A);
            u += ge * c[j] - be * sn[j];
            v += ge * sn[j] + be * c[j];
        }
        if (s->has_inf_bus) {
            u += s->E[i] * s->Vinf * s->Ginf[i];
            v += s->E[i] * s->Vinf * s->Binf[i];
        }
        p.pst[i] = (float)((c[i] * u + sn[i] * v) * h);
        p.qst[i] = (float)((c[i] * v - sn[i] * u) * h);
        p.dst[i] = (float)delta0[i];
        p.Dh[i] = (float)(s->D[i] * h);
        for (int q = 0; q < d; ++q) p.injh[i][q] = (float)(s->inject[i * d + q] * h);
    }
    for (int q = 0; q < d; ++q) {
        p.ou_a[q] = (float)(1.0 - s->theta[q] * s->dt);
        p.ou_s[q] = (float)s->sigma[q];
        p.th[q] = (float)s->theta[q];
    }
    double hsum = 0.0;
    for (int i = 0; i < n; ++i) hsum += s->H[i];
    for (int i = 0; i < n; ++i) p.hw[i] = (float)(s->H[i] / hsum);
    build_ito<ND>(s, p.ito);
    p.ev_slot = -1;
    p.ev_step = 0;
    if (s->event_machine >= 0) {
        // the event rides in the spare slot d: held at 0 before, 1 from the event step
        p.ev_slot = d;
        p.ev_step = event_step_of(s);
        p.injh[s->event_machine][d] = (float)(s->event_dpm / (2.0 * s->H[s->event_machine]));
        p.ou_a[d] = 1.f;
        p.ou_s[d] = 0.f;
    }
    p.omega_s = (float)s->omega_s;
    p.dt = (float)s->dt;
    p.d = d;
    p.n = n;
    p.integrator = s->integrator;
    p.rel = rel ? 1 : 0;
}

template <int NM>
static void build_params_nd(int nd, const fmc_scenario* s, const double* delta0, std::vector<unsigned char>& out)
{
    switch (nd) {
        case 1: build_params<NM, 1>(s, delta0, out); break;
        case 2: build_params<NM, 2>(s, delta0, out); break;
        case 4: build_params<NM, 4>(s, delta0, out); break;
        default: build_params<NM, 8>(s, delta0, out); break;
    }
}

static void build_params_bucket(int nm, int nd, const fmc_scenario* s, const double* delta0,
                                std::vector<unsigned char>& out)
{
    switch (nm) {
        case 1: build_params_nd<1>(nd, s, delta0, out); break;
        case 2: build_params_nd<2>(nd, s, delta0, out); break;
        case 4: build_params_nd<4>(nd, s, delta0, out); break;
        case 8: build_params_nd<8>(nd, s, delta0, out); break;
        case 10: build_params_nd<10>(nd, s, delta0, out); break;
        case 12: build_params_nd<12>(nd, s, delta0, out); break;
        default: build_params_nd<16>(nd, s, delta0, out); break;
    }
}

// Nearest TF32 value (ties to even) of x, as an FP32 number.
static float tf32_round(double x)
{
    float f = (float)x;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) {
        u += 0x0fffu + ((u >> 13) & 1u);
        u &= 0xffffe000u;
    }
    std::memcpy(&f, &u, 4);
    return f;
}

// Offset (floats) of the tensor-core network matrix in the constant block.
static size_t wide_net_offset(int n, int nmt, int nd) { return ((size_t)wide_const_floats(n, nmt, nd) + 31) & ~(size_t)31; }

// The network matrix of the tensor-core sum (wide_tc.cuh) into hi_lo (FP32
// [2][NN][NN], zeroed here): Net[(i, u|v)][(j, gamma|eta)] =
//   u: ( GE_ij, -BE_ij ),  v: ( BE_ij, GE_ij ),  diagonal and padding zero,
// row and column of machine i at (i mod H) KH + 2 (i / H), as Net_hi = TF32(Net)
// and Net_lo = TF32(Net - Net_hi); an infinite bus is a node in the last machine
// slot (E = V, G_ib = Ginf_i, B_ib = Binf_i), which the kernel fills with the
// bus's deviation in its shifted frame.
static void build_wide_net(const fmc_scenario* s, int nmt, int H, float* hi_lo)
{
    const int n = s->n, KH = wide_kh(nmt), NN = wide_nn(nmt, H);
    float* hi = hi_lo;
    float* lo = hi + (size_t)NN * NN;
    std::fill(hi, hi + 2 * (size_t)NN * NN, 0.f);
    auto put = [&](int row, int col, double x) {
        const float h = tf32_round(x);
        hi[(size_t)row * NN + col] = h;
        lo[(size_t)row * NN + col] = tf32_round(x - (double)h);
    };
    for (int i = 0; i < n; ++i) {
        const int ru = (i % H) * KH + 2 * (i / H);
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            const int cg = (j % H) * KH + 2 * (j / H);
            const double ge = s->E[i] * s->E[j] * s->G[i * n + j];
            const double be = s->E[i] * s->E[j] * s->B[i * n + j];
            put(ru, cg, ge);
            put(ru, cg + 1, -be);
            put(ru + 1, cg, be);
            put(ru + 1, cg + 1, ge);
        }
        if (s->has_inf_bus) {
            const int nb = H * nmt - 1;  // the last machine slot (free: n < H nmt)
            const int cb = (nb % H) * KH + 2 * (nb / H);
            const double ge = s->E[i] * s->Vinf * s->Ginf[i];
            const double be = s->E[i] * s->Vinf * s->Binf[i];
            put(ru, cb, ge);
            put(ru, cb + 1, -be);
            put(ru + 1, cb, be);
            put(ru + 1, cb + 1, ge);
        }
    }
}

// Constant block of the large-system kernel (layout at wide_const_floats): the
// same deviation-form constants as build_params, with the network matrices
// arranged [j][h][k] for machine i = h + 4k; with tcn, the tensor-core network
// matrix after it.
static void build_wide_consts(const fmc_scenario* s, const double* delta0, int nmt, int nd, bool tcn, int H,
                              std::vector<float>& out)
{
    const int n = s->n, d = s->d, nmtp = wide_nmtp(nmt), g4 = 4 * nmt;
    out.assign(wide_const_floats(n, nmt, nd), 0.f);  // nd: the kernel's disturbance-slot bucket
    float* GB = out.data();  // [j][h][GE row | BE row], nmtp each
    float* pm = GB + 2 * n * 4 * nmtp;
    const bool rel = !s->has_inf_bus;
    std::vector<double> c(n), sn(n);
    for (int j = 0; j < n; ++j) {
        double a = rel ? delta0[j] - delta0[0] : delta0[j];
        c[j] = std::cos(a);
        sn[j] = std::sin(a);
    }
    for (int i = 0; i < n; ++i) {
        const int h = i % 4, k = i / 4;
        double u = 0.0, v = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double ge = s->E[i] * s->E[j] * s->G[i * n + j];
            double be = s->E[i] * s->E[j] * s->B[i * n + j];
            GB[(j * 4 + h) * 2 * nmtp + k] = (float)ge;
            GB[(j * 4 + h) * 2 * nmtp + nmtp + k] = (float)(wide_packed(nmt) ? -be : be);  // see the kernel's network sum
            u += ge * c[j] - be * sn[j];
            v += ge * sn[j] + be * c[j];
        }
        if (s->has_inf_bus) {
            u += s->E[i] * s->Vinf * s->Ginf[i];
            v += s->E[i] * s->Vinf * s->Binf[i];
        }
        pm[0 * g4 + i] = (float)c[i];
        pm[1 * g4 + i] = (float)sn[i];
        pm[2 * g4 + i] = (float)u;
        pm[3 * g4 + i] = (float)v;
        pm[4 * g4 + i] = (float)delta0[i];
        pm[5 * g4 + i] = (float)(1.0 / (2.0 * s->H[i]));
        pm[6 * g4 + i] = (float)s->D[i];
        for (int q = 0; q < d; ++q) pm[(8 + q) * g4 + i] = (float)s->inject[i * d + q];
    }
    double hsum = 0.0;
    for (int i = 0; i < n; ++i) hsum += s->H[i];
    for (int i = 0; i < n; ++i) pm[7 * g4 + i] = (float)(s->H[i] / hsum);
    if (s->event_machine >= 0) pm[(8 + d) * g4 + s->event_machine] = (float)s->event_dpm;
    // (GB and pm point into out: nothing below writes through them, out may move)
    if (tcn) {
        // the network matrix of the tensor-core sum, 128-byte aligned after the
        // constant block
        const int NN = wide_nn(nmt, H);
        const size_t base = (out.size() + 31) & ~(size_t)31;
        out.resize(base + 2 * (size_t)NN * NN, 0.f);
        build_wide_net(s, nmt, H, out.data() + base);
    }
}

// Copies the system arrays to the device and launches the FP64 Newton kernel.
// eq: [delta0 n][pm n][shift 2n]; status: iteration count or -1.
static int run_equilibrium_ws(fmc_ctx* ctx, Workspace& ws, const fmc_scenario* s, cudaStream_t st)
{
    const int n = s->n;
    size_t nd = (size_t)2 * n * n + 5 * (size_t)n;
    int rc = ensure(ctx, ws.scen, nd * sizeof(double));
    if (rc) return rc;
    rc = ensure(ctx, ws.eq, 4 * (size_t)n * sizeof(double));
    if (rc) return rc;
    rc = ensure(ctx, ws.status, 64);
    if (rc) return rc;
    std::vector<double> h(nd, 0.0);
    double* G = h.data();
    double* B = G + n * n;
    double* Gi = B + n * n;
    double* Bi = Gi + n;
    double* E = Bi + n;
    double* Pm = E + n;
    memcpy(G, s->G, sizeof(double) * n * n);
    memcpy(B, s->B, sizeof(double) * n * n);
    if (s->has_inf_bus) {
        memcpy(Gi, s->Ginf, sizeof(double) * n);
        memcpy(Bi, s->Binf, sizeof(double) * n);
    }
    memcpy(E, s->E, sizeof(double) * n);
    memcpy(Pm, s->Pm, sizeof(double) * n);
    double* dG = (double*)ws.scen.ptr;
    FMC_CUDA(ctx, cudaMemcpyAsync(dG, h.data(), nd * sizeof(double), cudaMemcpyHostToDevice, st), "copy scenario");
    ProfRec* pr;
    prof_begin(ctx, PH_EQ, st, &pr);
    FMC_CUDA(ctx,
             launch_equilibrium(n, s->has_inf_bus, s->Vinf, dG, dG + n * n, dG + 2 * n * n, dG + 2 * n * n + n,
                                dG + 2 * n * n + 2 * n, dG + 2 * n * n + 3 * n, (double*)ws.eq.ptr,
                                (int*)ws.status.ptr, st),
             "equilibrium kernel");
    prof_end(pr, st);
    return FMC_OK;
}

static int run_equilibrium(fmc_ctx* ctx, const fmc_scenario* s, cudaStream_t st)
{
    return run_equilibrium_ws(ctx, ctx->ws, s, st);
}

// Tensor map of the tensor-core network matrix: FP32 [2 NN][NN] (Net_hi rows,
// then Net_lo rows), boxes of 16 values x NN rows, 64-byte swizzle.
static int make_map_net(fmc_ctx* ctx, CUtensorMap* m, const void* base, int NN)
{
    PFN_encodeTiled enc = get_encode();
    if (!enc) return fail(ctx, FMC_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)NN, (cuuint64_t)(2 * NN)};
    cuuint64_t strides[1] = {(cuuint64_t)NN * 4};
    cuuint32_t box[2] = {16, (cuuint32_t)NN};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, FMC_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return FMC_OK;
}

static int make_map_bf16(fmc_ctx* ctx, CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer,
                         uint32_t box_inner, uint32_t box_outer)
{
    PFN_encodeTiled enc = get_encode();
    if (!enc) return fail(ctx, FMC_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, FMC_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return FMC_OK;
}

// Tensor maps of the split operands: zeta [rows][d*Ks] in tiles of TM rows,
// phi [Nt][Kpad] in tiles of TN rows.
static int make_contract_maps_at(fmc_ctx* ctx, CUtensorMap maps[4], const void* zhi, const void* zlo, const void* phi_hi,
                                 const void* phi_lo, int64_t rows, int d, int Ks, int Nt, int Kpad, int TN, int split,
                                 int TM = TC_M)
{
    int rc = make_map_bf16(ctx, &maps[0], zhi, (uint64_t)d * Ks, (uint64_t)rows, TC_BK, (uint32_t)TM);
    if (rc) return rc;
    rc = make_map_bf16(ctx, &maps[2], phi_hi, (uint64_t)Kpad, (uint64_t)Nt, TC_BK, (uint32_t)TN);
    if (rc) return rc;
    if (split) {
        rc = make_map_bf16(ctx, &maps[1], zlo, (uint64_t)d * Ks, (uint64_t)rows, TC_BK, (uint32_t)TM);
        if (rc) return rc;
        rc = make_map_bf16(ctx, &maps[3], phi_lo, (uint64_t)Kpad, (uint64_t)Nt, TC_BK, (uint32_t)TN);
        if (rc) return rc;
    } else {
        maps[1] = maps[0];
        maps[3] = maps[2];
    }
    return FMC_OK;
}

static int make_contract_maps(fmc_ctx* ctx, CUtensorMap maps[4], int64_t rows, int d, int Ks, int Nt, int Kpad, int TN,
                              int split)
{
    return make_contract_maps_at(ctx, maps, ctx->zeta_hi.ptr, ctx->zeta_lo.ptr, ctx->phi_hi.ptr, ctx->phi_lo.ptr, rows,
                                 d, Ks, Nt, Kpad, TN, split);
}

// ---- scratch of the allocation-free reconstruction -----------------------------
// A fixed device array of this module serves as the only working memory of
// fmc_kle_reconstruct_noalloc.  Host code may not use the array's name as a
// device address: the address is obtained once per device, with that device
// current, by cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FMC_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64];

static int noalloc_scratch(fmc_ctx* ctx, unsigned char** out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const int dev = ctx->device;
    if (dev < 0 || dev >= 64) return fail(ctx, FMC_EUNSUPPORTED, "device ordinal %d above 63", dev);
    if (!g_noalloc_addr[dev]) {
        int prev = -1;
        FMC_CUDA(ctx, cudaGetDevice(&prev), "cudaGetDevice");
        if (prev != dev) FMC_CUDA(ctx, cudaSetDevice(dev), "cudaSetDevice");
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (prev != dev) cudaSetDevice(prev);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
    return FMC_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// The first bytes of the scratch array: word 1 is the last allocation-free
// call's device error code (0: none), read by fmc_device_status.
static constexpr size_t NOALLOC_STATUS_BYTES = 256;

// The device address of the scratch array on the context's device if an
// allocation-free call (or the self-check) has looked it up, else nullptr.
static void* noalloc_scratch_if_known(const fmc_ctx* ctx)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const int dev = ctx->device;
    return (dev >= 0 && dev < 64) ? g_noalloc_addr[dev] : nullptr;
}

extern "C" {

int fmc_create(fmc_ctx** out, int device, size_t mem_budget_bytes)
{
    if (!out) {
        g_create_err = "out is NULL";
        return FMC_EINVAL;
    }
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        g_create_err = std::string("no CUDA device ") + std::to_string(device) + ": " + cudaGetErrorString(e);
        cudaGetLastError();
        return FMC_ECUDA;
    }
    e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        g_create_err = cudaGetErrorString(e);
        return FMC_ECUDA;
    }
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        g_create_err = cudaGetErrorString(e);
        return FMC_ECUDA;
    }
    if (prop.major * 10 + prop.minor < 100) {
        g_create_err = "this library needs a Blackwell GPU (sm_103a)";
        return FMC_EUNSUPPORTED;
    }
    fmc_ctx* c = new fmc_ctx();
    c->device = device;
    c->sms = prop.multiProcessorCount;
    c->l2_bytes = prop.l2CacheSize;
    snprintf(c->name, sizeof c->name, "%s", prop.name);
    c->budget = mem_budget_bytes;
    *out = c;
    return FMC_OK;
}

int fmc_destroy(fmc_ctx* ctx)
{
    if (!ctx) return FMC_EINVAL;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    prof_clear(ctx);
    DevBuf* bufs[] = {&ctx->zeta_hi, &ctx->zeta_lo, &ctx->phi_hi, &ctx->phi_lo, &ctx->phi32,  &ctx->dW,
                      &ctx->traj,    &ctx->part,    &ctx->eq,     &ctx->scen,   &ctx->status, &ctx->zeta32,
                      &ctx->wconst,  &ctx->rrfbuf, &ctx->ws.ic, &ctx->ws.ic_strata,
                      &ctx->ws.ident};
    for (DevBuf* b : bufs)
        if (b->ptr) cudaFree(b->ptr);
    delete ctx;
    return FMC_OK;
}

const char* fmc_last_error(const fmc_ctx* ctx)
{
    if (!ctx) return g_create_err.c_str();
    return ctx->err.c_str();
}

int fmc_device_info(const fmc_ctx* ctx, int* sm_count, char* name, size_t name_len)
{
    if (!ctx) return FMC_EINVAL;
    if (sm_count) *sm_count = ctx->sms;
    if (name && name_len) snprintf(name, name_len, "%s", ctx->name);
    return FMC_OK;
}

int fmc_lhs_sample(fmc_ctx* ctx, uint64_t seed, int64_t N, int64_t k0, int64_t count, int32_t M, int32_t mode,
                   float* zeta_dev, uint32_t* strata_dev, void* stream)
{
    if (!ctx) return FMC_EINVAL;
    if (N < 1 || N > (int64_t(1) << 30)) return fail(ctx, FMC_EINVAL, "N = %lld outside [1, 2^30]", (long long)N);
    if (M < 1) return fail(ctx, FMC_EINVAL, "M = %d < 1", M);
    if (k0 < 0 || count < 0 || k0 + count > N) return fail(ctx, FMC_EINVAL, "rows [k0, k0+count) outside [0, N)");
    if (mode < 0 || mode > 2) return fail(ctx, FMC_EINVAL, "mode %d", mode);
    if (!zeta_dev && !strata_dev) return fail(ctx, FMC_EINVAL, "both outputs are NULL");
    cudaStream_t st = (cudaStream_t)stream;
    ProfRec* pr;
    prof_begin(ctx, PH_LHS, st, &pr);
    FMC_CUDA(ctx, launch_lhs_f32(seed, N, k0, count, M, mode, zeta_dev, strata_dev, ctx->sms, st), "lhs kernel");
    prof_end(pr, st);
    return FMC_OK;
}

int fmc_lhs_sample_split(fmc_ctx* ctx, uint64_t seed, int64_t N, int64_t k0, int64_t count, int32_t d, int32_t K,
                         int32_t mode, uint16_t* hi_dev, uint16_t* lo_dev, void* stream)
{
    if (!ctx) return FMC_EINVAL;
    if (N < 1 || N > (int64_t(1) << 30)) return fail(ctx, FMC_EINVAL, "N = %lld outside [1, 2^30]", (long long)N);
    if (d < 1 || K < 1) return fail(ctx, FMC_EINVAL, "d = %d, K = %d", d, K);
    if (k0 < 0 || count < 0 || k0 + count > N) return fail(ctx, FMC_EINVAL, "rows [k0, k0+count) outside [0, N)");
    if (mode < 0 || mode > 2) return fail(ctx, FMC_EINVAL, "mode %d", mode);
    if (!hi_dev) return fail(ctx, FMC_EINVAL, "hi output is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    FMC_CUDA(ctx, launch_lhs_split(seed, N, k0, count, d, K, mode, hi_dev, lo_dev, ctx->sms, st), "lhs kernel");
    return FMC_OK;
}

}  // extern "C"

// The correlation-reducing permutation of the whole N-sample design (see
// fmc_lhs_decorrelate) into ws.ic_strata [M][N]; synchronises st to read back
// whether the score correlation factorised.
static int run_decorrelate(fmc_ctx* ctx, Workspace& ws, uint64_t seed, int64_t N, int M, cudaStream_t st)
{
    int rc;
    const size_t NM = (size_t)N * M, MM = (size_t)M * M;
    const size_t sort = ic_sort_bytes(N, M);
    // carve the working memory: a, mom, G | R, Rs, A, B | vals, vals_out | off, ok | sort
    size_t off[16], o = 0;
    auto take = [&](int k, size_t bytes) { off[k] = o; o += (bytes + 255) & ~(size_t)255; };
    take(0, N * sizeof(double));
    take(1, 2 * sizeof(double));
    take(2, MM * sizeof(double));
    take(3, NM * sizeof(float));
    take(4, NM * sizeof(float));
    take(5, MM * sizeof(float));
    take(6, MM * sizeof(float));
    take(7, NM * sizeof(uint32_t));
    take(8, NM * sizeof(uint32_t));
    take(9, (M + 1) * sizeof(int));
    take(10, sizeof(int));
    take(11, sort);
    if ((rc = ensure(ctx, ws.ic, o))) return rc;
    if ((rc = ensure(ctx, ws.ic_strata, NM * sizeof(uint32_t)))) return rc;
    char* b = static_cast<char*>(ws.ic.ptr);
    IcWork w{reinterpret_cast<double*>(b + off[0]), reinterpret_cast<double*>(b + off[1]),
             reinterpret_cast<float*>(b + off[3]),  reinterpret_cast<float*>(b + off[4]),
             reinterpret_cast<double*>(b + off[2]), reinterpret_cast<float*>(b + off[5]),
             reinterpret_cast<float*>(b + off[6]),  reinterpret_cast<uint32_t*>(b + off[7]),
             reinterpret_cast<uint32_t*>(b + off[8]), reinterpret_cast<int*>(b + off[9]),
             reinterpret_cast<int*>(b + off[10]),   b + off[11], sort};
    FMC_CUDA(ctx, launch_ic_strata(seed, N, M, w, (uint32_t*)ws.ic_strata.ptr, ctx->sms, st),
             "correlation-reducing permutation");
    int ok = 0;
    FMC_CUDA(ctx, cudaMemcpyAsync(&ok, w.ok, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
    FMC_CUDA(ctx, cudaStreamSynchronize(st), "sync");
    if (!ok) return fail(ctx, FMC_EINVAL, "the design's score correlation is not positive definite");
    return FMC_OK;
}

extern "C" {

int fmc_lhs_decorrelate(fmc_ctx* ctx, uint64_t seed, int64_t N, int32_t M, int32_t mode, float* zeta_dev,
                        uint32_t* strata_dev, void* stream)
{
    if (!ctx) return FMC_EINVAL;
    if (mode != FMC_LHS && mode != FMC_LHS_MIDPOINT) return fail(ctx, FMC_EINVAL, "mode %d is not an LHS mode", mode);
    if (N < 2 || M < 1 || M >= N || M > 4096 || N * (int64_t)M >= (int64_t(1) << 31))
        return fail(ctx, FMC_EINVAL, "N = %lld, M = %d: needs 2 <= N, M < N, M <= 4096, N M < 2^31", (long long)N, M);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = run_decorrelate(ctx, ctx->ws, seed, N, M, st);
    if (rc) return rc;
    const uint32_t* strata = (const uint32_t*)ctx->ws.ic_strata.ptr;
    if (zeta_dev) FMC_CUDA(ctx, launch_ic_values(seed, N, 0, N, M, mode, strata, zeta_dev, ctx->sms, st), "values");
    if (strata_dev)
        FMC_CUDA(ctx, cudaMemcpyAsync(strata_dev, strata, (size_t)N * M * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st),
                 "copy");
    return FMC_OK;
}

}  // extern "C"

// L' (and with derivs its gradient and Hessian) of the record at q, read back:
// h_out [43]; returns FMC_OK, with *finite = 0 where some D_j <= 0.
static int ident_eval(fmc_ctx* ctx, int kind, const double* q, const double* xi, int64_t n, double h, int derivs,
                      double* h_out, int* finite, cudaStream_t st)
{
    int rc;
    if ((rc = ensure(ctx, ctx->ws.ident, 512))) return rc;
    double* out = static_cast<double*>(ctx->ws.ident.ptr);
    int* bad = reinterpret_cast<int*>(out + 43);
    FMC_CUDA(ctx, launch_ito_objective(kind, q, xi, n, h, derivs, out, bad, ctx->sms, st), "objective kernel");
    int hb = 0;
    FMC_CUDA(ctx, cudaMemcpyAsync(h_out, out, sizeof(double) * (derivs ? 43 : 1), cudaMemcpyDeviceToHost, st), "copy");
    FMC_CUDA(ctx, cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
    FMC_CUDA(ctx, cudaStreamSynchronize(st), "sync");
    *finite = hb == 0 && std::isfinite(h_out[0]);
    return FMC_OK;
}

static int ident_check(fmc_ctx* ctx, int32_t kind, const double* xi, int64_t n, double h)
{
    if (kind != FMC_IDENT_SIGMA && kind != FMC_IDENT_SIGMA2) return fail(ctx, FMC_EINVAL, "identification kind %d", kind);
    if (!xi || n < 8) return fail(ctx, FMC_EINVAL, "the record needs at least 8 values");
    if (!(h > 0.0) || !std::isfinite(h)) return fail(ctx, FMC_EINVAL, "sampling interval h = %g", h);
    return FMC_OK;
}

extern "C" {

int fmc_ito_objective(fmc_ctx* ctx, int32_t kind, const double* q, const double* xi_dev, int64_t n, double h,
                      double* L, double* grad, double* hess, void* stream)
{
    if (!ctx) return FMC_EINVAL;
    int rc = ident_check(ctx, kind, xi_dev, n, h);
    if (rc) return rc;
    if (!q || !L) return fail(ctx, FMC_EINVAL, "NULL q or L");
    double o[43];
    int finite = 0;
    const int derivs = (grad || hess) ? 1 : 0;
    if ((rc = ident_eval(ctx, kind, q, xi_dev, n, h, derivs, o, &finite, (cudaStream_t)stream))) return rc;
    *L = finite ? o[0] : HUGE_VAL;
    if (grad) memcpy(grad, o + 1, 6 * sizeof(double));
    if (hess) memcpy(hess, o + 7, 36 * sizeof(double));
    return FMC_OK;
}

int fmc_ito_identify(fmc_ctx* ctx, int32_t kind, const double* xi_dev, int64_t n, double h, double* q,
                     int32_t* iterations, void* stream)
{
    if (!ctx) return FMC_EINVAL;
    int rc = ident_check(ctx, kind, xi_dev, n, h);
    if (rc) return rc;
    if (!q) return fail(ctx, FMC_EINVAL, "NULL q");
    cudaStream_t st = (cudaStream_t)stream;
    double o[43];
    int finite = 0;
    if ((rc = ident_eval(ctx, kind, q, xi_dev, n, h, 1, o, &finite, st))) return rc;
    if (!finite) return fail(ctx, FMC_EINVAL, "the start gives a non-positive diffusion on the record");
    double* dev = static_cast<double*>(ctx->ws.ident.ptr);
    double* step_dev = dev + 44;
    int* ok_dev = reinterpret_cast<int*>(dev + 50);
    double L = o[0];
    for (int it = 1; it <= 200; ++it) {
        double dmax = 0.0;
        for (int a = 0; a < 6; ++a) dmax = std::max(dmax, std::fabs(o[7 + a * 7]));
        // the sums of the current point are on the device (out); shift until the
        // Cholesky factorisation succeeds
        double lambda = 0.0, step[6];
        for (;;) {
            int ok = 0;
            FMC_CUDA(ctx, launch_ito_newton_step(dev, lambda, step_dev, ok_dev, st), "newton step kernel");
            FMC_CUDA(ctx, cudaMemcpyAsync(&ok, ok_dev, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
            FMC_CUDA(ctx, cudaMemcpyAsync(step, step_dev, sizeof step, cudaMemcpyDeviceToHost, st), "copy");
            FMC_CUDA(ctx, cudaStreamSynchronize(st), "sync");
            if (ok) break;
            lambda = lambda == 0.0 ? 1e-10 * dmax : 10.0 * lambda;
            if (lambda > 1e30) return fail(ctx, FMC_ENOCONVERGE, "the Hessian could not be made positive definite");
        }
        // the Newton decrement: once the predicted decrease is below the rounding of
        // the sums (whose order the atomics leave free), the point is the minimum
        double pred = 0.0;
        for (int a = 0; a < 6; ++a) pred -= o[1 + a] * step[a];
        if (lambda == 0.0 && pred <= 1e-12 * std::max(1.0, std::fabs(L))) {
            if (iterations) *iterations = it;
            return FMC_OK;
        }
        double t = 1.0, qn[6], Ln = HUGE_VAL;
        int f2 = 0;
        for (int ls = 0; ls < 60; ++ls, t *= 0.5) {
            for (int a = 0; a < 6; ++a) qn[a] = q[a] + t * step[a];
            double l1;
            if ((rc = ident_eval(ctx, kind, qn, xi_dev, n, h, 0, &l1, &f2, st))) return rc;
            Ln = f2 ? l1 : HUGE_VAL;
            if (Ln <= L) break;
        }
        if (!(Ln <= L)) return fail(ctx, FMC_ENOCONVERGE, "the line search found no decrease");
        double dq = 0.0, qs = 0.0;
        for (int a = 0; a < 6; ++a) {
            dq += (qn[a] - q[a]) * (qn[a] - q[a]);
            qs += qn[a] * qn[a];
            q[a] = qn[a];
        }
        if ((rc = ident_eval(ctx, kind, q, xi_dev, n, h, 1, o, &finite, st))) return rc;
        L = o[0];
        if (lambda == 0.0 && dq <= 1e-24 * (qs + 1e-300)) {
            if (iterations) *iterations = it;
            return FMC_OK;
        }
    }
    return fail(ctx, FMC_ENOCONVERGE, "no convergence in 200 Newton iterations");
}

int fmc_kl_basis(fmc_ctx* ctx, int32_t K, double T, int32_t Nt, int32_t basis, float* phi_dev, void* stream)
{
    if (!ctx) return FMC_EINVAL;
    if (basis != FMC_BASIS_SINE && basis != FMC_BASIS_COSINE) return fail(ctx, FMC_EINVAL, "basis %d", basis);
    if (K < 1 || Nt < 1 || !(T > 0.0)) return fail(ctx, FMC_EINVAL, "K = %d, Nt = %d, T = %g", K, Nt, T);
    if (!phi_dev) return fail(ctx, FMC_EINVAL, "phi is NULL");
    FMC_CUDA(ctx, launch_basis_f32(K, Nt, T, basis, phi_dev, ctx->sms, (cudaStream_t)stream), "basis kernel");
    return FMC_OK;
}

int fmc_kle_reconstruct(fmc_ctx* ctx, const float* zeta_dev, int64_t count, int32_t d, int32_t K, double T, double dt,
                        int32_t precision, float* dW_dev, void* stream)
{
    if (!ctx) return FMC_EINVAL;
    if (count < 1 || d < 1 || K < 1) return fail(ctx, FMC_EINVAL, "count, d, K must be >= 1");
    if (!zeta_dev || !dW_dev) return fail(ctx, FMC_EINVAL, "NULL buffer");
    int Nt = 0;
    int rc = steps_of(ctx, T, dt, &Nt);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == FMC_PREC_F32) {
        rc = ensure(ctx, ctx->phi32, (size_t)K * Nt * sizeof(float));
        if (rc) return rc;
        FMC_CUDA(ctx, launch_basis_f32(K, Nt, T, FMC_BASIS_SINE, (float*)ctx->phi32.ptr, ctx->sms, st), "basis kernel");
        FMC_CUDA(ctx, launch_sgemm_nn(count * d, Nt, K, zeta_dev, (const float*)ctx->phi32.ptr, dW_dev, st),
                 "sgemm kernel");
        return FMC_OK;
    }
    if (precision != FMC_PREC_BF16 && precision != FMC_PREC_BF16X3)
        return fail(ctx, FMC_EINVAL, "precision %d", precision);
    if (count > (int64_t(1) << 31) - 256) return fail(ctx, FMC_EINVAL, "count too large for the tensor-core path");
    const int split = (precision == FMC_PREC_BF16X3);
    const int Ks = round_up(K, 8);
    const int Kpad = round_up(K, TC_BK);
    const int nkb = (Ks + TC_BK - 1) / TC_BK;
    const int TN = 64;
    // split zeta [count][d*K] FP32 -> [count][d][Ks] BF16 hi/lo via a tiny conversion on the device
    size_t zbytes = (size_t)count * d * Ks * 2;
    if ((rc = ensure(ctx, ctx->zeta_hi, zbytes))) return rc;
    if ((rc = ensure(ctx, ctx->zeta_lo, zbytes))) return rc;
    if ((rc = ensure(ctx, ctx->phi_hi, (size_t)Nt * Kpad * 2))) return rc;
    if ((rc = ensure(ctx, ctx->phi_lo, (size_t)Nt * Kpad * 2))) return rc;
    if ((rc = ensure(ctx, ctx->status, 64))) return rc;
    FMC_CUDA(ctx, launch_split_rows(zeta_dev, count, d, K, Ks, ctx->zeta_hi.ptr, ctx->zeta_lo.ptr, st), "split");
    FMC_CUDA(ctx, launch_basis_split(K, Nt, T, FMC_BASIS_SINE, Kpad, ctx->phi_hi.ptr, ctx->phi_lo.ptr, ctx->sms, st), "basis");
    CUtensorMap maps[4];
    if ((rc = make_contract_maps(ctx, maps, count, d, Ks, Nt, Kpad, TN, split))) return rc;
    FMC_CUDA(ctx, cudaMemsetAsync(ctx->status.ptr, 0, 64, st), "memset");
    FMC_CUDA(ctx, launch_contract_tc(maps, count, d, Ks, nkb, Nt, TN, split, dW_dev, (int*)ctx->status.ptr + 1, st),
             "tensor-core contraction");
    return FMC_OK;
}

int fmc_kle_reconstruct_noalloc(fmc_ctx* ctx, const float* zeta_dev, int64_t count, int32_t d, int32_t K, double T,
                                double dt, int32_t precision, float* dW_dev, void* stream)
{
    if (!ctx) return FMC_EINVAL;
    if (count < 1 || d < 1 || K < 1) return fail(ctx, FMC_EINVAL, "count, d, K must be >= 1");
    if (!zeta_dev || !dW_dev) return fail(ctx, FMC_EINVAL, "NULL buffer");
    int Nt = 0;
    int rc = steps_of(ctx, T, dt, &Nt);
    if (rc) return rc;
    if (precision != FMC_PREC_F32 && precision != FMC_PREC_BF16 && precision != FMC_PREC_BF16X3)
        return fail(ctx, FMC_EINVAL, "precision %d", precision);
    cudaStream_t st = (cudaStream_t)stream;
    // the kernels run on the caller's current device, which must be the one whose
    // scratch array is addressed
    int cur = -1;
    FMC_CUDA(ctx, cudaGetDevice(&cur), "cudaGetDevice");
    if (cur != ctx->device)
        return fail(ctx, FMC_EINVAL, "the current device (%d) is not the context's device (%d)", cur, ctx->device);
    const int Ks = round_up(K, 8);
    const int Kpad = round_up(K, TC_BK);
    // layout of the scratch array for this call: the status words first, at a
    // fixed place that fmc_device_status reads, then the working buffers
    size_t need;
    const size_t o_status = 0;
    size_t o_zhi = 0, o_zlo = 0, o_phi_hi = 0, o_phi_lo = 0, o_phi32 = 0;
    if (precision == FMC_PREC_F32) {
        o_phi32 = NOALLOC_STATUS_BYTES;
        need = o_phi32 + align256((size_t)K * Nt * sizeof(float));
    } else {
        const size_t zb = align256((size_t)count * d * Ks * 2);
        const size_t pb = align256((size_t)Nt * Kpad * 2);
        o_zhi = NOALLOC_STATUS_BYTES;
        o_zlo = o_zhi + zb;
        o_phi_hi = o_zlo + zb;
        o_phi_lo = o_phi_hi + pb;
        need = o_phi_lo + pb;
    }
    if (need > (size_t)FMC_NOALLOC_SCRATCH_BYTES)
        return fail(ctx, FMC_EINVAL,
                    "this reconstruction needs %zu bytes of working memory; the allocation-free form has %zu "
                    "(use fmc_kle_reconstruct)",
                    need, (size_t)FMC_NOALLOC_SCRATCH_BYTES);
    if (count > (int64_t(1) << 31) - 256) return fail(ctx, FMC_EINVAL, "count too large for the tensor-core path");
    unsigned char* base = nullptr;
    if ((rc = noalloc_scratch(ctx, &base))) return rc;
    int* status = reinterpret_cast<int*>(base + o_status);
    // the array keeps the previous call's contents: the error word must start at zero
    FMC_CUDA(ctx, cudaMemsetAsync(status, 0, NOALLOC_STATUS_BYTES, st), "memset");
    if (precision == FMC_PREC_F32) {
        float* phi32 = reinterpret_cast<float*>(base + o_phi32);
        FMC_CUDA(ctx, launch_basis_f32(K, Nt, T, FMC_BASIS_SINE, phi32, ctx->sms, st), "basis kernel");
        FMC_CUDA(ctx, launch_sgemm_nn(count * d, Nt, K, zeta_dev, phi32, dW_dev, st), "sgemm kernel");
        return FMC_OK;
    }
    const int split = (precision == FMC_PREC_BF16X3);
    const int nkb = (Ks + TC_BK - 1) / TC_BK;
    const int TN = 64;
    void* zhi = base + o_zhi;
    void* zlo = base + o_zlo;
    void* phi_hi = base + o_phi_hi;
    void* phi_lo = base + o_phi_lo;
    FMC_CUDA(ctx, launch_split_rows(zeta_dev, count, d, K, Ks, zhi, zlo, st), "split");
    FMC_CUDA(ctx, launch_basis_split(K, Nt, T, FMC_BASIS_SINE, Kpad, phi_hi, phi_lo, ctx->sms, st), "basis");
    CUtensorMap maps[4];
    if ((rc = make_contract_maps_at(ctx, maps, zhi, zlo, phi_hi, phi_lo, count, d, Ks, Nt, Kpad, TN, split)))
        return rc;
    FMC_CUDA(ctx, launch_contract_tc(maps, count, d, Ks, nkb, Nt, TN, split, dW_dev, status + 1, st),
             "tensor-core contraction");
    return FMC_OK;
}

int fmc_equilibrium(fmc_ctx* ctx, const fmc_scenario* scen, double* delta0, double* pm_eq)
{
    if (!ctx) return FMC_EINVAL;
    int Nt;
    int rc = check_scenario(ctx, scen, &Nt);
    if (rc) return rc;
    if (!delta0 || !pm_eq) return fail(ctx, FMC_EINVAL, "NULL output");
    cudaStream_t st = 0;
    if ((rc = run_equilibrium(ctx, scen, st))) return rc;
    const int n = scen->n;
    std::vector<double> h(2 * n);
    int status = 0;
    FMC_CUDA(ctx, cudaMemcpyAsync(h.data(), ctx->eq.ptr, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
    FMC_CUDA(ctx, cudaMemcpyAsync(&status, ctx->status.ptr, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
    FMC_CUDA(ctx, cudaStreamSynchronize(st), "sync");
    if (status < 0) return fail(ctx, FMC_ENOCONVERGE, "equilibrium Newton iteration did not converge");
    memcpy(delta0, h.data(), n * sizeof(double));
    memcpy(pm_eq, h.data() + n, n * sizeof(double));
    return FMC_OK;
}

// A scenario made ready for the device: checked, equilibrium solved (FP64 on the
// GPU, read back once), integrator constants formed for the parameter block.
struct Prepared {
    fmc_scenario s{};

    int Nt = 0, nm = 0, nd = 0, path = 0;
    int nmt = 0;  // > 0: the large-system kernel with nmt machine slots per thread
    bool tcn = false;  // the large-system kernel sums the network on the tensor cores
    int H = 4;         // its warps per sample (2: two CTAs per SM, nmt slots of 2)
    bool bus = false;  // ... for a system with an infinite bus (its own instantiations)
    bool exclusive = true;  // the launch has the GPU to itself (see fused_shape)
    int64_t k0 = 0, count = 0;
    std::vector<unsigned char> params;
};

// The fused kernel a launch takes and its layout (host logic only): the
// per-sample kernel, or the split kernel with its slots per thread, warps per
// sample, tensor-core network sum and infinite-bus form; and the disturbance-slot
// bucket.  user_policy: the caller's FMC_KERNEL_* (AUTO lets a matching rule of
// `rules`, if given, choose).  Messages go to ctx when it is given.
struct KernelChoice {
    int nm = 0, nmt = 0, nd = 0;
    bool tcn = false;  // the split kernel's network sums on the tensor cores
    int H = 4;         // its warps per sample (2: two CTAs per SM)
    bool bus = false;  // ... for a system with an infinite bus (its own instantiations)
};

// The first rule of `rules` that holds the scenario and sample count, or nullptr.
static const fmc_launch_rule* find_rule_in(const std::vector<fmc_launch_rule>& rules, const fmc_scenario* s,
                                           int64_t count)
{
    for (const fmc_launch_rule& r : rules)
        if (s->n >= r.n_min && s->n <= r.n_max && s->d >= r.d_min && s->d <= r.d_max && count >= r.N_min &&
            count <= r.N_max)
            return &r;
    return nullptr;
}

// The first launch rule that holds the scenario and sample count, or nullptr.
static const fmc_launch_rule* find_rule(const fmc_ctx* ctx, const fmc_scenario* s, int64_t count)
{
    return find_rule_in(ctx->rules, s, count);
}

static int choose_kernel(fmc_ctx* ctx, const std::vector<fmc_launch_rule>* rules, const fmc_scenario* s,
                         int64_t count, int32_t path, int32_t user_policy, KernelChoice& C)
{
    const int n = s->n;
    C.nm = nm_bucket_for(n);
    // four warps per sample for systems above 16 machines (or on request)
    int policy = user_policy;
    if (policy == FMC_KERNEL_AUTO && path == FMC_PATH_FUSED && rules) {
        // (a rule's kernel that cannot take this system is ignored: a bucket's
        // rule was measured at its largest machine count)
        const fmc_launch_rule* rule = find_rule_in(*rules, s, count);
        if (rule && rule->kernel != FMC_KERNEL_AUTO && !(rule->kernel == FMC_KERNEL_PER_SAMPLE && C.nm < 0) &&
            !(rule->kernel == FMC_KERNEL_SPLIT_TC && !wide_tc_built(wide_nmt_for(n))))
            policy = rule->kernel;
    }
    const bool per_sample = policy == FMC_KERNEL_PER_SAMPLE;
    if (path == FMC_PATH_FUSED && per_sample && C.nm < 0)
        return fail(ctx, FMC_EUNSUPPORTED, "the per-sample kernel handles up to %d machines (n = %d)",
                    FMC_MAX_MACHINES_PLAIN, n);
    if (path == FMC_PATH_FUSED && (policy == FMC_KERNEL_SPLIT || policy == FMC_KERNEL_SPLIT_TC))
        C.nmt = wide_nmt_for(n);
    else if (path == FMC_PATH_FUSED && per_sample)
        C.nmt = 0;
    else
        C.nmt = (C.nm < 0) ? wide_nmt_for(n) : 0;
    C.tcn = C.nmt > 0 && (policy == FMC_KERNEL_SPLIT_TC || (policy == FMC_KERNEL_AUTO && wide_tc_built(C.nmt)));
    if (policy == FMC_KERNEL_SPLIT_TC && !wide_tc_built(C.nmt))
        return fail(ctx, FMC_EUNSUPPORTED, "the tensor-core network sum handles 13 to %d machines (n = %d)",
                    FMC_MAX_MACHINES, n);
    // 17..28 machines: two warps per sample and two CTAs per SM (9 .. 14 slots
    // per thread), whose barriers and product waits overlap, where the halved
    // TMEM share holds the product's columns and a 16-step chunk of the
    // disturbances (up to 7 with 9..12 slots, 4 with 13 and 14)
    if (C.tcn && (C.nmt == 5 || C.nmt == 7)) {
        const int h2 = n <= 18 ? 9 : n <= 20 ? 10 : n <= 22 ? 11 : n <= 24 ? 12 : n <= 26 ? 13 : 14;
        // (13 and 14 slots are built for the disturbance-slot buckets up to 4,
        // the generator-trip slot included)
        const int ndx = nd_bucket_for(s->d + (s->event_machine >= 0 ? 1 : 0));
        if (16 * s->d + wide_tc_cols(h2, 2) <= 256 && (h2 < 13 || ndx <= 4)) {
            C.H = 2;
            C.nmt = h2;
        }
    }
    // an infinite bus: the tensor-core layout holds it in its last machine slot
    // (instantiated for four warps per sample and the 8-disturbance bucket)
    if (C.tcn && s->has_inf_bus) {
        C.H = 4;
        C.nmt = wide_nmt_for(n);
        C.bus = true;
        if (n >= 4 * C.nmt) {
            if (user_policy == FMC_KERNEL_SPLIT_TC)
                return fail(ctx, FMC_EUNSUPPORTED,
                            "the tensor-core network sum needs a free machine slot for the infinite bus (n = %d)",
                            n);
            C.tcn = false;
            C.bus = false;
        }
    }
    if (path == FMC_PATH_FUSED && s->forcing == FMC_FORCING_SMOOTH && C.nmt > 0)
        return fail(ctx, FMC_EUNSUPPORTED,
                    "the smooth forcing runs on the per-sample fused kernel (up to %d machines) and the plain path",
                    FMC_MAX_MACHINES_PLAIN);
    C.nd = C.bus ? 8 : nd_bucket_for(s->d + (s->event_machine >= 0 ? 1 : 0));
    return FMC_OK;
}

static int prepare(fmc_ctx* ctx, Workspace& ws, const fmc_scenario* s, int64_t k0, int64_t count, int32_t path,
                   cudaStream_t st, Prepared& P, bool exclusive = true)
{
    int Nt = 0;
    int rc = check_scenario(ctx, s, &Nt);
    if (rc) return rc;
    if (k0 < 0 || count < 1 || k0 + count > s->N)
        return fail(ctx, FMC_EINVAL, "sample block [%lld, %lld) outside [0, N)", (long long)k0,
                    (long long)(k0 + count));
    if (path != FMC_PATH_FUSED && path != FMC_PATH_PLAIN) return fail(ctx, FMC_EINVAL, "path %d", path);
    if (path == FMC_PATH_PLAIN && s->precision != FMC_PREC_F32)
        return fail(ctx, FMC_EINVAL, "the plain path computes in FP32 (precision FMC_PREC_F32)");
    if (path == FMC_PATH_FUSED && s->precision == FMC_PREC_F32)
        return fail(ctx, FMC_EINVAL, "the fused path contracts on tensor cores (BF16 or BF16X3)");
    const int n = s->n;
    if (path == FMC_PATH_PLAIN && n > FMC_MAX_MACHINES_PLAIN)
        return fail(ctx, FMC_EUNSUPPORTED, "the plain path handles up to %d machines (n = %d)",
                    FMC_MAX_MACHINES_PLAIN, n);
    P.s = *s;
    P.Nt = Nt;
    P.exclusive = exclusive;
    KernelChoice C;
    if ((rc = choose_kernel(ctx, &ctx->rules, s, count, path, exclusive ? ctx->kernel_policy : FMC_KERNEL_AUTO, C)))
        return rc;
    P.nm = C.nm;
    P.nmt = C.nmt;
    P.nd = C.nd;
    P.tcn = C.tcn;
    P.H = C.H;
    P.bus = C.bus;
    P.path = path;
    P.k0 = k0;
    P.count = count;
    // FP64 Newton on the GPU; its angles come back to the host (one stream
    // synchronisation) to form the integrator's constants in the parameter block
    if ((rc = run_equilibrium_ws(ctx, ws, s, st))) return rc;
    std::vector<double> delta0(n);
    int eq_status = 0;
    FMC_CUDA(ctx, cudaMemcpyAsync(delta0.data(), ws.eq.ptr, n * sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
    FMC_CUDA(ctx, cudaMemcpyAsync(&eq_status, ws.status.ptr, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
    FMC_CUDA(ctx, cudaStreamSynchronize(st), "sync");
    if (eq_status < 0) return fail(ctx, FMC_ENOCONVERGE, "equilibrium Newton iteration did not converge");
    // the correlation-reducing permutation of the whole design, here (it reads
    // back a status, outside any stream capture)
    if (s->correlation == FMC_CORR_RANK && (rc = run_decorrelate(ctx, ws, s->seed, s->N, s->d * s->K, st)))
        return rc;
    if (P.nmt > 0) {
        // constants of the large-system kernel go to the device once, here
        // (outside any stream capture)
        std::vector<float> wc;
        build_wide_consts(s, delta0.data(), P.nmt, P.nd, P.tcn, P.H, wc);
        if ((rc = ensure(ctx, ws.wconst, wc.size() * sizeof(float)))) return rc;
        FMC_CUDA(ctx, cudaMemcpyAsync(ws.wconst.ptr, wc.data(), wc.size() * sizeof(float), cudaMemcpyHostToDevice, st),
                 "copy constants");
        FMC_CUDA(ctx, cudaStreamSynchronize(st), "sync");
        return FMC_OK;
    }
    build_params_bucket(P.nm, P.nd, s, delta0.data(), P.params);
    return FMC_OK;
}

// Time chunk TC of the fused kernels.  A CTA's accumulator holds d x TC FP32
// TMEM columns (512 per SM), and every chunk boundary reloads the CTA's design
// tile through the shared-memory ring (a latency the CTA waits out).  When the
// GPU is the call's alone and the tiles need fewer than four CTAs per SM, each
// CTA may take more columns, so the chunk grows (up to 256 steps) and the
// boundaries become rarer; launches that share the GPU (batches, the server)
// keep 128 columns per CTA.
//
// Samples per CTA: 128 (four warps) when the GPU is shared.  The kernel also
// runs 64-sample CTAs (two warps); they would even out the warps per SM of 2^16
// samples, but their TMEM share forces 16-step chunks and the doubled
// design-tile reloads cost more than the balance gains (38.9 vs 35.1 ms), so the
// automatic shape keeps 128.
//
// With N = 2^16 the 2048 warps of 4-warp CTAs leave 3.37 warps per SM
// sub-partition on average against at most 4 (56 SMs with four CTAs, 96 with
// three), and the launch lasts as long as the 4-warp sub-partitions: a
// quantisation of whole warps that no CTA shape removes.  (A form with one CTA
// of 14 integrating warps and a producer warp per SM, the contraction
// double-buffered in TMEM, measured no faster: two of its four sub-partitions
// still hold four warps.)
struct FusedShape {
    int rows;       // samples per CTA
    int max_ctas;   // resident CTAs per SM allowed
    int TC;         // time chunk
    int64_t ctas;   // grid
};

static FusedShape fused_shape(const fmc_ctx* ctx, const Prepared& P)
{
    const int d = P.s.d, sms = ctx->sms;
    const bool wide = P.nmt > 0;
    const int64_t full = (P.count + TC_M - 1) / TC_M;
    FusedShape f{TC_M, 4, 32, 0};
    if (P.exclusive) {
        const int64_t need = (full + sms - 1) / sms;
        f.max_ctas = wide ? 1 : (need >= 3 ? 4 : (int)(need < 1 ? 1 : need));
    }
    const fmc_launch_rule* rule = find_rule(ctx, &P.s, P.count);
    if (rule && rule->max_ctas > 0 && !wide) f.max_ctas = rule->max_ctas;
    // a CTA's TMEM columns: the largest power of two within its share of the SM's
    // 512 (allocations are powers of two)
    int cols = 512;
    while (cols * f.max_ctas > 512) cols >>= 1;
    // columns a step takes per disturbance: the path value, or the smooth form's
    // forcing at two half steps
    const int per = P.s.forcing == FMC_FORCING_SMOOTH ? 2 : 1;
    while (per * d * 16 > cols && f.max_ctas > 1) {
        f.max_ctas = f.max_ctas > 2 ? 2 : 1;
        cols = 512 / f.max_ctas;
    }
    // the large-system kernel's shared memory leaves room for a ring of 128-step
    // chunks; a chunk's basis rows (TC, or 2 TC for the smooth form) are one MMA's
    // N and one tensor-map box, at most 256
    int TC = (wide || per == 2) ? 128 : 256;
    if (rule && rule->TC > 0 && rule->TC < TC) TC = rule->TC;
    while (TC > 16 && per * d * TC > cols) TC >>= 1;
    if (P.tcn) {
        // the network sum's A_hi, A_lo and D columns come first: the chunk takes
        // the largest multiple of 16 steps that the rest holds
        const int t = ((512 / (4 / P.H) - wide_tc_cols(P.nmt, P.H)) / d) & ~15;
        if (t < TC) TC = t < 16 ? 16 : t;
    }
    f.TC = TC;
    f.ctas = (P.count + f.rows - 1) / f.rows;
    return f;
}

// All device buffers the enqueue of P needs (grows the workspace; may allocate).
// per_tile_partials = false: the fused kernel adds its sums with FP64 atomics
// and needs no partial buffer.
static int reserve(fmc_ctx* ctx, Workspace& ws, const Prepared& P, bool want_traj, bool per_tile_partials)
{
    const int n = P.s.n, d = P.s.d, K = P.s.K, Nt = P.Nt;
    const int64_t count = P.count, Nt1 = (int64_t)Nt + 1;
    const int S = 2 * n;
    int rc;
    const bool em = (P.s.sampling == FMC_SRS_EM);
    if (P.path == FMC_PATH_PLAIN) {
        const int M = d * K;
        // the smooth form takes the forcing at the 2 Nt + 1 half-step times
        const int64_t cols = P.s.forcing == FMC_FORCING_SMOOTH ? 2 * (int64_t)Nt + 1 : (int64_t)Nt;
        if (!em && (rc = ensure(ctx, ws.zeta32, (size_t)count * M * sizeof(float)))) return rc;
        if (!em && (rc = ensure(ctx, ws.phi32, (size_t)K * cols * sizeof(float)))) return rc;
        if ((rc = ensure(ctx, ws.dW, (size_t)count * d * cols * sizeof(float)))) return rc;
        if (!want_traj && (rc = ensure(ctx, ws.traj, (size_t)count * Nt1 * S * sizeof(float)))) return rc;
        return FMC_OK;
    }
    const int split = (P.s.precision == FMC_PREC_BF16X3);
    const int Ks = round_up(K, 8);
    const int Kpad = round_up(K, TC_BK);
    const int64_t ntiles = fused_shape(ctx, P).ctas;
    size_t zbytes = (size_t)count * d * Ks * 2;
    if (!em) {
        if ((rc = ensure(ctx, ws.zeta_hi, zbytes))) return rc;
        if (split && (rc = ensure(ctx, ws.zeta_lo, zbytes))) return rc;
        // the increment basis [Nt][Kpad], or the smooth form's forcing at the half steps
        const size_t brows = P.s.forcing == FMC_FORCING_SMOOTH ? 2 * (size_t)Nt + 1 : (size_t)Nt;
        if ((rc = ensure(ctx, ws.phi_hi, brows * Kpad * 2))) return rc;
        if (split && (rc = ensure(ctx, ws.phi_lo, brows * Kpad * 2))) return rc;
    }
    if (per_tile_partials && (rc = ensure(ctx, ws.part, (size_t)ntiles * Nt1 * 3 * S * sizeof(float)))) return rc;
    return FMC_OK;
}

// Enqueues the path for P on `st` (no allocation, no synchronisation: usable
// under stream capture once reserve() has run).  S1, S2 [Nt+1][2n] receive the
// shifted sums over the block; the shift is at ws.eq + 2n.
// R > 1 (replicates): the block holds R designs of count / R samples each, the
// design of replicate k from seeds[k] in rows k count/R ..; their moment sums go
// to S1 + k (Nt+1) 2n and S2 + k (Nt+1) 2n (per-tile partials; count / R a
// multiple of 128, so that no tile straddles two designs).
static int enqueue(fmc_ctx* ctx, Workspace& ws, const Prepared& P, double* S1, double* S2, float* traj_dev,
                   bool per_tile_partials, cudaStream_t st, double* rrf = nullptr, int R = 1,
                   const uint64_t* seeds = nullptr)
{
    const fmc_scenario* s = &P.s;
    const int n = s->n, d = s->d, K = s->K, Nt = P.Nt;
    const int64_t N = s->N, k0 = P.k0, count = P.count;
    const int64_t Nt1 = (int64_t)Nt + 1;
    const int S = 2 * n;
    const double* eq = (const double*)ws.eq.ptr;
    const double* shift = eq + 2 * n;
    int rc;
    ProfRec* pr;

    const bool em = (s->sampling == FMC_SRS_EM);
    EmSpec ems{em ? 1 : 0, (uint32_t)s->seed, (uint32_t)(s->seed >> 32), k0, (float)std::sqrt(s->dt)};

    if (P.path == FMC_PATH_PLAIN) {
        const int M = d * K;
        float* traj = traj_dev ? traj_dev : (float*)ws.traj.ptr;
        if (em) {
            prof_begin(ctx, PH_LHS, st, &pr);
            FMC_CUDA(ctx, launch_em_increments(s->seed, k0, count, d, Nt, s->dt, (float*)ws.dW.ptr, ctx->sms, st),
                     "increments kernel");
            prof_end(pr, st);
        } else {
            prof_begin(ctx, PH_LHS, st, &pr);
            FMC_CUDA(ctx,
                     s->correlation == FMC_CORR_RANK
                         ? launch_ic_values(s->seed, N, k0, count, M, s->sampling, (const uint32_t*)ws.ic_strata.ptr,
                                            (float*)ws.zeta32.ptr, ctx->sms, st)
                         : launch_lhs_f32(s->seed, N, k0, count, M, s->sampling, (float*)ws.zeta32.ptr, nullptr,
                                          ctx->sms, st),
                     "lhs kernel");
            prof_end(pr, st);
            // the increment basis [K][Nt], or the smooth form's forcing basis [K][2 Nt + 1]
            const bool smooth = (s->forcing == FMC_FORCING_SMOOTH);
            const int cols = smooth ? 2 * Nt + 1 : Nt;
            prof_begin(ctx, PH_BASIS, st, &pr);
            if (smooth)
                FMC_CUDA(ctx, launch_forcing_f32(K, Nt, s->T, s->basis, (float*)ws.phi32.ptr, ctx->sms, st),
                         "forcing basis kernel");
            else
                FMC_CUDA(ctx, launch_basis_f32(K, Nt, s->T, s->basis, (float*)ws.phi32.ptr, ctx->sms, st),
                         "basis kernel");
            prof_end(pr, st);
            prof_begin(ctx, PH_CONTRACT, st, &pr);
            FMC_CUDA(ctx,
                     launch_sgemm_nn(count * d, cols, K, (const float*)ws.zeta32.ptr, (const float*)ws.phi32.ptr,
                                     (float*)ws.dW.ptr, st),
                     "sgemm kernel");
            prof_end(pr, st);
        }
        prof_begin(ctx, PH_INTEGRATE, st, &pr);
        FMC_CUDA(ctx,
                 launch_simulate_plain(P.nm, P.nd, P.params.data(), eq, (const float*)ws.dW.ptr, count, Nt, traj, rrf,
                                       s->forcing == FMC_FORCING_SMOOTH ? 1 : 0, st),
                 "plain integrator");
        prof_end(pr, st);
        prof_begin(ctx, PH_MOMENTS, st, &pr);
        FMC_CUDA(ctx, launch_traj_sums(traj, count, Nt1 * S, shift, S, S1, S2, ctx->sms, st), "moments kernel");
        prof_end(pr, st);
        return FMC_OK;
    }

    // fused path
    const int split = (s->precision == FMC_PREC_BF16X3);
    const int Ks = round_up(K, 8);
    const int Kpad = round_up(K, TC_BK);
    const int nkb = (Ks + TC_BK - 1) / TC_BK;
    const FusedShape shape = fused_shape(ctx, P);
    const int64_t ntiles = shape.ctas;
    const int TC = shape.TC;
    uint32_t tmem_cols = 32;
    const bool smooth = (s->forcing == FMC_FORCING_SMOOTH);
    const int cw = smooth ? 2 * TC : TC;  // TMEM columns (basis rows) per disturbance and chunk
    while (tmem_cols < (uint32_t)(d * cw)) tmem_cols <<= 1;
    CUtensorMap maps[4];
    if (em) {
        // no design and no contraction: the kernels draw the increments
        memset(maps, 0, sizeof maps);
    } else {
        prof_begin(ctx, PH_LHS, st, &pr);
        if (R > 1) {
            const int64_t per = count / R;
            const size_t rb = (size_t)per * d * Ks * 2;  // bytes of one design (BF16 rows of d Ks)
            for (int k = 0; k < R; ++k)
                FMC_CUDA(ctx,
                         launch_lhs_split(seeds[k], per, 0, per, d, K, s->sampling, (char*)ws.zeta_hi.ptr + k * rb,
                                          split ? (char*)ws.zeta_lo.ptr + k * rb : nullptr, ctx->sms, st),
                         "lhs kernel");
        } else {
            FMC_CUDA(ctx,
                     s->correlation == FMC_CORR_RANK
                         ? launch_ic_split(s->seed, N, k0, count, d, K, s->sampling,
                                           (const uint32_t*)ws.ic_strata.ptr, ws.zeta_hi.ptr,
                                           split ? ws.zeta_lo.ptr : nullptr, ctx->sms, st)
                         : launch_lhs_split(s->seed, N, k0, count, d, K, s->sampling, ws.zeta_hi.ptr,
                                            split ? ws.zeta_lo.ptr : nullptr, ctx->sms, st),
                     "lhs kernel");
        }
        prof_end(pr, st);
        prof_begin(ctx, PH_BASIS, st, &pr);
        FMC_CUDA(ctx,
                 smooth ? launch_forcing_split(K, Nt, s->T, s->basis, Kpad, ws.phi_hi.ptr, split ? ws.phi_lo.ptr : nullptr,
                                               ctx->sms, st)
                        : launch_basis_split(K, Nt, s->T, s->basis, Kpad, ws.phi_hi.ptr, split ? ws.phi_lo.ptr : nullptr,
                                             ctx->sms, st),
                 "basis kernel");
        prof_end(pr, st);
        if ((rc = make_contract_maps_at(ctx, maps, ws.zeta_hi.ptr, ws.zeta_lo.ptr, ws.phi_hi.ptr, ws.phi_lo.ptr, count, d,
                                        Ks, smooth ? 2 * Nt + 1 : Nt, Kpad, cw, split, shape.rows)))
            return rc;
    }
    FMC_CUDA(ctx, cudaMemsetAsync((char*)ws.status.ptr + 4, 0, 4, st), "memset");
    if (!per_tile_partials) {
        FMC_CUDA(ctx, cudaMemsetAsync(S1, 0, Nt1 * S * sizeof(double), st), "memset");
        FMC_CUDA(ctx, cudaMemsetAsync(S2, 0, Nt1 * S * sizeof(double), st), "memset");
    }
    prof_begin(ctx, PH_FUSED, st, &pr);
    int occ = 0;
    cudaError_t e;
    if (P.nmt > 0) {
        WideArgs wa{};
        wa.count = count;
        wa.Nt = Nt;
        wa.TC = TC;
        wa.d = d;
        wa.Ks = Ks;
        wa.nkb = nkb;
        wa.split = split;
        wa.n = n;
        wa.tmem_cols = tmem_cols;
        wa.integrator = s->integrator;
        wa.rel = s->has_inf_bus ? 0 : 1;
        wa.omega_s = (float)s->omega_s;
        wa.dt = (float)s->dt;
        for (int q = 0; q < d; ++q) {
            wa.ou_a[q] = (float)(1.0 - s->theta[q] * s->dt);
            wa.ou_s[q] = (float)s->sigma[q];
        }
        wa.consts = (const float*)ws.wconst.ptr;
        wa.part = per_tile_partials ? (float*)ws.part.ptr : nullptr;
        wa.S1 = per_tile_partials ? nullptr : S1;
        wa.S2 = per_tile_partials ? nullptr : S2;
        wa.traj = traj_dev;
        wa.err = (int*)ws.status.ptr + 1;
        wa.em = ems;
        wa.dx = d + (s->event_machine >= 0 ? 1 : 0);
        wa.ev_step = s->event_machine >= 0 ? event_step_of(s) : 0;
        if (s->event_machine >= 0) {
            wa.ou_a[d] = 1.f;
            wa.ou_s[d] = 0.f;
        }
        wa.rrf = rrf;
        build_ito<8>(s, wa.ito);
        if (P.tcn) {
            CUtensorMap maps5[5] = {maps[0], maps[1], maps[2], maps[3], {}};
            if ((rc = make_map_net(ctx, &maps5[4], (const float*)ws.wconst.ptr + wide_net_offset(n, P.nmt, P.nd),
                                   wide_nn(P.nmt, P.H))))
                return rc;
            wa.tmem_cols = tmem_cols = 512 / (4 / P.H);
            e = launch_simulate_wide_tc(P.nmt, P.H, P.nd, P.bus, maps5, wa, st, &occ);
        } else {
            e = launch_simulate_wide(P.nmt, P.nd, maps, wa, st, &occ);
        }
    } else {
        // a launch that has the GPU to itself keeps as many design tiles in L2 as
        // 60 % of it holds: every chunk re-reads each tile, and the whole design
        // may not fit
        L2Keep keep{ws.zeta_hi.ptr, split ? ws.zeta_lo.ptr : nullptr, (int64_t)d * Ks * 2, 0};
        if (!em && P.exclusive && ctx->l2_bytes > 0) {
            const double tile_bytes = (double)shape.rows * keep.row_bytes * (split ? 2 : 1);
            const double t = 0.6 * (double)ctx->l2_bytes / tile_bytes;
            keep.tiles = t >= (double)ntiles ? (int)ntiles : (int)t;
        }
        e = launch_simulate_fused(P.nm, P.nd, P.params.data(), maps, count, Nt, TC, d, Ks, nkb, split, tmem_cols,
                                  shape.rows, shape.max_ctas, eq, per_tile_partials ? (float*)ws.part.ptr : nullptr,
                                  per_tile_partials ? nullptr : S1, per_tile_partials ? nullptr : S2, traj_dev,
                                  (int*)ws.status.ptr + 1, ems, rrf, keep, smooth ? 1 : 0, st, &occ);
    }
    ctx->last_fused_ctas_per_sm = occ;
    if (e == cudaErrorInvalidConfiguration)
        return fail(ctx, FMC_EUNSUPPORTED, "fused kernel: %d CTAs per SM x %u TMEM columns exceeds 512", occ,
                    tmem_cols);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fused simulation kernel");
    prof_end(pr, st);
    if (per_tile_partials) {
        prof_begin(ctx, PH_REDUCE, st, &pr);
        if (R > 1) {
            const int64_t tiles = ntiles / R;
            for (int k = 0; k < R; ++k)
                FMC_CUDA(ctx,
                         launch_fused_sums((const float*)ws.part.ptr + (size_t)k * tiles * Nt1 * 3 * S, (int)tiles,
                                           Nt1, S, count / R, shape.rows, S1 + (size_t)k * Nt1 * S,
                                           S2 + (size_t)k * Nt1 * S, st),
                         "moment sums");
        } else {
            FMC_CUDA(ctx, launch_fused_sums((const float*)ws.part.ptr, (int)ntiles, Nt1, S, count, shape.rows, S1, S2, st),
                     "moment sums");
        }
        prof_end(pr, st);
    }
    return FMC_OK;
}

// Samples k0 .. k0+count-1 of the N-sample design: equilibrium, LHS, KL
// increments, integration and per-time shifted sums S1, S2 [Nt+1][2n] (FP64).
// The shift (FP64 [2n]: delta*, then zeros) is left at ctx->eq + 2n.
static int simulate_core(fmc_ctx* ctx, const fmc_scenario* s, int64_t k0, int64_t count, int32_t path, double* S1,
                         double* S2, float* traj_dev, cudaStream_t st, double* rrf = nullptr)
{
    if (!S1 || !S2) return fail(ctx, FMC_EINVAL, "moment outputs are NULL");
    Prepared P;
    int rc = prepare(ctx, ctx->ws, s, k0, count, path, st, P);
    if (rc) return rc;
    if ((rc = reserve(ctx, ctx->ws, P, traj_dev != nullptr, true))) return rc;
    return enqueue(ctx, ctx->ws, P, S1, S2, traj_dev, true, st, rrf);
}

}  // extern "C"

int fmc::simulate_moments(fmc_ctx* ctx, const fmc_scenario* s, int32_t path, double* mean_dev, double* var_dev,
                          bool per_tile_partials, cudaStream_t st)
{
    if (!ctx) return FMC_EINVAL;
    if (!s || !mean_dev || !var_dev) return fail(ctx, FMC_EINVAL, "NULL scenario or output");
    if (ctx->stream_ordered) ctx->ws_stream = st;
    Prepared P;
    int rc = prepare(ctx, ctx->ws, s, 0, s->N, path, st, P, false);  // requests of the server share the GPU
    if (rc) return rc;
    const bool tiles = per_tile_partials || path == FMC_PATH_PLAIN;
    if ((rc = reserve(ctx, ctx->ws, P, false, tiles))) return rc;
    if ((rc = enqueue(ctx, ctx->ws, P, mean_dev, var_dev, nullptr, tiles, st))) return rc;
    FMC_CUDA(ctx,
             launch_finalize(mean_dev, var_dev, (const double*)ctx->eq.ptr + 2 * s->n, s->N, (int64_t)P.Nt + 1,
                             2 * s->n, mean_dev, var_dev, st),
             "moment finalize");
    return FMC_OK;
}

int fmc::simulate_moments_replicates(fmc_ctx* ctx, const fmc_scenario* s, int32_t path, int R,
                                     const uint64_t* seeds, double* mean_dev, double* var_dev, cudaStream_t st)
{
    if (!ctx) return FMC_EINVAL;
    if (!s || !seeds || !mean_dev || !var_dev || R < 2) return fail(ctx, FMC_EINVAL, "replicates");
    if (path != FMC_PATH_FUSED || s->sampling == FMC_SRS_EM || s->correlation == FMC_CORR_RANK || s->N % TC_M != 0)
        return fail(ctx, FMC_EUNSUPPORTED, "replicates in one launch: fused path, a KL design, N a multiple of 128");
    if (ctx->stream_ordered) ctx->ws_stream = st;
    fmc_scenario sr = *s;
    sr.N = (int64_t)R * s->N;
    Prepared P;
    int rc = prepare(ctx, ctx->ws, &sr, 0, sr.N, path, st, P, false);  // requests of the server share the GPU
    if (rc) return rc;
    if ((rc = reserve(ctx, ctx->ws, P, false, true))) return rc;
    if ((rc = enqueue(ctx, ctx->ws, P, mean_dev, var_dev, nullptr, true, st, nullptr, R, seeds))) return rc;
    const int64_t Nt1 = (int64_t)P.Nt + 1;
    const size_t cols = (size_t)Nt1 * 2 * s->n;
    for (int k = 0; k < R; ++k)
        FMC_CUDA(ctx,
                 launch_finalize(mean_dev + k * cols, var_dev + k * cols, (const double*)ctx->eq.ptr + 2 * s->n, s->N,
                                 Nt1, 2 * s->n, mean_dev + k * cols, var_dev + k * cols, st),
                 "moment finalize");
    return FMC_OK;
}

void fmc::set_stream_ordered(fmc_ctx* ctx, bool on)
{
    if (ctx) ctx->stream_ordered = on;
}

int fmc::release_workspace(fmc_ctx* ctx, cudaStream_t st)
{
    if (!ctx) return FMC_EINVAL;
    // the buffers that scale with the samples or the horizon; the small ones stay
    DevBuf* big[] = {&ctx->ws.zeta_hi, &ctx->ws.zeta_lo, &ctx->ws.phi_hi, &ctx->ws.phi_lo, &ctx->ws.phi32,
                     &ctx->ws.dW,      &ctx->ws.traj,    &ctx->ws.part,   &ctx->ws.zeta32,
                     &ctx->ws.ic,      &ctx->ws.ic_strata};
    for (DevBuf* b : big) {
        if (!b->ptr) continue;
        if (ctx->stream_ordered)
            cudaFreeAsync(b->ptr, st);
        else
            cudaFree(b->ptr);
        ctx->used -= b->bytes;
        b->ptr = nullptr;
        b->bytes = 0;
    }
    return FMC_OK;
}

int fmc::reserve_workspace(fmc_ctx* ctx, const fmc_scenario* s, int32_t path, int64_t count, cudaStream_t st)
{
    if (!ctx || !s) return FMC_EINVAL;
    int Nt = 0;
    int rc = check_scenario(ctx, s, &Nt);
    if (rc) return rc;
    if (ctx->stream_ordered) ctx->ws_stream = st;
    // the sizes simulate_moments will need (a shared GPU: AUTO's kernel, atomics)
    Prepared P;
    P.s = *s;
    P.Nt = Nt;
    P.nm = nm_bucket_for(s->n);
    P.nmt = P.nm < 0 ? wide_nmt_for(s->n) : 0;
    P.nd = nd_bucket_for(s->d + (s->event_machine >= 0 ? 1 : 0));
    P.path = path;
    P.exclusive = false;
    P.k0 = 0;
    P.count = count;
    return reserve(ctx, ctx->ws, P, false, path == FMC_PATH_PLAIN);
}

extern "C" {

int fmc_simulate(fmc_ctx* ctx, const fmc_scenario* s, int32_t path, double* mean_dev, double* var_dev,
                 float* traj_dev, void* stream)
{
    if (!ctx) return FMC_EINVAL;
    if (!s) return fail(ctx, FMC_EINVAL, "scenario is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = simulate_core(ctx, s, 0, s->N, path, mean_dev, var_dev, traj_dev, st);
    if (rc) return rc;
    int Nt = 0;
    steps_of(ctx, s->T, s->dt, &Nt);
    ProfRec* pr;
    prof_begin(ctx, PH_REDUCE, st, &pr);
    FMC_CUDA(ctx,
             launch_finalize(mean_dev, var_dev, (const double*)ctx->eq.ptr + 2 * s->n, s->N, (int64_t)Nt + 1, 2 * s->n,
                             mean_dev, var_dev, st),
             "moment finalize");
    prof_end(pr, st);
    return FMC_OK;
}

int fmc_simulate_rrf(fmc_ctx* ctx, const fmc_scenario* s, int32_t path, double* rrf_dev, double* mean_dev,
                     double* var_dev, void* stream)
{
    if (!ctx) return FMC_EINVAL;
    if (!s || !rrf_dev) return fail(ctx, FMC_EINVAL, "NULL scenario or output");
    if ((mean_dev == nullptr) != (var_dev == nullptr)) return fail(ctx, FMC_EINVAL, "give both moment outputs or none");
    int Nt = 0;
    int rc = check_scenario(ctx, s, &Nt);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cols = (size_t)(Nt + 1) * 2 * s->n;
    // [0] sum RRF, [1] sum RRF^2, [2] zero shift, [3] pad, then moments if the caller gives none
    if ((rc = ensure(ctx, ctx->rrfbuf, sizeof(double) * (4 + (mean_dev ? 0 : 2 * cols))))) return rc;
    double* buf = (double*)ctx->rrfbuf.ptr;
    if (!mean_dev) {
        mean_dev = buf + 4;
        var_dev = buf + 4 + cols;
    }
    FMC_CUDA(ctx, cudaMemsetAsync(buf, 0, 4 * sizeof(double), st), "memset");
    if ((rc = simulate_core(ctx, s, 0, s->N, path, mean_dev, var_dev, nullptr, st, buf))) return rc;
    FMC_CUDA(ctx,
             launch_finalize(mean_dev, var_dev, (const double*)ctx->eq.ptr + 2 * s->n, s->N, (int64_t)Nt + 1, 2 * s->n,
                             mean_dev, var_dev, st),
             "moment finalize");
    FMC_CUDA(ctx, launch_finalize(buf, buf + 1, buf + 2, s->N, 1, 1, rrf_dev, rrf_dev + 1, st), "rrf finalize");
    return FMC_OK;
}

int fmc_simulate_sums(fmc_ctx* ctx, const fmc_scenario* s, int64_t k0, int64_t count, int32_t path, double* S1_dev,
                      double* S2_dev, double* shift_dev, float* traj_dev, void* stream)
{
    if (!ctx) return FMC_EINVAL;
    if (!s) return fail(ctx, FMC_EINVAL, "scenario is NULL");
    if (!shift_dev) return fail(ctx, FMC_EINVAL, "shift output is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = simulate_core(ctx, s, k0, count, path, S1_dev, S2_dev, traj_dev, st);
    if (rc) return rc;
    FMC_CUDA(ctx,
             cudaMemcpyAsync(shift_dev, (const double*)ctx->eq.ptr + 2 * s->n, 2 * s->n * sizeof(double),
                             cudaMemcpyDeviceToDevice, st),
             "copy shift");
    return FMC_OK;
}

int fmc_moments_from_sums(fmc_ctx* ctx, const double* S1_dev, const double* S2_dev, const double* shift_dev, int64_t N,
                          int64_t T1, int32_t S, double* mean_dev, double* var_dev, void* stream)
{
    if (!ctx) return FMC_EINVAL;
    if (N < 1 || T1 < 1 || S < 1) return fail(ctx, FMC_EINVAL, "N, rows and states must be >= 1");
    if (!S1_dev || !S2_dev || !shift_dev || !mean_dev || !var_dev) return fail(ctx, FMC_EINVAL, "NULL buffer");
    FMC_CUDA(ctx, launch_finalize(S1_dev, S2_dev, shift_dev, N, T1, S, mean_dev, var_dev, (cudaStream_t)stream),
             "moment finalize");
    return FMC_OK;
}

// ---- many scenarios ------------------------------------------------------------

struct fmc_batch {
    fmc_ctx* ctx = nullptr;
    std::vector<std::unique_ptr<fmc::OwnedScenario>> owned;  // the batch's own copies of the scenarios
    std::vector<Workspace*> ws;
    std::vector<Prepared> prep;
    std::vector<double*> mean, var;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static void batch_free(fmc_batch* b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaEvent_t e : b->done) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (Workspace* w : b->ws) {
        DevBuf* bufs[] = {&w->zeta_hi, &w->zeta_lo, &w->phi_hi, &w->phi_lo, &w->phi32,  &w->dW,
                          &w->traj,    &w->part,    &w->eq,     &w->scen,   &w->status, &w->zeta32,
                          &w->wconst,  &w->rrf,    &w->ic,     &w->ic_strata};
        for (DevBuf* d : bufs)
            if (d->ptr) {
                cudaFree(d->ptr);
                b->ctx->used -= d->bytes;
            }
        delete w;
    }
    delete b;
}

// Enqueue every scenario: fork from `st` onto the batch's streams, one scenario
// per stream in turn (so that independent scenarios share the GPU), join back.
static int batch_enqueue(fmc_batch* b, cudaStream_t st)
{
    fmc_ctx* ctx = b->ctx;
    FMC_CUDA(ctx, cudaEventRecord(b->fork, st), "event");
    for (cudaStream_t s : b->streams) FMC_CUDA(ctx, cudaStreamWaitEvent(s, b->fork, 0), "wait");
    for (size_t i = 0; i < b->prep.size(); ++i) {
        cudaStream_t s = b->streams[i % b->streams.size()];
        const Prepared& P = b->prep[i];
        Workspace& w = *b->ws[i];
        int rc = enqueue(ctx, w, P, b->mean[i], b->var[i], nullptr, P.path == FMC_PATH_PLAIN, s);
        if (rc) return rc;
        FMC_CUDA(ctx,
                 launch_finalize(b->mean[i], b->var[i], (const double*)w.eq.ptr + 2 * P.s.n, P.s.N, (int64_t)P.Nt + 1,
                                 2 * P.s.n, b->mean[i], b->var[i], s),
                 "moment finalize");
    }
    for (size_t k = 0; k < b->streams.size(); ++k) {
        FMC_CUDA(ctx, cudaEventRecord(b->done[k], b->streams[k]), "event");
        FMC_CUDA(ctx, cudaStreamWaitEvent(st, b->done[k], 0), "wait");
    }
    return FMC_OK;
}

int fmc_batch_create(fmc_ctx* ctx, const fmc_scenario* scen, int32_t n_scen, int32_t path, double* const* mean_dev,
                     double* const* var_dev, int32_t use_graph, fmc_batch** out)
{
    if (!ctx) return FMC_EINVAL;
    if (!out) return fail(ctx, FMC_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_scen < 1 || !scen || !mean_dev || !var_dev) return fail(ctx, FMC_EINVAL, "empty or NULL batch");
    fmc_batch* b = new fmc_batch();
    b->ctx = ctx;
    prof_clear(ctx);
    const bool prof_was = ctx->prof;
    ctx->prof = false;  // no event records inside the batch
    int rc = FMC_OK;
    cudaStream_t st0 = 0;
    for (int i = 0; i < n_scen && rc == FMC_OK; ++i) {
        if (!mean_dev[i] || !var_dev[i]) {
            rc = fail(ctx, FMC_EINVAL, "scenario %d: NULL output", i);
            break;
        }
        Workspace* w = new Workspace();
        b->ws.push_back(w);
        b->prep.emplace_back();
        b->owned.push_back(std::make_unique<fmc::OwnedScenario>(scen[i]));
        const fmc_scenario* si = &b->owned.back()->s;
        rc = prepare(ctx, *w, si, 0, si->N, path, st0, b->prep.back(), false);  // scenarios share the GPU
        if (rc == FMC_OK) rc = reserve(ctx, *w, b->prep.back(), false, path == FMC_PATH_PLAIN);
        b->mean.push_back(mean_dev[i]);
        b->var.push_back(var_dev[i]);
    }
    const int nstreams = n_scen < 16 ? n_scen : 16;
    for (int k = 0; k < nstreams && rc == FMC_OK; ++k) {
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            rc = fail(ctx, FMC_ECUDA, "stream/event creation failed");
        else {
            b->streams.push_back(s);
            b->done.push_back(e);
        }
    }
    if (rc == FMC_OK && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
        rc = fail(ctx, FMC_ECUDA, "event creation failed");
    if (rc == FMC_OK && use_graph) {
        // capture the whole batch once; fmc_batch_launch replays it
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
            rc = fail(ctx, FMC_ECUDA, "stream creation failed");
        } else {
            cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) rc = cuda_fail(ctx, e, "cudaStreamBeginCapture");
            if (rc == FMC_OK) {
                int rc2 = batch_enqueue(b, cap);
                e = cudaStreamEndCapture(cap, &b->graph);
                if (rc2) rc = rc2;
                else if (e != cudaSuccess) rc = cuda_fail(ctx, e, "cudaStreamEndCapture");
            }
            if (rc == FMC_OK) {
                e = cudaGraphInstantiate(&b->exec, b->graph, 0);
                if (e != cudaSuccess) rc = cuda_fail(ctx, e, "cudaGraphInstantiate");
            }
            cudaStreamDestroy(cap);
        }
    }
    ctx->prof = prof_was;
    if (rc != FMC_OK) {
        std::string msg = ctx->err;
        batch_free(b);
        ctx->err = msg;
        return rc;
    }
    *out = b;
    return FMC_OK;
}

int fmc_batch_launch(fmc_batch* b, void* stream)
{
    if (!b) return FMC_EINVAL;
    fmc_ctx* ctx = b->ctx;
    cudaStream_t st = (cudaStream_t)stream;
    if (b->exec) {
        ProfRec* pr;
        prof_begin(ctx, PH_BATCH, st, &pr);
        FMC_CUDA(ctx, cudaGraphLaunch(b->exec, st), "cudaGraphLaunch");
        prof_end(pr, st);
        return FMC_OK;
    }
    const bool prof_was = ctx->prof;
    ctx->prof = false;
    int rc = batch_enqueue(b, st);
    ctx->prof = prof_was;
    return rc;
}

int fmc_batch_destroy(fmc_batch* b)
{
    if (!b) return FMC_EINVAL;
    batch_free(b);
    return FMC_OK;
}

int fmc_simulate_batch(fmc_ctx* ctx, const fmc_scenario* scen, int32_t n_scen, int32_t path, double* const* mean_dev,
                       double* const* var_dev, void* stream)
{
    fmc_batch* b = nullptr;
    int rc = fmc_batch_create(ctx, scen, n_scen, path, mean_dev, var_dev, 0, &b);
    if (rc) return rc;
    rc = fmc_batch_launch(b, stream);
    if (rc == FMC_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        rc = fail(ctx, FMC_ECUDA, "batch failed on the device");
    fmc_batch_destroy(b);
    return rc;
}

int fmc_moments(fmc_ctx* ctx, const float* x_dev, int64_t N, int64_t C, double* mean_dev, double* var_dev, void* stream)
{
    if (!ctx) return FMC_EINVAL;
    if (N < 1 || C < 1) return fail(ctx, FMC_EINVAL, "N = %lld, C = %lld", (long long)N, (long long)C);
    if (!x_dev || !mean_dev || !var_dev) return fail(ctx, FMC_EINVAL, "NULL buffer");
    cudaStream_t st = (cudaStream_t)stream;
    ProfRec* pr;
    prof_begin(ctx, PH_MOMENTS, st, &pr);
    FMC_CUDA(ctx, launch_moments(x_dev, N, C, mean_dev, var_dev, ctx->sms, st), "moments kernel");
    prof_end(pr, st);
    return FMC_OK;
}

}  // extern "C"

// ---- diagnostics -------------------------------------------------------------

int fmc::device_status_on(fmc_ctx* ctx, cudaStream_t st)
{
    if (!ctx) return FMC_EINVAL;
    if (!ctx->status.ptr) return FMC_OK;
    int h[2] = {0, 0};
    FMC_CUDA(ctx, cudaMemcpyAsync(h, ctx->status.ptr, sizeof h, cudaMemcpyDeviceToHost, st), "copy");
    FMC_CUDA(ctx, cudaStreamSynchronize(st), "sync");
    if (h[0] < 0) return fail(ctx, FMC_ENOCONVERGE, "equilibrium Newton iteration did not converge");
    if (h[1] == DEV_TIMEOUT_MMA || h[1] == DEV_TIMEOUT_TMA)
        return fail(ctx, FMC_ETIMEOUT, "a bounded device wait gave up (code %d)", h[1]);
    if (h[1] != 0) return fail(ctx, FMC_ECUDA, "device error %d", h[1]);
    return FMC_OK;
}

extern "C" {

int fmc_device_status(fmc_ctx* ctx, int* eq_iterations, int* kernel_error)
{
    if (!ctx) return FMC_EINVAL;
    int h[2] = {0, 0};
    int hn[2] = {0, 0};
    void* scratch = noalloc_scratch_if_known(ctx);
    if (ctx->status.ptr || scratch) FMC_CUDA(ctx, cudaDeviceSynchronize(), "sync");
    if (ctx->status.ptr) FMC_CUDA(ctx, cudaMemcpy(h, ctx->status.ptr, sizeof h, cudaMemcpyDeviceToHost), "copy");
    // the allocation-free reconstruction keeps its error word in the scratch array
    if (scratch) FMC_CUDA(ctx, cudaMemcpy(hn, scratch, sizeof hn, cudaMemcpyDeviceToHost), "copy");
    if (eq_iterations) *eq_iterations = h[0];
    if (kernel_error) *kernel_error = h[1] != 0 ? h[1] : hn[1];
    if (h[0] < 0) return fail(ctx, FMC_ENOCONVERGE, "equilibrium Newton iteration did not converge");
    if (h[1] == DEV_TIMEOUT_MMA || h[1] == DEV_TIMEOUT_TMA)
        return fail(ctx, FMC_ETIMEOUT, "a bounded device wait gave up (code %d)", h[1]);
    if (h[1] != 0) return fail(ctx, FMC_ECUDA, "device error %d", h[1]);
    if (hn[1] == DEV_TIMEOUT_MMA || hn[1] == DEV_TIMEOUT_TMA)
        return fail(ctx, FMC_ETIMEOUT, "a bounded device wait of the allocation-free reconstruction gave up (code %d)",
                    hn[1]);
    if (hn[1] != 0) return fail(ctx, FMC_ECUDA, "allocation-free reconstruction: device error %d", hn[1]);
    return FMC_OK;
}

int fmc_check_wait_path(fmc_ctx* ctx, int32_t target, int64_t poll_limit, void* stream)
{
    if (!ctx) return FMC_EINVAL;
    if (target != 0 && target != 1) return fail(ctx, FMC_EINVAL, "target %d", target);
    if (poll_limit < 1 || poll_limit > (int64_t)TC_WAIT_LIMIT)
        return fail(ctx, FMC_EINVAL, "poll limit %lld outside 1..%u", (long long)poll_limit, TC_WAIT_LIMIT);
    cudaStream_t st = (cudaStream_t)stream;
    int* word = nullptr;
    int rc;
    if (target == 0) {
        if ((rc = ensure(ctx, ctx->status, 64))) return rc;
        FMC_CUDA(ctx, cudaMemsetAsync(ctx->status.ptr, 0, 64, st), "memset");
        word = (int*)ctx->status.ptr + 1;
    } else {
        int cur = -1;
        FMC_CUDA(ctx, cudaGetDevice(&cur), "cudaGetDevice");
        if (cur != ctx->device)
            return fail(ctx, FMC_EINVAL, "the current device (%d) is not the context's device (%d)", cur, ctx->device);
        unsigned char* base = nullptr;
        if ((rc = noalloc_scratch(ctx, &base))) return rc;
        FMC_CUDA(ctx, cudaMemsetAsync(base, 0, NOALLOC_STATUS_BYTES, st), "memset");
        word = reinterpret_cast<int*>(base) + 1;
    }
    FMC_CUDA(ctx, launch_wait_check(word, (uint32_t)poll_limit, st), "wait check kernel");
    return FMC_OK;
}

int fmc_profile(fmc_ctx* ctx, int32_t enable, int64_t max_records)
{
    if (!ctx) return FMC_EINVAL;
    cudaDeviceSynchronize();
    prof_clear(ctx);
    ctx->prof = enable != 0;
    ctx->prof_cap = max_records > 0 ? (size_t)max_records : 0;
    ctx->recs.reserve(ctx->prof_cap);
    return FMC_OK;
}

int fmc_profile_read(fmc_ctx* ctx, int32_t phase, double* total_ms, int64_t* launches)
{
    if (!ctx) return FMC_EINVAL;
    FMC_CUDA(ctx, cudaDeviceSynchronize(), "sync");
    double tot = 0.0;
    int64_t cnt = 0;
    for (auto& r : ctx->recs) {
        if (r.phase != phase) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            tot += ms;
            ++cnt;
        }
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = cnt;
    return FMC_OK;
}

int fmc_test_sincos(fmc_ctx* ctx, const float* x_dev, int64_t n, float* s_dev, float* c_dev, float* s_ref_dev,
                    float* c_ref_dev, void* stream)
{
    if (!ctx) return FMC_EINVAL;
    if (n < 0 || (n > 0 && (!x_dev || !s_dev || !c_dev || !s_ref_dev || !c_ref_dev)))
        return fail(ctx, FMC_EINVAL, "bad arguments");
    FMC_CUDA(ctx, launch_sincos_probe(x_dev, n, s_dev, c_dev, s_ref_dev, c_ref_dev, (cudaStream_t)stream),
             "sincos probe");
    return FMC_OK;
}

int fmc_set_launch_rules(fmc_ctx* ctx, const fmc_launch_rule* rules, int32_t count)
{
    if (!ctx) return FMC_EINVAL;
    if (count < 0 || (count > 0 && !rules)) return fail(ctx, FMC_EINVAL, "rules");
    for (int32_t k = 0; k < count; ++k) {
        const fmc_launch_rule& r = rules[k];
        const bool tc_ok = r.TC == 0 || (r.TC >= 16 && r.TC <= 256 && (r.TC & (r.TC - 1)) == 0);
        if (r.n_min > r.n_max || r.d_min > r.d_max || r.N_min > r.N_max || r.kernel < FMC_KERNEL_AUTO ||
            r.kernel > FMC_KERNEL_SPLIT_TC || r.max_ctas < 0 || r.max_ctas > 4 || !tc_ok)
            return fail(ctx, FMC_EINVAL, "launch rule %d is malformed", k);
    }
    ctx->rules.assign(rules, rules + count);
    return FMC_OK;
}

int fmc_set_kernel_policy(fmc_ctx* ctx, int32_t policy)
{
    if (!ctx) return FMC_EINVAL;
    if (policy < FMC_KERNEL_AUTO || policy > FMC_KERNEL_SPLIT_TC)
        return fail(ctx, FMC_EINVAL, "kernel policy %d", policy);
    ctx->kernel_policy = policy;
    return FMC_OK;
}

int fmc_last_fused_occupancy(const fmc_ctx* ctx, int* ctas_per_sm)
{
    if (!ctx || !ctas_per_sm) return FMC_EINVAL;
    *ctas_per_sm = ctx->last_fused_ctas_per_sm;
    return FMC_OK;
}

int fmc_diag_net_matrix(const fmc_scenario* scen, int32_t nmt, int32_t H, float* out, int64_t out_floats)
{
    if (!scen || !out || scen->n < 1 || scen->n > FMC_MAX_MACHINES || !scen->G || !scen->B || !scen->E)
        return FMC_EINVAL;
    if ((H != 2 && H != 4) || nmt < 1 || nmt > 16 || scen->n > H * nmt ||
        (scen->has_inf_bus && (scen->n >= H * nmt || !scen->Ginf || !scen->Binf)))
        return FMC_EINVAL;
    const int NN = wide_nn(nmt, H);
    if (out_floats < 2 * (int64_t)NN * NN) return FMC_EINVAL;
    build_wide_net(scen, nmt, H, out);
    return FMC_OK;
}

int fmc_diag_kernel_choice(const fmc_scenario* scen, int32_t path, int32_t policy, int64_t count, int32_t* out)
{
    if (!scen || !out || scen->n < 1 || scen->n > FMC_MAX_MACHINES || scen->d < 1 || scen->d > 8 || count < 1 ||
        (path != FMC_PATH_FUSED && path != FMC_PATH_PLAIN) || policy < FMC_KERNEL_AUTO ||
        policy > FMC_KERNEL_SPLIT_TC)
        return FMC_EINVAL;
    KernelChoice C;
    const int rc = choose_kernel(nullptr, nullptr, scen, count, path, policy, C);
    if (rc) return rc;
    out[0] = C.nmt == 0 ? FMC_KERNEL_PER_SAMPLE : (C.tcn ? FMC_KERNEL_SPLIT_TC : FMC_KERNEL_SPLIT);
    out[1] = C.nmt;
    out[2] = C.H;
    out[3] = C.nd;
    out[4] = C.bus ? 1 : 0;
    return FMC_OK;
}

}  // extern "C"
