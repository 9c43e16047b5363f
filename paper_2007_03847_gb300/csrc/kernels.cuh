// Host-side launchers of the fastmc kernels (one translation unit each).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fmc {

// General Ito disturbances (fmc_ito) as the kernels see them: in the deviation
// y = xi - x0, mu(y) = c0 + c1 y + c2 y^2; sigma(y) = e0 + e1 y + e2 y^2 (kind
// POLY) or sqrt(max(0, e0 + e1 y + e2 y^2 + e3 |y - ap|)) (kind SQRT); strat = 1:
// subtract sigma sigma'/2 (KL paths).  kind OU: the ou_a / ou_s pair.
template <int ND>
struct ItoParams {
    int on;      // any disturbance not OU
    float strat;
    int kind[ND];
    float c0[ND], c1[ND], c2[ND];
    float e0[ND], e1[ND], e2[ND], e3[ND], ap[ND];
};

// The per-step-normal Monte Carlo (FMC_SRS_EM): increments drawn in the
// simulation kernels instead of read from the KL contraction.
struct EmSpec {
    int on;
    uint32_t key0, key1;  // Philox key (the scenario's seed)
    int64_t k0;           // design index of the launch's first sample
    float sqdt;           // sqrt(dt)
};


cudaError_t launch_lhs_f32(uint64_t seed, int64_t N, int64_t k0, int64_t count, int M, int mode, float* zeta,
                           uint32_t* strata, int sms, cudaStream_t st);
cudaError_t launch_lhs_split(uint64_t seed, int64_t N, int64_t k0, int64_t count, int d, int K, int mode, void* hi,
                             void* lo, int sms, cudaStream_t st);
cudaError_t launch_em_increments(uint64_t seed, int64_t k0, int64_t count, int d, int Nt, double dt, float* dW,
                                 int sms, cudaStream_t st);
cudaError_t launch_basis_f32(int K, int Nt, double T, int basis, float* phi, int sms, cudaStream_t st);
// the smooth form's forcing basis mdot [K][2 Nt + 1] (half-step times), FP32
cudaError_t launch_forcing_f32(int K, int Nt, double T, int basis, float* mdot, int sms, cudaStream_t st);
cudaError_t launch_basis_split(int K, int Nt, double T, int basis, int Kpad, void* hi, void* lo, int sms,
                               cudaStream_t st);
// the smooth form's forcing basis in split BF16, time-major [2 Nt + 1][Kpad]
cudaError_t launch_forcing_split(int K, int Nt, double T, int basis, int Kpad, void* hi, void* lo, int sms,
                                 cudaStream_t st);
cudaError_t launch_sgemm_nn(int64_t R, int Ncols, int K, const float* A, const float* B, float* C, cudaStream_t st);
cudaError_t launch_contract_tc(const CUtensorMap* maps, int64_t count, int d, int Ks, int nkb, int Nt, int TN,
                               int split, float* dW, int* err, cudaStream_t st);
cudaError_t launch_split_rows(const float* z, int64_t count, int d, int K, int Ks, void* hi, void* lo, cudaStream_t st);
cudaError_t launch_equilibrium(int n, int has_inf, double Vinf, const double* G, const double* B, const double* Ginf,
                               const double* Binf, const double* E, const double* Pm, double* out, int* status,
                               cudaStream_t st);
// rrf (nullable): [2] FP64 sums of the response function and its square
// dW: increments [count][d][Nt]; smooth: the forcing [count][d][2 Nt + 1] instead
cudaError_t launch_simulate_plain(int nm_bucket, int nd_bucket, const void* params, const double* eq, const float* dW,
                                  int64_t count, int Nt, float* traj, double* rrf, int smooth, cudaStream_t st);
int fused_smem_bytes(int nm_bucket, int TC, int split, int max_ctas_per_sm, int rows);
// L2 residency of the design rows [count][row_bytes] (BF16 hi and lo): the first
// `tiles` tiles of a fused launch load theirs with evict_last, the rest with
// evict_first; tiles 0: no hint
struct L2Keep {
    const void* hi;
    const void* lo;
    int64_t row_bytes;
    int tiles;
};
// rows: samples per CTA, 128 (four warps) or 64 (two warps); max_ctas: resident
// CTAs per SM allowed (further limited by the TMEM columns)
cudaError_t launch_simulate_fused(int nm_bucket, int nd_bucket, const void* params, const CUtensorMap* maps,
                                  int64_t count, int Nt, int TC, int d, int Ks, int nkb, int split, uint32_t tmem_cols,
                                  int rows, int max_ctas, const double* eq, float* part, double* S1, double* S2,
                                  float* traj, int* err, const EmSpec& em, double* rrf, const L2Keep& keep,
                                  int smooth, cudaStream_t st, int* max_ctas_per_sm);
cudaError_t launch_moments(const float* x, int64_t N, int64_t C, double* mean, double* var, int sms, cudaStream_t st);
cudaError_t launch_traj_sums(const float* x, int64_t N, int64_t C, const double* shift, int S, double* S1, double* S2,
                             int sms, cudaStream_t st);
cudaError_t launch_fused_sums(const float* part, int nblk, int64_t Nt1, int S, int64_t count, int rows, double* S1,
                              double* S2, cudaStream_t st);
cudaError_t launch_finalize(const double* S1, const double* S2, const double* shift, int64_t N, int64_t Nt1, int S,
                            double* mean, double* var, cudaStream_t st);

// Fused kernel with four warps per sample group: 17..52 machines, or few
// samples of any system.  Machine slots per thread NMT in {1, 2, 3, 4, 5, 7,
// 10, 13}: n <= 4 NMT.
struct WideArgs {
    int64_t count;
    int Nt, TC, d, Ks, nkb, split, n;
    int ns;  // ring stages (set by the launcher)
    uint32_t tmem_cols;
    int integrator, rel;
    float omega_s, dt;
    float ou_a[8], ou_s[8];
    const float* consts;  // device copy of the constant block (wide_const_floats floats)
    float* part;          // [tiles][Nt+1][4n], or nullptr: add into S1, S2 with FP64 atomics
    double* S1;           // [Nt+1][2n] when part == nullptr
    double* S2;
    float* traj;          // [count][Nt+1][2n] or nullptr
    int* err;
    EmSpec em;
    int dx;               // disturbance slots in use: d, or d + 1 with the event slot (index d)
    int ev_step;          // grid step of the event (see SwingParams)
    double* rrf;          // [2]: sums of the response function and its square, or nullptr
    ItoParams<8> ito;     // general disturbances (ito.on == 0: all OU)
};

__host__ __device__ constexpr int wide_nmtp(int nmt) { return (nmt + 3) & ~3; }

#ifndef FMC_PACKED_FP32
#define FMC_PACKED_FP32 1
#endif

// Whether the wide kernel of nmt machine slots sums the network in packed FP32
// (where it measured faster: 7 and 10 slots; the odd pair of 5 and 13 slots and
// the second pass of 13 cost more than they save).
__host__ __device__ constexpr bool wide_packed(int nmt) { return FMC_PACKED_FP32 && (nmt == 7 || nmt == 10); }

// Constant block of the wide kernel (floats):
//   [n][4][2][NMTP]: for (j, h) the row GE (k) = E_i E_j G_ij, then the row BE (k) =
//     E_i E_j B_ij (stored negated when wide_packed), machine i = h + 4k, zero on the
//     diagonal and for padded i;
//   then eight rows of 4 NMT per machine: cos D*, sin D*, u*, v*, delta*, 1/(2H), D,
//   H / sum H (centre-of-inertia weight);
//   then the injection map, nd rows of 4 NMT (nd: the kernel's disturbance-slot
//   bucket; the event slot's row at index d, the rows past the slots in use zero).
__host__ __device__ inline int wide_const_floats(int n, int nmt, int nd)
{
    return 2 * n * 4 * wide_nmtp(nmt) + (8 + nd) * 4 * nmt;
}

int wide_nmt_for(int n);
cudaError_t launch_simulate_wide(int nmt, int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st,
                                 int* max_ctas_per_sm);

// Section IV-B step 2, the correlation-reducing permutation (rank method of
// Iman and Conover): working buffers of launch_ic_strata for N samples and M
// dimensions (a: N doubles; mom: 2 doubles; R, Rs: N*M floats; G: M*M doubles;
// A, B: M*M floats; vals, vals_out: N*M uint32; off: M+1 ints; ok: 1 int, 1 if
// the score correlation was positive definite; sort_tmp: sort_bytes bytes)
struct IcWork {
    double* a;
    double* mom;
    float* R;
    float* Rs;
    double* G;
    float* A;
    float* B;
    uint32_t* vals;
    uint32_t* vals_out;
    int* off;
    int* ok;
    void* sort_tmp;
    size_t sort_bytes;
};
size_t ic_sort_bytes(int64_t N, int M);
// strata [M][N] of the decorrelated design (M <= 4096, N*M < 2^31)
cudaError_t launch_ic_strata(uint64_t seed, int64_t N, int M, const IcWork& w, uint32_t* strata, int sms,
                             cudaStream_t st);
// design values of rows k0..k0+count-1 from strata [M][N]: zeta [count][M] FP32,
// or the split-BF16 layout [count][d][round_up(K, 8)]
cudaError_t launch_ic_values(uint64_t seed, int64_t N, int64_t k0, int64_t count, int M, int mode,
                             const uint32_t* strata, float* zeta, int sms, cudaStream_t st);
cudaError_t launch_ic_split(uint64_t seed, int64_t N, int64_t k0, int64_t count, int d, int K, int mode,
                            const uint32_t* strata, void* hi, void* lo, int sms, cudaStream_t st);

// The Appendix's identification: the objective L' of a record xi [n] (FP64)
// for the coefficients q (kind 1: sigma polynomial; kind 2: sigma^2
// polynomial) into out [43] = (L', gradient [6], Hessian [6][6]); *bad = 1 if
// some D_j <= 0.  derivs 0: L' only.
struct ItoQ {
    double c[6];
};
cudaError_t launch_ito_objective(int kind, const double* q, const double* xi, int64_t n, double h, int derivs,
                                 double* out, int* bad, int sms, cudaStream_t st);
// step [6] = -(H + lambda I)^-1 g from out's gradient and Hessian; *ok = 0 if
// the shifted Hessian is not positive definite
cudaError_t launch_ito_newton_step(const double* gH, double lambda, double* step, int* ok, cudaStream_t st);

// one CTA whose bounded mbarrier wait runs out; records DEV_TIMEOUT_MMA in *err
cudaError_t launch_wait_check(int* err, uint32_t limit, cudaStream_t st);

cudaError_t launch_sincos_probe(const float* x, int64_t n, float* s_cw, float* c_cw, float* s_ref, float* c_ref,
                                cudaStream_t st);

}  // namespace fmc
