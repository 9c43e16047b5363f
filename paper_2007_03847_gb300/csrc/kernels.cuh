// Host-side launchers of the fastmc kernels (one translation unit each).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fmc {

cudaError_t launch_lhs_f32(uint64_t seed, int64_t N, int64_t k0, int64_t count, int M, int mode, float* zeta,
                           uint32_t* strata, int sms, cudaStream_t st);
cudaError_t launch_lhs_split(uint64_t seed, int64_t N, int64_t k0, int64_t count, int d, int K, int mode, void* hi,
                             void* lo, int sms, cudaStream_t st);
cudaError_t launch_basis_f32(int K, int Nt, double T, float* phi, int sms, cudaStream_t st);
cudaError_t launch_basis_split(int K, int Nt, double T, int Kpad, void* hi, void* lo, int sms, cudaStream_t st);
cudaError_t launch_sgemm_nn(int64_t R, int Ncols, int K, const float* A, const float* B, float* C, cudaStream_t st);
cudaError_t launch_contract_tc(const CUtensorMap* maps, int64_t count, int d, int Ks, int nkb, int Nt, int TN,
                               int split, float* dW, int* err, cudaStream_t st);
cudaError_t launch_split_rows(const float* z, int64_t count, int d, int K, int Ks, void* hi, void* lo, cudaStream_t st);
cudaError_t launch_equilibrium(int n, int has_inf, double Vinf, const double* G, const double* B, const double* Ginf,
                               const double* Binf, const double* E, const double* Pm, double* out, int* status,
                               cudaStream_t st);
cudaError_t launch_simulate_plain(int nm_bucket, int nd_bucket, const void* params, const double* eq, const float* dW,
                                  int64_t count, int Nt, float* traj, cudaStream_t st);
int fused_smem_bytes(int nm_bucket, int TC, int split, int max_ctas_per_sm);
cudaError_t launch_simulate_fused(int nm_bucket, int nd_bucket, const void* params, const CUtensorMap* maps,
                                  int64_t count, int Nt, int TC, int d, int Ks, int nkb, int split, uint32_t tmem_cols,
                                  const double* eq, float* part, double* S1, double* S2, float* traj, int* err,
                                  cudaStream_t st, int* max_ctas_per_sm);
cudaError_t launch_moments(const float* x, int64_t N, int64_t C, double* mean, double* var, int sms, cudaStream_t st);
cudaError_t launch_traj_sums(const float* x, int64_t N, int64_t C, const double* shift, int S, double* S1, double* S2,
                             int sms, cudaStream_t st);
cudaError_t launch_fused_sums(const float* part, int nblk, int64_t Nt1, int S, double* S1, double* S2,
                              cudaStream_t st);
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
};

__host__ __device__ constexpr int wide_nmtp(int nmt) { return (nmt + 3) & ~3; }

// Constant block of the wide kernel (floats):
//   GE [n][4][NMTP], BE [n][4][NMTP]: entry (j, h, k) = E_i E_j G_ij (resp. B_ij)
//     for machine i = h + 4k, zero on the diagonal and for padded i;
//   then seven rows of 4 NMT per machine: cos D*, sin D*, u*, v*, delta*, 1/(2H), D;
//   then the injection map, d rows of 4 NMT.
__host__ __device__ inline int wide_const_floats(int n, int nmt, int d)
{
    return 2 * n * 4 * wide_nmtp(nmt) + (7 + d) * 4 * nmt;
}

int wide_nmt_for(int n);
cudaError_t launch_simulate_wide(int nmt, int nd, const CUtensorMap* maps, const WideArgs& a, cudaStream_t st,
                                 int* max_ctas_per_sm);

cudaError_t launch_sincos_probe(const float* x, int64_t n, float* s_cw, float* c_cw, float* s_ref, float* c_ref,
                                cudaStream_t st);

}  // namespace fmc
