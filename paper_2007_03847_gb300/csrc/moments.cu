// Algorithm 1 step 4: expectation and unbiased variance over the samples.
//
// Values are shifted by a reference c (row 0 of the data, or the undisturbed
// equilibrium for the fused simulation).  Over short runs of rows the FP32 sum
// about the run's first value and the squared deviations from the run's own mean
// are formed (two passes), and the runs are combined in FP64:
//   mean = c + S1/N,  var = (S2 - S1^2/N) / (N - 1),
//   S1 = sum (x - c),  S2 = sum_runs (M2_run + S1_run^2 / n_run) = sum (x - c)^2,
//   S1_run = n_run (x_first - c) + sum (x - x_first) (formed in FP64).
// The FP32 work only ever sums deviations from one of the run's own values and
// squares deviations from a run mean, so the variance keeps FP32 accuracy
// relative to the spread even when the values drift far from c (a common-mode
// response); the FP64 combine carries the rest.
#include "fmc_common.cuh"
#include "kernels.cuh"

namespace fmc {

constexpr int MOM_THREADS = 256;
constexpr int MOM_RUN = 32;  // rows summed in FP32 before moving into FP64

// grid.x: column blocks; grid.y: row slabs of `rows_per_slab` rows.  The shift
// of column c is x[0][c] (shift == nullptr) or (float)shift[c % S].
__global__ void __launch_bounds__(MOM_THREADS) moments_partial_kernel(const float* __restrict__ x, int64_t N, int64_t C,
                                                                      int64_t rows_per_slab, const double* __restrict__ shift_s,
                                                                      int S, double* __restrict__ S1,
                                                                      double* __restrict__ S2)
{
    int64_t c = (int64_t)blockIdx.x * MOM_THREADS + threadIdx.x;
    if (c >= C) return;
    int64_t r0 = (int64_t)blockIdx.y * rows_per_slab;
    int64_t r1 = r0 + rows_per_slab;
    if (r1 > N) r1 = N;
    const float shift = shift_s ? (float)shift_s[c % S] : x[c];
    double s1 = 0.0, s2 = 0.0;
    for (int64_t r = r0; r < r1; r += MOM_RUN) {
        int64_t re = r + MOM_RUN < r1 ? r + MOM_RUN : r1;
        // about the run's first value (one of the values: the FP32 sums stay on
        // the scale of the spread), carried into FP64 separately
        const float ref = x[r * C + c];
        float a1 = 0.f;
        for (int64_t q = r; q < re; ++q) a1 += x[q * C + c] - ref;
        const float mu = a1 / (float)(re - r);
        float m2 = 0.f;
        for (int64_t q = r; q < re; ++q) {
            const float dv = (x[q * C + c] - ref) - mu;
            m2 = fmaf(dv, dv, m2);
        }
        const double nr = (double)(re - r);
        const double rs1 = fma(nr, (double)ref - (double)shift, (double)a1);  // the run's sum about the shift
        s1 += rs1;
        s2 += (double)m2 + rs1 * rs1 / nr;
    }
    atomicAdd(&S1[c], s1);
    atomicAdd(&S2[c], s2);
}

// In place: mean <- shift + S1/N, var <- (S2 - S1^2/N)/(N-1).
__global__ void moments_finalize_kernel(const float* __restrict__ x, int64_t N, int64_t C, double* __restrict__ mean,
                                        double* __restrict__ var)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    double s1 = mean[c], s2 = var[c];
    double n = (double)N;
    mean[c] = (double)x[c] + s1 / n;
    var[c] = (N > 1) ? (s2 - s1 * s1 / n) / (n - 1.0) : __longlong_as_double(0x7ff8000000000000LL);
}

static cudaError_t launch_partial(const float* x, int64_t N, int64_t C, const double* shift, int S, double* S1,
                                  double* S2, int sms, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(S1, 0, sizeof(double) * C, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(S2, 0, sizeof(double) * C, st);
    if (e != cudaSuccess) return e;
    int64_t gx = (C + MOM_THREADS - 1) / MOM_THREADS;
    // enough slabs to fill the GPU a few times over, each at least a few runs long
    int64_t want_blocks = (int64_t)sms * 8;
    int64_t slabs = (want_blocks + gx - 1) / gx;
    int64_t max_slabs = (N + 4 * MOM_RUN - 1) / (4 * MOM_RUN);
    if (slabs > max_slabs) slabs = max_slabs;
    if (slabs < 1) slabs = 1;
    if (slabs > 65535) slabs = 65535;
    int64_t rows = (N + slabs - 1) / slabs;
    rows = (rows + MOM_RUN - 1) / MOM_RUN * MOM_RUN;
    slabs = (N + rows - 1) / rows;
    if (gx > 2147483647LL) return cudaErrorInvalidValue;
    dim3 grid((unsigned)gx, (unsigned)slabs);
    moments_partial_kernel<<<grid, MOM_THREADS, 0, st>>>(x, N, C, rows, shift, S, S1, S2);
    return cudaGetLastError();
}

cudaError_t launch_moments(const float* x, int64_t N, int64_t C, double* mean, double* var, int sms, cudaStream_t st)
{
    cudaError_t e = launch_partial(x, N, C, nullptr, 1, mean, var, sms, st);
    if (e != cudaSuccess) return e;
    moments_finalize_kernel<<<(unsigned)((C + 255) / 256), 256, 0, st>>>(x, N, C, mean, var);
    return cudaGetLastError();
}

// Shifted sums of trajectories x [N][Nt1*S] with the per-state shift[S].
cudaError_t launch_traj_sums(const float* x, int64_t N, int64_t C, const double* shift, int S, double* S1, double* S2,
                             int sms, cudaStream_t st)
{
    return launch_partial(x, N, C, shift, S, S1, S2, sms, st);
}

// Fused-simulation partials: part [nblk][Nt1][3][S] floats holding, per block of
// `rows` samples (the last block count - (nblk-1) rows), grid time t and state j,
// a reference value c (one of the block's samples), the block's sum about it
// dv = sum (x - c) and its squared deviations from its own mean m2 (the x are
// deviations from the shift).  Combined into the sums about the shift,
//   S1 = sum_b (n_b c_b + dv_b),  S2 = sum_b (m2_b + (n_b c_b + dv_b)^2 / n_b);
// out: S1, S2 [Nt1][S].
//
// FP64 throughput is a small fraction of FP32 here, so the full blocks are first
// merged in FP32 in groups of FS_G (equal block sizes n) about the group's first
// reference c_g: delta_b = n (c_b - c_g) + dv_b is the block's sum about c_g, on
// the scale of the spread; d_g = sum delta_b (compensated two-sum) and
// m2_g = sum m2_b + (1/n) sum (delta_b - d_g / G)^2 (parallel-variance combine).
// Each group then enters FP64 once: s1_g = G n c_g + d_g, S1 += s1_g,
// S2 += m2_g + s1_g^2 / (G n).  The partial last block enters FP64 on its own.
// One thread per (t, j); a CTA owns 32 consecutive pairs, its 8 warps stride
// over the groups (warp g takes groups g, g+8, ...), and the 8 partial sums are
// added in warp order, so the result does not depend on scheduling.
constexpr int FS_COLS = 32, FS_GROUPS = 8, FS_G = 8;

__global__ void __launch_bounds__(FS_COLS * FS_GROUPS) fused_sums_kernel(const float* __restrict__ part, int nblk,
                                                                         int64_t Nt1, int S, int64_t count, int rows,
                                                                         double* __restrict__ S1o,
                                                                         double* __restrict__ S2o)
{
    __shared__ double red1[FS_GROUPS][FS_COLS], red2[FS_GROUPS][FS_COLS];
    const int cx = threadIdx.x % FS_COLS, g = threadIdx.x / FS_COLS;
    const int64_t total = Nt1 * S;        // (t, j) pairs
    const int64_t blk = Nt1 * 3 * S;      // floats per block
    const int64_t q = (int64_t)blockIdx.x * FS_COLS + cx;
    double a1 = 0.0, a2 = 0.0;
    if (q < total) {
        const int64_t t = q / S;
        const int j = (int)(q - t * S);
        const float* p = part + t * 3 * S + j;  // c at p[0], dv at p[S], m2 at p[2 S] of block 0
        const int64_t last_n = count - (int64_t)(nblk - 1) * rows;
        const int nfull = last_n == rows ? nblk : nblk - 1;  // blocks of `rows` samples
        const float fn = (float)rows, inv_n = 1.f / (float)rows;
        for (int g0 = g * FS_G; g0 < nfull; g0 += FS_GROUPS * FS_G) {
            const int gc = nfull - g0 < FS_G ? nfull - g0 : FS_G;
            const float cg = p[(int64_t)g0 * blk];
            float dl[FS_G], hi = 0.f, lo = 0.f, mt = 0.f;
#pragma unroll
            for (int k = 0; k < FS_G; ++k) {
                dl[k] = 0.f;
                if (k < gc) {
                    const float* pb = p + (int64_t)(g0 + k) * blk;
                    dl[k] = fmaf(fn, pb[0] - cg, pb[S]);
                    mt += pb[2 * S];
                    // two-sum: hi + lo carries the exact sum of the dl
                    const float tt = hi + dl[k];
                    const float z = tt - hi;
                    lo += (hi - (tt - z)) + (dl[k] - z);
                    hi = tt;
                }
            }
            const float mean = (hi + lo) / (float)gc;
            float dd = 0.f;
#pragma unroll
            for (int k = 0; k < FS_G; ++k)
                if (k < gc) {
                    const float dv = dl[k] - mean;
                    dd = fmaf(dv, dv, dd);
                }
            const double ng = (double)gc * (double)rows;
            const double s1 = fma(ng, (double)cg, (double)hi) + (double)lo;
            a1 += s1;
            a2 += (double)fmaf(dd, inv_n, mt) + s1 * s1 / ng;
        }
        // the partial last block, by the warp whose turn it would be
        if (nfull < nblk && g == (nfull / FS_G) % FS_GROUPS) {
            const float* pb = p + (int64_t)(nblk - 1) * blk;
            const double s1 = fma((double)last_n, (double)pb[0], (double)pb[S]);
            a1 += s1;
            a2 += (double)pb[2 * S] + s1 * s1 / (double)last_n;
        }
    }
    red1[g][cx] = a1;
    red2[g][cx] = a2;
    __syncthreads();
    if (g == 0 && q < total) {
        double t1 = 0.0, t2 = 0.0;
#pragma unroll
        for (int k = 0; k < FS_GROUPS; ++k) {
            t1 += red1[k][cx];
            t2 += red2[k][cx];
        }
        S1o[q] = t1;
        S2o[q] = t2;
    }
}

cudaError_t launch_fused_sums(const float* part, int nblk, int64_t Nt1, int S, int64_t count, int rows, double* S1,
                              double* S2, cudaStream_t st)
{
    const int64_t total = Nt1 * S;
    fused_sums_kernel<<<(unsigned)((total + FS_COLS - 1) / FS_COLS), FS_COLS * FS_GROUPS, 0, st>>>(
        part, nblk, Nt1, S, count, rows, S1, S2);
    return cudaGetLastError();
}

// mean = shift + S1/N, var = (S2 - S1^2/N)/(N-1) with the FP32 rounding of the
// per-state shift (the value the kernels subtracted); NaN variance for N = 1.
// May run in place (mean == S1, var == S2).
__global__ void finalize_kernel(const double* S1, const double* S2, const double* __restrict__ shift, int64_t N,
                                int64_t Nt1, int S, double* mean, double* var)
{
    int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= Nt1 * S) return;
    const int s = (int)(col % S);
    const double s1 = S1[col], s2 = S2[col];
    const double nn = (double)N;
    mean[col] = (double)(float)shift[s] + s1 / nn;
    var[col] = (N > 1) ? (s2 - s1 * s1 / nn) / (nn - 1.0) : __longlong_as_double(0x7ff8000000000000LL);
}

cudaError_t launch_finalize(const double* S1, const double* S2, const double* shift, int64_t N, int64_t Nt1, int S,
                            double* mean, double* var, cudaStream_t st)
{
    int64_t cols = Nt1 * S;
    finalize_kernel<<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(S1, S2, shift, N, Nt1, S, mean, var);
    return cudaGetLastError();
}

}  // namespace fmc
