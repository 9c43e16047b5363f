// Algorithm 1 step 4: expectation and unbiased variance over the samples.
//
// Values are shifted by a reference c (row 0 of the data, or the undisturbed
// equilibrium for the fused simulation).  Over short runs of rows the FP32 sum
// and the squared deviations from the run's own mean are formed (two passes),
// and the runs are combined in FP64:
//   mean = c + S1/N,  var = (S2 - S1^2/N) / (N - 1),
//   S1 = sum (x - c),  S2 = sum_runs (M2_run + S1_run^2 / n_run) = sum (x - c)^2.
// The FP32 work only ever squares deviations from a run mean, so the variance
// keeps FP32 accuracy relative to the spread even when the values drift far from
// c (a common-mode response); the FP64 combine carries the rest.
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
        float a1 = 0.f;
        for (int64_t q = r; q < re; ++q) a1 += x[q * C + c] - shift;
        const float mu = a1 / (float)(re - r);
        float m2 = 0.f;
        for (int64_t q = r; q < re; ++q) {
            const float dv = (x[q * C + c] - shift) - mu;
            m2 = fmaf(dv, dv, m2);
        }
        s1 += (double)a1;
        s2 += (double)m2 + (double)a1 * (double)a1 / (double)(re - r);
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

// Fused-simulation partials: part [nblk][Nt1][2*S] floats holding, per block of
// `rows` samples (the last block count - (nblk-1) rows) and per grid time, the
// FP32 sum of the shifted values (states 0..S-1) and their squared deviations
// from the block's own mean (states 0..S-1).  Combined into the sums about the
// shift, S1 = sum_b s1_b and S2 = sum_b (m2_b + s1_b^2 / n_b); out: S1, S2 [Nt1][S].
//
// FP64 throughput is a small fraction of FP32 here, so the full blocks are first
// merged in FP32 in groups of FS_G: the sums s1_g = sum s1_b with a compensated
// (two-sum) addition, the squared deviations by the parallel-variance combine
// (equal block sizes n), m2_g = sum m2_b + (1/n) sum (s1_b - s1_g/G)^2, which stays
// on the scale of the spread (FP32-relative accuracy); each group then enters
// FP64 once, as s1_g and m2_g + s1_g^2 / (G n).  The partial last block enters
// FP64 on its own.  A CTA owns 32 consecutive entries q of a part row; its 8 warps
// stride over the groups (warp g takes groups g, g+8, ...), and the 8 partial sums
// are added in warp order, so the result does not depend on scheduling.
constexpr int FS_COLS = 32, FS_GROUPS = 8, FS_G = 8;

__global__ void __launch_bounds__(FS_COLS * FS_GROUPS) fused_sums_kernel(const float* __restrict__ part, int nblk,
                                                                         int64_t Nt1, int S, int64_t count, int rows,
                                                                         double* __restrict__ S1o,
                                                                         double* __restrict__ S2o)
{
    __shared__ double red[FS_GROUPS][FS_COLS];
    const int cx = threadIdx.x % FS_COLS, g = threadIdx.x / FS_COLS;
    const int64_t row = 2 * (int64_t)S;
    const int64_t total = Nt1 * row;
    const int64_t q = (int64_t)blockIdx.x * FS_COLS + cx;
    double acc = 0.0;
    if (q < total) {
        const float* p = part + q;
        const bool second = (q % row) >= S;  // squared deviations (s1 of the same state S entries before)
        const int64_t last_n = count - (int64_t)(nblk - 1) * rows;
        const int nfull = last_n == rows ? nblk : nblk - 1;  // blocks of `rows` samples
        const float inv_n = 1.f / (float)rows;
        const double inv_gn = 1.0 / ((double)FS_G * (double)rows);
        for (int g0 = g * FS_G; g0 < nfull; g0 += FS_GROUPS * FS_G) {
            const int gc = nfull - g0 < FS_G ? nfull - g0 : FS_G;
            float sv[FS_G], st = 0.f, mt = 0.f;
#pragma unroll
            for (int k = 0; k < FS_G; ++k) {
                sv[k] = 0.f;
                if (k < gc) {
                    const float* pb = p + (int64_t)(g0 + k) * total;
                    if (second) {
                        sv[k] = pb[-S];
                        mt += pb[0];
                    } else {
                        sv[k] = pb[0];
                    }
                    st += sv[k];
                }
            }
            if (!second) {
                // the group's sum, compensated (Knuth's two-sum: the rounding error
                // of every addition is carried), so that it enters FP64 as exactly as
                // the blocks would one by one
                float hi = 0.f, lo = 0.f;
#pragma unroll
                for (int k = 0; k < FS_G; ++k) {
                    const float t = hi + sv[k];
                    const float z = t - hi;
                    lo += (hi - (t - z)) + (sv[k] - z);
                    hi = t;
                }
                acc += (double)hi + (double)lo;
            } else {
                const float sb = gc == FS_G ? st * (1.f / FS_G) : st / (float)gc;
                float dd = 0.f;
#pragma unroll
                for (int k = 0; k < FS_G; ++k)
                    if (k < gc) {
                        const float dv = sv[k] - sb;
                        dd = fmaf(dv, dv, dd);
                    }
                const double ig = gc == FS_G ? inv_gn : 1.0 / ((double)gc * (double)rows);
                acc += (double)fmaf(dd, inv_n, mt) + (double)st * (double)st * ig;
            }
        }
        // the partial last block, by the warp whose turn it would be
        if (nfull < nblk && g == (nfull / FS_G) % FS_GROUPS) {
            const float* pb = p + (int64_t)(nblk - 1) * total;
            double t = (double)pb[0];
            if (second) {
                const double s1 = (double)pb[-S];
                t += s1 * s1 / (double)last_n;
            }
            acc += t;
        }
    }
    red[g][cx] = acc;
    __syncthreads();
    if (g == 0 && q < total) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < FS_GROUPS; ++k) t += red[k][cx];
        const int64_t n = q / row;
        const int v = (int)(q - n * row);
        if (v < S)
            S1o[n * S + v] = t;
        else
            S2o[n * S + (v - S)] = t;
    }
}

cudaError_t launch_fused_sums(const float* part, int nblk, int64_t Nt1, int S, int64_t count, int rows, double* S1,
                              double* S2, cudaStream_t st)
{
    int64_t total = Nt1 * 2 * S;
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
