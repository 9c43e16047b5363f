// Section IV-B step 2 on the GPU: a permutation of the primary sampling matrix
// that minimises the correlation between its columns.  The paper names a
// Cholesky-based method without giving it; this is the rank method of Iman and
// Conover (1982) with the identity as target correlation:
//   R[k][i] = a(pi_i(k)),  a(s) = Phi^-1((s + 1) / (N + 1)) - mean  (centred
//            van der Waerden scores paired by the design's own permutations),
//   T = R^T R / (N var a) = Q Q^T,   R* = R Q^-T,
//   pi'_i(k) = rank of R*[k][i] in column i (ascending, ties by sample index),
// and every sample keeps its uniform inside its new stratum.
//
// Kernels: the score table (FP64, one value per stratum), the centred score
// matrix [N][M] (FP32), its Gram matrix (FP32 tiles summed in FP64), a one-CTA
// Cholesky factorisation and triangular inverse in FP32 (T is within O(1/sqrt N)
// of the identity), R* by the FP32 GEMM, the per-column ranks by a segmented
// radix sort (CUB), and the design values from the new strata.
#include <cuda_bf16.h>

#include <cub/device/device_segmented_radix_sort.cuh>

#include "fmc_common.cuh"
#include "kernels.cuh"
#include "lhs_feistel.cuh"

namespace fmc {

// a(s) = Phi^-1((s + 1) / (N + 1)) in FP64, s < N; the tails through erfcinv so
// that the smallest probabilities keep their relative accuracy.
__global__ void ic_score_table_kernel(uint32_t N, double* __restrict__ a)
{
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        const double p = ((double)s + 1.0) / ((double)N + 1.0);
        const double SQRT2 = 1.4142135623730951;
        double z;
        if (p < 0.25)
            z = -SQRT2 * erfcinv(2.0 * p);
        else if (p > 0.75)
            z = SQRT2 * erfcinv(2.0 * (((double)N - (double)s) / ((double)N + 1.0)));
        else
            z = SQRT2 * erfinv(2.0 * p - 1.0);
        a[s] = z;
    }
}

// mean and sum of squares about it of the N scores (one CTA of 1024 threads)
__global__ void ic_score_moments_kernel(uint32_t N, const double* __restrict__ a, double* __restrict__ out)
{
    __shared__ double red[1024];
    double s = 0.0;
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) s += a[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double mean = red[0] / (double)N;
    __syncthreads();
    double q = 0.0;
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) q += (a[i] - mean) * (a[i] - mean);
    red[threadIdx.x] = q;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = mean;
        out[1] = red[0];
    }
}

// R[k][i] = a(pi_i(k)) - mean, FP32, row-major [N][M]
__global__ void ic_scores_kernel(uint32_t k0s, uint32_t k1s, uint32_t N, int M, int h, uint32_t mask,
                                 const double* __restrict__ a, const double* __restrict__ mom, float* __restrict__ R)
{
    const int64_t total = (int64_t)N * M;
    const double mean = mom[0];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / M;
        const int i = (int)(t - k * M);
        const uint32_t s = stratum((uint32_t)k, (uint32_t)i, N, h, mask, k0s, k1s);
        R[t] = (float)(a[s] - mean);
    }
}

// G = R^T R (FP64 [M][M], zeroed by the caller): a CTA of 256 threads sums a
// 64 x 64 tile over a range of IC_GRAM_ROWS rows in FP32 (4 x 4 outputs per
// thread, rows staged through shared memory) and adds it into G in FP64.
constexpr int IC_GT = 64, IC_GK = 32, IC_GRAM_ROWS = 1024;

__global__ void __launch_bounds__(256) ic_gram_kernel(int64_t N, int M, const float* __restrict__ R,
                                                      double* __restrict__ G)
{
    __shared__ float As[IC_GK][IC_GT];
    __shared__ float Bs[IC_GK][IC_GT];
    const int bi = blockIdx.x, bj = blockIdx.y;
    if (bj > bi) return;  // lower triangle of tiles; mirrored below
    const int i0 = bi * IC_GT, j0 = bj * IC_GT;
    const int64_t r0 = (int64_t)blockIdx.z * IC_GRAM_ROWS;
    const int64_t r1 = (r0 + IC_GRAM_ROWS < N) ? r0 + IC_GRAM_ROWS : N;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int64_t k0 = r0; k0 < r1; k0 += IC_GK) {
        for (int e = threadIdx.x; e < IC_GK * IC_GT; e += 256) {
            const int kk = e / IC_GT, c = e % IC_GT;
            const int64_t k = k0 + kk;
            As[kk][c] = (k < r1 && i0 + c < M) ? R[k * M + i0 + c] : 0.f;
            Bs[kk][c] = (k < r1 && j0 + c < M) ? R[k * M + j0 + c] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < IC_GK; ++kk) {
            float av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = i0 + ty * 4 + a, j = j0 + tx * 4 + b;
            if (i < M && j <= i) atomicAdd(&G[(int64_t)i * M + j], (double)acc[a][b]);
        }
}

// Cholesky factor Q of T = corr(R) (T_ij = G_ij / sqrt(G_ii G_jj)), right-looking,
// in place in the lower triangle of A [M][M] (FP32), by one CTA: column j is
// scaled by the square root of its pivot and the trailing lower triangle takes
// the rank-one update, warp by warp over its rows.  *ok = 0 if a pivot is not
// positive (T not positive definite).
constexpr int IC_MAX_M = 4096;

__global__ void __launch_bounds__(1024) ic_cholesky_kernel(int M, const double* __restrict__ G, float* __restrict__ A,
                                                           int* __restrict__ ok)
{
    __shared__ float col[IC_MAX_M];
    __shared__ float piv;
    __shared__ int good;
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid / 32, lane = tid % 32, nw = nt / 32;
    for (int64_t e = tid; e < (int64_t)M * M; e += nt) {
        const int i = (int)(e / M), j = (int)(e % M);
        float v = 0.f;
        if (i == j)
            v = 1.f;
        else if (j < i)
            v = (float)(G[e] / sqrt(G[(int64_t)i * M + i] * G[(int64_t)j * M + j]));
        A[e] = v;
    }
    if (tid == 0) good = 1;
    __syncthreads();
    for (int j = 0; j < M; ++j) {
        if (tid == 0) {
            const float d = A[(int64_t)j * M + j];
            if (!(d > 0.f)) good = 0;
            piv = d > 0.f ? sqrtf(d) : 1.f;
            A[(int64_t)j * M + j] = piv;
        }
        __syncthreads();
        if (!good) break;
        for (int i = j + 1 + tid; i < M; i += nt) {
            const float v = A[(int64_t)i * M + j] / piv;
            A[(int64_t)i * M + j] = v;
            col[i] = v;
        }
        __syncthreads();
        for (int i = j + 1 + warp; i < M; i += nw) {
            const float ci = col[i];
            float* row = A + (int64_t)i * M;
            for (int k = j + 1 + lane; k <= i; k += 32) row[k] = fmaf(-ci, col[k], row[k]);
        }
        __syncthreads();
    }
    if (tid == 0) *ok = good;
}

// B = Q^-T [M][M] (row-major): thread c solves Q w = e_c by forward
// substitution and writes w as row c of B (B[c][r] = (Q^-1)[r][c]).
__global__ void ic_inverse_kernel(int M, const float* __restrict__ Q, float* __restrict__ B)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= M) return;
    float* w = B + (int64_t)c * M;
    for (int r = 0; r < c; ++r) w[r] = 0.f;
    w[c] = 1.f / Q[(int64_t)c * M + c];
    for (int r = c + 1; r < M; ++r) {
        const float* q = Q + (int64_t)r * M;
        float v = 0.f;
        for (int k = c; k < r; ++k) v = fmaf(q[k], w[k], v);
        w[r] = -v / q[r];
    }
}

// keys for the per-column ranking: column i of R* [N][M] as order-preserving
// unsigned integers, transposed to [M][N], with the sample indices as values
__global__ void ic_keys_kernel(int64_t N, int M, const float* __restrict__ Rs, uint32_t* __restrict__ keys,
                               uint32_t* __restrict__ vals)
{
    const int64_t total = N * M;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / N);
        const int64_t k = t - (int64_t)i * N;
        uint32_t b = __float_as_uint(Rs[k * M + i]);
        b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
        keys[t] = b;
        vals[t] = (uint32_t)k;
    }
}

// strata [M][N]: sample sorted[i][r] takes stratum r of dimension i
__global__ void ic_ranks_kernel(int64_t N, int M, const uint32_t* __restrict__ sorted, uint32_t* __restrict__ strata)
{
    const int64_t total = N * M;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / N);
        const int64_t r = t - (int64_t)i * N;
        strata[(int64_t)i * N + sorted[t]] = (uint32_t)r;
    }
}

__global__ void ic_segments_kernel(int M, int64_t N, int* __restrict__ off)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= M) off[i] = (int)((int64_t)i * N);
}

// The design values of given strata [M][N]: zeta = Phi^-1((s + u) / N) with the
// sample's own uniform u (LHS) or u = 1/2 (midpoint), as the plain design does.
__device__ __forceinline__ float ic_value(uint32_t k, uint32_t i, uint32_t s, uint32_t N, int mode, uint32_t k0s,
                                          uint32_t k1s)
{
    uint64_t num2;
    if (mode == FMC_LHS_MIDPOINT) {
        num2 = ((uint64_t)s << 33) + (1ull << 32);
    } else {
        const uint32_t r = philox4x32_10(U4{k, i, 0u, 0u}, k0s, k1s).x;
        num2 = ((uint64_t)s << 33) + 2ull * r + 1ull;
    }
    return normal_from_fraction(num2, N);
}

// rows k0 .. k0+count-1: zeta [count][M] FP32
__global__ void ic_values_kernel(uint32_t k0s, uint32_t k1s, uint32_t N, int64_t k0, int64_t count, int M, int mode,
                                 const uint32_t* __restrict__ strata, float* __restrict__ zeta)
{
    const int64_t total = count * M;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / M;
        const int i = (int)(t - j * M);
        const int64_t k = k0 + j;
        zeta[t] = ic_value((uint32_t)k, (uint32_t)i, strata[(int64_t)i * N + k], N, mode, k0s, k1s);
    }
}

// rows k0 .. k0+count-1 in the split-BF16 layout [count][d][Ks] of the fused path
__global__ void ic_split_kernel(uint32_t k0s, uint32_t k1s, uint32_t N, int64_t k0, int64_t count, int d, int K, int Ks,
                                int mode, const uint32_t* __restrict__ strata, __nv_bfloat16* __restrict__ hi,
                                __nv_bfloat16* __restrict__ lo)
{
    const int64_t row = (int64_t)d * Ks;
    const int64_t total = count * row;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / row;
        const int rem = (int)(t - j * row);
        const int w = rem / Ks, kk = rem - w * Ks;
        float z = 0.f;
        if (kk < K) {
            const uint32_t i = (uint32_t)(w * K + kk);
            const int64_t k = k0 + j;
            z = ic_value((uint32_t)k, i, strata[(int64_t)i * N + k], N, mode, k0s, k1s);
        }
        const __nv_bfloat16 zh = __float2bfloat16_rn(z);
        hi[t] = zh;
        if (lo) lo[t] = __float2bfloat16_rn(z - __bfloat162float(zh));
    }
}

static int ic_grid(int64_t total, int block, int sms)
{
    int64_t g = (total + block - 1) / block;
    const int64_t cap = (int64_t)sms * 32;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

size_t ic_sort_bytes(int64_t N, int M)
{
    size_t bytes = 0;
    cub::DeviceSegmentedRadixSort::SortPairs(nullptr, bytes, (const uint32_t*)nullptr, (uint32_t*)nullptr,
                                             (const uint32_t*)nullptr, (uint32_t*)nullptr, (int64_t)N * M, M,
                                             (const int*)nullptr, (const int*)nullptr);
    return bytes;
}

cudaError_t launch_ic_strata(uint64_t seed, int64_t N, int M, const IcWork& w, uint32_t* strata, int sms,
                             cudaStream_t st)
{
    if (M > IC_MAX_M || N < 2 || N > 2147483647LL || (int64_t)N * M > 2147483647LL) return cudaErrorInvalidValue;
    const FeistelShape f = feistel_shape(N);
    const uint32_t k0s = (uint32_t)seed, k1s = (uint32_t)(seed >> 32);
    const int64_t NM = N * (int64_t)M;
    cudaError_t e;
    ic_score_table_kernel<<<ic_grid(N, 256, sms), 256, 0, st>>>((uint32_t)N, w.a);
    ic_score_moments_kernel<<<1, 1024, 0, st>>>((uint32_t)N, w.a, w.mom);
    ic_scores_kernel<<<ic_grid(NM, 256, sms), 256, 0, st>>>(k0s, k1s, (uint32_t)N, M, f.h, f.mask, w.a, w.mom, w.R);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(w.G, 0, sizeof(double) * (size_t)M * M, st)) != cudaSuccess) return e;
    const int tiles = (M + IC_GT - 1) / IC_GT;
    const int64_t slices = (N + IC_GRAM_ROWS - 1) / IC_GRAM_ROWS;
    if (slices > 65535) return cudaErrorInvalidValue;
    ic_gram_kernel<<<dim3(tiles, tiles, (unsigned)slices), 256, 0, st>>>(N, M, w.R, w.G);
    ic_cholesky_kernel<<<1, 1024, 0, st>>>(M, w.G, w.A, w.ok);
    ic_inverse_kernel<<<(M + 63) / 64, 64, 0, st>>>(M, w.A, w.B);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // R* = R Q^-T
    if ((e = launch_sgemm_nn(N, M, M, w.R, w.B, w.Rs, st)) != cudaSuccess) return e;
    // keys in place of R, then the sort per column into (Rs, vals_out)
    uint32_t* keys = reinterpret_cast<uint32_t*>(w.R);
    uint32_t* keys_out = reinterpret_cast<uint32_t*>(w.Rs);
    ic_keys_kernel<<<ic_grid(NM, 256, sms), 256, 0, st>>>(N, M, w.Rs, keys, w.vals);
    ic_segments_kernel<<<(M + 1 + 255) / 256, 256, 0, st>>>(M, N, w.off);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    size_t bytes = w.sort_bytes;
    if ((e = cub::DeviceSegmentedRadixSort::SortPairs(w.sort_tmp, bytes, keys, keys_out, w.vals, w.vals_out, NM, M,
                                                      w.off, w.off + 1, 0, 32, st)) != cudaSuccess)
        return e;
    ic_ranks_kernel<<<ic_grid(NM, 256, sms), 256, 0, st>>>(N, M, w.vals_out, strata);
    return cudaGetLastError();
}

cudaError_t launch_ic_values(uint64_t seed, int64_t N, int64_t k0, int64_t count, int M, int mode,
                             const uint32_t* strata, float* zeta, int sms, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    ic_values_kernel<<<ic_grid(count * M, 256, sms), 256, 0, st>>>((uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)N,
                                                                   k0, count, M, mode, strata, zeta);
    return cudaGetLastError();
}

cudaError_t launch_ic_split(uint64_t seed, int64_t N, int64_t k0, int64_t count, int d, int K, int mode,
                            const uint32_t* strata, void* hi, void* lo, int sms, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    const int Ks = round_up(K, 8);
    ic_split_kernel<<<ic_grid(count * d * Ks, 256, sms), 256, 0, st>>>(
        (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)N, k0, count, d, K, Ks, mode, strata,
        (__nv_bfloat16*)hi, (__nv_bfloat16*)lo);
    return cudaGetLastError();
}

}  // namespace fmc
