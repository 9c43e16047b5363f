/*
 * fmc_oracle.c -- plain, slow, FP64 CPU oracle for the fast Monte Carlo method
 * of Qiu, Lin, Chen, Liu and Song, "Fast Monte Carlo Simulation of Dynamic Power
 * Systems Under Continuous Random Disturbances" (arXiv 2007.03847).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA library is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library; both sides are written from
 * the paper and from the published definitions they cite.
 *
 * Every function follows one step of Algorithm 1 (Section IV-C):
 *   step 1  Latin hypercube sampling of the KL coefficients      (Section IV-B)
 *   step 2  reconstruction of the disturbance paths              (Eqs. kl, kle, eqkl)
 *   step 3  the dynamic simulation of every sample               (Eqs. state, algebra)
 *   step 4  expectation and variance of the response             (Algorithm 1 step 4)
 * The order of arithmetic is the order of the definitions; nothing is blocked,
 * fused or reordered for speed.
 *
 * Readings of points the paper leaves open (listed with reasons in the design
 * notes of the repository):
 *   - KL basis: the eigenfunctions of the Brownian covariance min(s,t),
 *     W(t) = sum_k zeta_k sqrt(2T)/((k-1/2)pi) sin((k-1/2)pi t/T).
 *   - The reconstructed path is consumed as increments dW_n = W(t_{n+1})-W(t_n).
 *   - Disturbance: Ornstein-Uhlenbeck dx = -theta x dt + sigma dW (Table I,
 *     Gaussian row with a general rate), advanced by Euler-Maruyama (Eq. distito
 *     with the missing xi_t restored).
 *   - System: Kron-reduced classical model, d(delta)/dt = omega_s * domega,
 *     2H d(domega)/dt = Pm + sum_w inj[i,w] x_w - Pe - D domega, with
 *     Pe_i = sum_j E_i E_j (G_ij cos(delta_i-delta_j) + B_ij sin(delta_i-delta_j))
 *            [+ E_i V (Ginf_i cos delta_i + Binf_i sin delta_i) with an infinite bus].
 *   - Integrator: classical RK4 (or Heun); the disturbance enters the stages at
 *     x_n, (x_n+x_{n+1})/2, (x_n+x_{n+1})/2, x_{n+1} (Heun: x_n, x_{n+1}).
 *   - Initial state: equilibrium at t = 0 (Section V-A), found by Newton; without
 *     an infinite bus machine 0 is the angle reference and balances power.
 *   - Variance: unbiased (N-1 denominator); NaN for N = 1.
 *   - LHS permutation: a keyed Feistel bijection with cycle walking, round
 *     function Philox4x32-10; uniform within the stratum from Philox4x32-10.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11.  Ten rounds of the 4x32 S-box with the published
 * multipliers and Weyl key increments.                                        */
/* ------------------------------------------------------------------------- */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {            /* key schedule: Weyl sequence */
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t philox_word0(uint64_t seed, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3)
{
    uint32_t ctr[4] = {w0, w1, w2, w3};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[0];
}

/* ------------------------------------------------------------------------- */
/* LHS permutation (Section IV-B, step 2: "random permutation").  For each
 * dimension i the permutation pi_i of {0..N-1} is a balanced Feistel network
 * on w = 2h bits (h = max(1, ceil(b/2)), 2^b the smallest power of two >= N),
 * six rounds, round function F_r(R) = Philox(key = seed,
 * counter = (R, i, 1 + r, 0)) word 0 masked to h bits, restricted to [0, N)
 * by cycle walking.                                                           */
/* ------------------------------------------------------------------------- */
#define ORACLE_FEISTEL_ROUNDS 6

static int bits_for(int64_t N)
{
    int b = 0;
    while (((int64_t)1 << b) < N) ++b;
    return b;
}

static uint32_t feistel_encrypt(uint64_t seed, uint32_t dim, int h, uint32_t x)
{
    uint32_t mask = (h >= 32) ? 0xFFFFFFFFu : ((1u << h) - 1u);
    uint32_t L = (x >> h) & mask;
    uint32_t R = x & mask;
    for (int r = 0; r < ORACLE_FEISTEL_ROUNDS; ++r) {
        uint32_t F = philox_word0(seed, R, dim, 1u + (uint32_t)r, 0u) & mask;
        uint32_t newL = R;
        uint32_t newR = L ^ F;
        L = newL;
        R = newR;
    }
    return (L << h) | R;
}

uint32_t oracle_lhs_stratum(uint64_t seed, int64_t N, int32_t dim, int64_t k)
{
    int b = bits_for(N);
    int h = (b + 1) / 2;
    if (h < 1) h = 1;
    uint32_t y = (uint32_t)k;
    do {
        y = feistel_encrypt(seed, (uint32_t)dim, h, y);
    } while ((int64_t)y >= N);
    return y;
}

/* Uniform in (0,1) attached to (sample k, dimension i): u = (r + 1/2) 2^-32
 * with r = Philox(key = seed, counter = (k, i, 0, 0)) word 0.                  */
double oracle_lhs_uniform(uint64_t seed, int32_t dim, int64_t k)
{
    uint32_t r = philox_word0(seed, (uint32_t)k, (uint32_t)dim, 0u, 0u);
    return ((double)r + 0.5) * (1.0 / 4294967296.0);
}

/* ------------------------------------------------------------------------- */
/* Inverse standard normal CDF: Wichura, "Algorithm AS 241: The percentage
 * points of the normal distribution", Applied Statistics 37 (1988), PPND16
 * (about 1e-16 relative accuracy).                                             */
/* ------------------------------------------------------------------------- */
double oracle_ppnd16(double p)
{
    if (p <= 0.0) return -INFINITY;
    if (p >= 1.0) return INFINITY;
    double q = p - 0.5;
    if (fabs(q) <= 0.425) {
        double r = 0.180625 - q * q;
        double num = (((((((2.5090809287301226727e+3 * r + 3.3430575583588128105e+4) * r
                        + 6.7265770927008700853e+4) * r + 4.5921953931549871457e+4) * r
                        + 1.3731693765509461125e+4) * r + 1.9715909503065514427e+3) * r
                        + 1.3314166789178437745e+2) * r + 3.3871328727963666080e+0);
        double den = (((((((5.2264952788528545610e+3 * r + 2.8729085735721942674e+4) * r
                        + 3.9307895800092710610e+4) * r + 2.1213794301586595867e+4) * r
                        + 5.3941960214247511077e+3) * r + 6.8718700749205790830e+2) * r
                        + 4.2313330701600911252e+1) * r + 1.0);
        return q * num / den;
    }
    double r = (q < 0.0) ? p : 1.0 - p;
    r = sqrt(-log(r));
    double val;
    if (r <= 5.0) {
        r -= 1.6;
        double num = (((((((7.74545014278341407640e-4 * r + 2.27238449892691845833e-2) * r
                        + 2.41780725177450611770e-1) * r + 1.27045825245236838258e+0) * r
                        + 3.64784832476320460504e+0) * r + 5.76949722146069140550e+0) * r
                        + 4.63033784615654529590e+0) * r + 1.42343711074968357734e+0);
        double den = (((((((1.05075007164441684324e-9 * r + 5.47593808499534494600e-4) * r
                        + 1.51986665636164571966e-2) * r + 1.48103976427480074590e-1) * r
                        + 6.89767334985100004550e-1) * r + 1.67638483018380384940e+0) * r
                        + 2.05319162663775882187e+0) * r + 1.0);
        val = num / den;
    } else {
        r -= 5.0;
        double num = (((((((2.01033439929228813265e-7 * r + 2.71155556874348757815e-5) * r
                        + 1.24266094738807843860e-3) * r + 2.65321895265761230930e-2) * r
                        + 2.96560571828504891230e-1) * r + 1.78482653991729133580e+0) * r
                        + 5.46378491116411436990e+0) * r + 6.65790464350110377720e+0);
        double den = (((((((2.04426310338993978564e-15 * r + 1.42151175831644588870e-7) * r
                        + 1.84631831751005468180e-5) * r + 7.86869131145613259100e-4) * r
                        + 1.48753612908506148525e-2) * r + 1.36929880922735805310e-1) * r
                        + 5.99832206555887937690e-1) * r + 1.0);
        val = num / den;
    }
    return (q < 0.0) ? -val : val;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1 step 1 / Section IV-B step 1: for dimension i and sample k the
 * stratum is s = pi_i(k), the probability p = (s + u)/N, and zeta = Phi^-1(p).
 * mode 0: LHS; mode 1: simple random sampling (p = u); mode 2: LHS at the
 * stratum midpoint (u = 1/2).  Rows k0 .. k0+count-1 of the N-sample design
 * are produced: zeta[(k-k0)*M + i], strata[i*count + (k-k0)] (may be NULL).    */
/* ------------------------------------------------------------------------- */
int oracle_lhs_sample(uint64_t seed, int64_t N, int64_t k0, int64_t count, int32_t M, int32_t mode,
                      double* zeta, uint32_t* strata)
{
    if (N < 1 || M < 1 || k0 < 0 || count < 0 || k0 + count > N || N > 2147483648LL) return -1;
    if (mode < 0 || mode > 2) return -1;
    for (int32_t i = 0; i < M; ++i) {
        for (int64_t j = 0; j < count; ++j) {
            int64_t k = k0 + j;
            double u = (mode == 2) ? 0.5 : oracle_lhs_uniform(seed, i, k);
            double p;
            uint32_t s = 0;
            if (mode == 1) {
                p = u;
                s = (uint32_t)k;
            } else {
                s = oracle_lhs_stratum(seed, N, i, k);
                p = ((double)s + u) / (double)N;
            }
            zeta[j * M + i] = oracle_ppnd16(p);
            if (strata) strata[(int64_t)i * count + j] = s;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Section IV-B step 2: a permutation of the primary sampling matrix that
 * minimises the correlation between its columns.  The paper points to a
 * Cholesky-based method without giving it; this is the rank method of Iman and
 * Conover ("A distribution-free approach to inducing rank correlation among
 * input variables", Commun. Statist. B 11 (1982)) with the identity as the
 * target correlation:
 *   1. score matrix R[k][i] = Phi^-1((pi_i(k) + 1) / (N + 1)) (van der Waerden
 *      scores, randomly paired by the design's own permutations pi_i);
 *   2. its sample correlation T = corr(R) and the Cholesky factor T = Q Q^T;
 *   3. R* = R Q^-T, whose sample correlation is the identity;
 *   4. each column of the design is rearranged to the ranks of the same column
 *      of R*: sample k of dimension i takes stratum pi'_i(k) = rank of R*[k][i]
 *      among R*[.][i] (ascending, ties by sample index), keeping its uniform
 *      u_ik, so zeta'[k][i] = Phi^-1((pi'_i(k) + u_ik) / N).
 * Every stratum is still hit once per dimension.  Needs N > M (T has full
 * rank) and an LHS mode.  Outputs (each may be NULL): zeta [N][M], strata
 * [M][N] (pi'), rstar [N][M].  Returns 0, or -1 on invalid arguments, -2 if T
 * is not positive definite.                                                   */
/* ------------------------------------------------------------------------- */
static const double* g_rank_col;   /* the column being ranked (qsort has no context) */
static int64_t g_rank_stride;

static int rank_cmp(const void* pa, const void* pb)
{
    int64_t a = *(const int64_t*)pa, b = *(const int64_t*)pb;
    double va = g_rank_col[a * g_rank_stride], vb = g_rank_col[b * g_rank_stride];
    if (va < vb) return -1;
    if (va > vb) return 1;
    return (a < b) ? -1 : (a > b);
}

int oracle_lhs_decorrelate(uint64_t seed, int64_t N, int32_t M, int32_t mode, double* zeta, uint32_t* strata,
                           double* rstar)
{
    if (N < 2 || M < 1 || N <= M || N > 2147483648LL || (mode != 0 && mode != 2)) return -1;
    double* R = (double*)malloc(sizeof(double) * (size_t)N * M);
    double* T = (double*)malloc(sizeof(double) * (size_t)M * M);
    double* mean = (double*)malloc(sizeof(double) * M);
    double* row = (double*)malloc(sizeof(double) * M);
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    uint32_t* sp = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
    int rc = 0;
    /* 1. scores */
    for (int64_t k = 0; k < N; ++k)
        for (int32_t i = 0; i < M; ++i)
            R[k * M + i] = oracle_ppnd16(((double)oracle_lhs_stratum(seed, N, i, k) + 1.0) / ((double)N + 1.0));
    /* 2. sample correlation and its Cholesky factor (lower triangle of T) */
    for (int32_t i = 0; i < M; ++i) {
        double m = 0.0;
        for (int64_t k = 0; k < N; ++k) m += R[k * M + i];
        mean[i] = m / (double)N;
    }
    for (int32_t i = 0; i < M; ++i)
        for (int32_t j = 0; j <= i; ++j) {
            double c = 0.0;
            for (int64_t k = 0; k < N; ++k) c += (R[k * M + i] - mean[i]) * (R[k * M + j] - mean[j]);
            T[i * M + j] = c;
        }
    for (int32_t i = 0; i < M; ++i)
        for (int32_t j = 0; j < i; ++j) T[i * M + j] /= sqrt(T[i * M + i] * T[j * M + j]);
    for (int32_t i = 0; i < M; ++i) T[i * M + i] = 1.0;
    for (int32_t j = 0; j < M && rc == 0; ++j) {
        double d = T[j * M + j];
        for (int32_t q = 0; q < j; ++q) d -= T[j * M + q] * T[j * M + q];
        if (!(d > 0.0)) {
            rc = -2;
            break;
        }
        d = sqrt(d);
        T[j * M + j] = d;
        for (int32_t i = j + 1; i < M; ++i) {
            double v = T[i * M + j];
            for (int32_t q = 0; q < j; ++q) v -= T[i * M + q] * T[j * M + q];
            T[i * M + j] = v / d;
        }
    }
    if (rc == 0) {
        /* 3. R* = R Q^-T, row by row: Q r*^T = r^T by forward substitution */
        for (int64_t k = 0; k < N; ++k) {
            for (int32_t i = 0; i < M; ++i) {
                double v = R[k * M + i];
                for (int32_t q = 0; q < i; ++q) v -= T[i * M + q] * row[q];
                row[i] = v / T[i * M + i];
            }
            for (int32_t i = 0; i < M; ++i) R[k * M + i] = row[i];
        }
        if (rstar) memcpy(rstar, R, sizeof(double) * (size_t)N * M);
        /* 4. ranks of R* per column; the design takes them as strata */
        for (int32_t i = 0; i < M; ++i) {
            for (int64_t k = 0; k < N; ++k) idx[k] = k;
            g_rank_col = R + i;
            g_rank_stride = M;
            qsort(idx, (size_t)N, sizeof(int64_t), rank_cmp);
            for (int64_t r = 0; r < N; ++r) sp[idx[r]] = (uint32_t)r;
            for (int64_t k = 0; k < N; ++k) {
                if (strata) strata[(int64_t)i * N + k] = sp[k];
                if (zeta) {
                    double u = (mode == 2) ? 0.5 : oracle_lhs_uniform(seed, i, k);
                    zeta[k * M + i] = oracle_ppnd16(((double)sp[k] + u) / (double)N);
                }
            }
        }
    }
    free(R); free(T); free(mean); free(row); free(idx); free(sp);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Appendix (Eqs. likelihood, like, reprob, ident): identification of a scalar
 * Ito model from a record xi_0, xi_h, ..., by minimising
 *   L'(q) = 1/4 sum_j (dxi_j - h mu_j)^2 / D_j + 1/2 sum_j log D_j,
 *   D_j = h sigma(xi_j)^2 / 2,  dxi_j = xi_{(j+1)h} - xi_{jh},
 * (the log-likelihood of the Euler-Maruyama transition densities, Eq. reprob,
 * without its constants; the sign of Eq. like read as the minimisation the
 * paper then performs).  Model: mu(x) = q0 + q1 x + q2 x^2 and either
 * sigma(x) = q3 + q4 x + q5 x^2 (kind 1, the form of Eq. windito) or
 * sigma(x)^2 = q3 + q4 x + q5 x^2 (kind 2, the Table I forms).
 * oracle_ito_objective returns L' and, if g / H are not NULL, its gradient [6]
 * and Hessian [6][6]; +inf where some D_j <= 0.                              */
/* ------------------------------------------------------------------------- */
double oracle_ito_objective(int32_t kind, const double* q, const double* xi, int64_t n, double h, double* g,
                            double* H)
{
    if (g) for (int a = 0; a < 6; ++a) g[a] = 0.0;
    if (H) for (int a = 0; a < 36; ++a) H[a] = 0.0;
    double L = 0.0;
    for (int64_t j = 0; j + 1 < n; ++j) {
        const double x = xi[j];
        const double phi[3] = {1.0, x, x * x};
        const double mu = q[0] + q[1] * x + q[2] * x * x;
        const double sp = q[3] + q[4] * x + q[5] * x * x;
        const double D = (kind == 1) ? 0.5 * h * sp * sp : 0.5 * h * sp;
        if (!(D > 0.0)) return INFINITY;
        const double r = (xi[j + 1] - x) - h * mu;
        L += 0.25 * r * r / D + 0.5 * log(D);
        if (!g && !H) continue;
        /* derivatives of l_j with respect to mu's coefficients and to D */
        const double lD = -0.25 * r * r / (D * D) + 0.5 / D;
        const double lDD = 0.5 * r * r / (D * D * D) - 0.5 / (D * D);
        double Dq[3], Dqq[3][3];
        for (int a = 0; a < 3; ++a) {
            Dq[a] = (kind == 1) ? h * sp * phi[a] : 0.5 * h * phi[a];
            for (int b = 0; b < 3; ++b) Dqq[a][b] = (kind == 1) ? h * phi[a] * phi[b] : 0.0;
        }
        if (g) {
            for (int a = 0; a < 3; ++a) {
                g[a] += -h * r * phi[a] / (2.0 * D);
                g[3 + a] += lD * Dq[a];
            }
        }
        if (H) {
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    H[a * 6 + b] += h * h * phi[a] * phi[b] / (2.0 * D);
                    const double mD = h * r * phi[a] / (2.0 * D * D) * Dq[b];
                    H[a * 6 + 3 + b] += mD;
                    H[(3 + b) * 6 + a] += mD;
                    H[(3 + a) * 6 + 3 + b] += lDD * Dq[a] * Dq[b] + lD * Dqq[a][b];
                }
        }
    }
    return L;
}

/* Cholesky solve of (A + lambda I) x = b on a 6 x 6 system; returns -1 if the
 * shifted matrix is not positive definite.                                    */
static int chol6(const double* A, double lambda, double* b)
{
    double Lm[36];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) {
            double v = A[i * 6 + j] + (i == j ? lambda : 0.0);
            for (int k = 0; k < j; ++k) v -= Lm[i * 6 + k] * Lm[j * 6 + k];
            if (i == j) {
                if (!(v > 0.0)) return -1;
                Lm[i * 6 + i] = sqrt(v);
            } else {
                Lm[i * 6 + j] = v / Lm[j * 6 + j];
            }
        }
    for (int i = 0; i < 6; ++i) {
        double v = b[i];
        for (int k = 0; k < i; ++k) v -= Lm[i * 6 + k] * b[k];
        b[i] = v / Lm[i * 6 + i];
    }
    for (int i = 5; i >= 0; --i) {
        double v = b[i];
        for (int k = i + 1; k < 6; ++k) v -= Lm[k * 6 + i] * b[k];
        b[i] = v / Lm[i * 6 + i];
    }
    return 0;
}

/* Newton's method on L' from the start q (overwritten by the estimate): the
 * Hessian is shifted by lambda I (Levenberg-Marquardt) until it is positive
 * definite, so every step descends, and a backtracking line search keeps L'
 * decreasing.  Stops when the step is below 1e-12 relative with an unshifted
 * (positive definite) Hessian.  Returns the iterations, or -1 if it did not
 * converge within 200.                                                        */
int oracle_ito_identify(int32_t kind, const double* xi, int64_t n, double h, double* q)
{
    if (n < 8 || !(h > 0.0) || (kind != 1 && kind != 2)) return -1;
    double g[6], H[36];
    double L = oracle_ito_objective(kind, q, xi, n, h, g, H);
    if (!isfinite(L)) return -1;
    for (int it = 1; it <= 200; ++it) {
        double step[6], lambda = 0.0, dmax = 0.0;
        for (int a = 0; a < 6; ++a) dmax = fmax(dmax, fabs(H[a * 6 + a]));
        for (;;) {
            for (int a = 0; a < 6; ++a) step[a] = -g[a];
            if (chol6(H, lambda, step) == 0) break;
            lambda = (lambda == 0.0) ? 1e-10 * dmax : 10.0 * lambda;
            if (lambda > 1e30) return -1;
        }
        double t = 1.0, qn[6], Ln = INFINITY;
        for (int ls = 0; ls < 60; ++ls, t *= 0.5) {
            for (int a = 0; a < 6; ++a) qn[a] = q[a] + t * step[a];
            Ln = oracle_ito_objective(kind, qn, xi, n, h, NULL, NULL);
            if (Ln <= L) break;
        }
        if (!(Ln <= L)) return -1;
        double dq = 0.0, qs = 0.0;
        for (int a = 0; a < 6; ++a) {
            dq += (qn[a] - q[a]) * (qn[a] - q[a]);
            qs += qn[a] * qn[a];
            q[a] = qn[a];
        }
        L = oracle_ito_objective(kind, q, xi, n, h, g, H);
        if (lambda == 0.0 && dq <= 1e-24 * (qs + 1e-300)) return it;
    }
    return -1;
}

/* ------------------------------------------------------------------------- */
/* The paper's "traditional MCs" (Section V-B): the disturbance advanced by the
 * scheme of Eq. (distito) with a fresh standard normal per step, i.e. Wiener
 * increments dW = sqrt(dt) zeta_{k,w,n} instead of a KL expansion.  The normal
 * of (sample k, disturbance w, step n) is Phi^-1(u), u = (r + 1/2) 2^-32 with
 * r = Philox(key = seed, counter = (k, n, 256, w / 4)) word (w mod 4).        */
/* ------------------------------------------------------------------------- */
#define ORACLE_TAG_EM 256u

double oracle_em_normal(uint64_t seed, int64_t k, int32_t w, int32_t n)
{
    uint32_t ctr[4] = {(uint32_t)k, (uint32_t)n, ORACLE_TAG_EM, (uint32_t)(w / 4)};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    double u = ((double)out[w % 4] + 0.5) * (1.0 / 4294967296.0);
    return oracle_ppnd16(u);
}

/* dW [count][d][Nt] of samples k0..k0+count-1. */
void oracle_em_increments(uint64_t seed, int64_t k0, int64_t count, int32_t d, int32_t Nt, double dt, double* dW)
{
    double sq = sqrt(dt);
    for (int64_t s = 0; s < count; ++s)
        for (int32_t w = 0; w < d; ++w)
            for (int32_t n = 0; n < Nt; ++n)
                dW[(s * d + w) * (int64_t)Nt + n] = sq * oracle_em_normal(seed, k0 + s, w, n);
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1 step 2, Eqs. (kl)/(kle): truncated KL expansion of a standard
 * Wiener process on [0,T] with the Brownian eigenbasis,
 *   W(t) = sum_{k=1..K} zeta_k c_k sin(a_k t),  a_k = (k-1/2) pi / T,
 *   c_k = sqrt(2T) / ((k-1/2) pi),
 * consumed as increments on the grid t_n = n dt, dt = T/Nt:
 *   phi[k-1][n] = c_k (sin(a_k t_{n+1}) - sin(a_k t_n)).                        */
/* ------------------------------------------------------------------------- */
void oracle_kl_increment_basis(int32_t K, double T, int32_t Nt, double* phi)
{
    double dt = T / (double)Nt;
    for (int32_t k = 1; k <= K; ++k) {
        double a = ((double)k - 0.5) * ORACLE_PI / T;
        double c = sqrt(2.0 * T) / (((double)k - 0.5) * ORACLE_PI);
        for (int32_t n = 0; n < Nt; ++n) {
            double t0 = (double)n * dt;
            double t1 = (double)(n + 1) * dt;
            phi[(int64_t)(k - 1) * Nt + n] = c * (sin(a * t1) - sin(a * t0));
        }
    }
}

/* The paper's own basis of Eq. (klb2): m_1(t) = 1/sqrt(T), m_j(t) = sqrt(2/T)
 * cos((j-1) pi t / T) for j >= 2, an orthonormal basis of white noise on [0, T].
 * Integrated from 0, as Eq. (kl) does: M_1(t) = t / sqrt(T) and
 * M_j(t) = sqrt(2T) / ((j-1) pi) sin((j-1) pi t / T); the increments are the
 * plain differences M_j(t_{n+1}) - M_j(t_n).                                 */
static double cos_basis_integral(int32_t j, double T, double t)
{
    if (j == 1) return t / sqrt(T);
    double a = (double)(j - 1) * ORACLE_PI / T;
    return sqrt(2.0 * T) / ((double)(j - 1) * ORACLE_PI) * sin(a * t);
}

/* basis 0: the Brownian eigenbasis above; basis 1: Eq. (klb2). */
void oracle_kl_increment_basis_ex(int32_t basis, int32_t K, double T, int32_t Nt, double* phi)
{
    if (basis == 0) {
        oracle_kl_increment_basis(K, T, Nt, phi);
        return;
    }
    double dt = T / (double)Nt;
    for (int32_t j = 1; j <= K; ++j)
        for (int32_t n = 0; n < Nt; ++n)
            phi[(int64_t)(j - 1) * Nt + n] =
                cos_basis_integral(j, T, (double)(n + 1) * dt) - cos_basis_integral(j, T, (double)n * dt);
}

/* W(t_n) itself (not used on the path; a pin for the covariance of the basis). */
void oracle_kl_path_basis(int32_t K, double T, int32_t Nt, double* psi)
{
    double dt = T / (double)Nt;
    for (int32_t k = 1; k <= K; ++k) {
        double a = ((double)k - 0.5) * ORACLE_PI / T;
        double c = sqrt(2.0 * T) / (((double)k - 0.5) * ORACLE_PI);
        for (int32_t n = 0; n <= Nt; ++n)
            psi[(int64_t)(k - 1) * (Nt + 1) + n] = c * sin(a * (double)n * dt);
    }
}

void oracle_kl_path_basis_ex(int32_t basis, int32_t K, double T, int32_t Nt, double* psi)
{
    if (basis == 0) {
        oracle_kl_path_basis(K, T, Nt, psi);
        return;
    }
    double dt = T / (double)Nt;
    for (int32_t j = 1; j <= K; ++j)
        for (int32_t n = 0; n <= Nt; ++n)
            psi[(int64_t)(j - 1) * (Nt + 1) + n] = cos_basis_integral(j, T, (double)n * dt);
}

/* The forcing of the random ODE of Eq. (eqkl): the time derivatives m_k(t) of
 * the KL basis functions, dW/dt = sum_k zeta_k m_k(t).  Brownian eigenbasis:
 * m_k(t) = sqrt(2/T) cos((k - 1/2) pi t / T); Eq. (klb2): m_1 = 1/sqrt(T),
 * m_j = sqrt(2/T) cos((j - 1) pi t / T).  Sampled at the half-step times
 * t = j dt / 2, j = 0 .. 2 Nt (the stage times of RK4 and Heun): mdot [K][2Nt+1]. */
void oracle_kl_forcing_basis_ex(int32_t basis, int32_t K, double T, int32_t Nt, double* mdot)
{
    const double hdt = 0.5 * T / (double)Nt;
    const int32_t J = 2 * Nt + 1;
    for (int32_t k = 1; k <= K; ++k) {
        double a, c;
        if (basis == 0) {
            a = ((double)k - 0.5) * ORACLE_PI / T;
            c = sqrt(2.0 / T);
        } else if (k == 1) {
            a = 0.0;
            c = 1.0 / sqrt(T);
        } else {
            a = (double)(k - 1) * ORACLE_PI / T;
            c = sqrt(2.0 / T);
        }
        for (int32_t j = 0; j < J; ++j) mdot[(int64_t)(k - 1) * J + j] = c * cos(a * (double)j * hdt);
    }
}

/* Eq. (eqkl) as increments: dW[s][w][n] = sum_k zeta[s][w*K + k] phi[k][n]. */
void oracle_kle_reconstruct(const double* zeta, int64_t count, int32_t d, int32_t K, const double* phi,
                            int32_t Nt, double* dW)
{
    for (int64_t s = 0; s < count; ++s)
        for (int32_t w = 0; w < d; ++w)
            for (int32_t n = 0; n < Nt; ++n) {
                double acc = 0.0;
                for (int32_t k = 0; k < K; ++k)
                    acc += zeta[s * (int64_t)d * K + (int64_t)w * K + k] * phi[(int64_t)k * Nt + n];
                dW[(s * d + w) * (int64_t)Nt + n] = acc;
            }
}

/* Euler-Maruyama for the OU disturbance driven by given increments (Eq. distito
 * with the drift of Table I's Gaussian row at rate theta):
 *   x_{n+1} = x_n - theta x_n dt + sigma dW_n,  x_0 = 0.
 * dW [count x Nt], x [count x (Nt+1)].                                          */
void oracle_ou_em(const double* dW, int64_t count, int32_t Nt, double dt, double theta, double sigma, double* x)
{
    for (int64_t s = 0; s < count; ++s) {
        double v = 0.0;
        x[s * (Nt + 1)] = 0.0;
        for (int32_t n = 0; n < Nt; ++n) {
            v = v + (-theta * v) * dt + sigma * dW[s * Nt + n];
            x[s * (Nt + 1) + n + 1] = v;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* General one-dimensional Ito disturbances (Section II, Table I; the wind model
 * of Eq. windito): d xi = mu(xi) dt + sigma(xi) dW with
 *   mu(x)       = m0 + m1 x + m2 x^2,
 *   kind 1:  sigma(x)   = s0 + s1 x + s2 x^2                 (Eq. windito),
 *   kind 2:  sigma(x)^2 = v0 + v1 x + v2 x^2 + v3 |x - a|    (Table I; sigma = 0 where negative),
 * started at x(0) = x0.  Advanced by the scheme of Eq. (distito),
 *   x_{n+1} = x_n + (mu(x_n) - c sigma(x_n) sigma'(x_n) / 2) dt + sigma(x_n) dW_n,
 * where c = 1 when the increments come from a (smooth) KL expansion: such paths
 * converge to the Stratonovich solution, and the term restores the Ito drift;
 * c = 0 for per-step normal increments.                                       */
/* ------------------------------------------------------------------------- */
typedef struct oracle_ito {
    int32_t kind;   /* 0: Ornstein-Uhlenbeck from the system's theta/sigma; 1, 2 as above */
    int32_t pad;
    double m0, m1, m2;
    double s0, s1, s2;
    double v0, v1, v2, v3, a;
    double x0;
} oracle_ito;

static double ito_sigma(const oracle_ito* p, double x)
{
    if (p->kind == 1) return p->s0 + p->s1 * x + p->s2 * x * x;
    double v = p->v0 + p->v1 * x + p->v2 * x * x + p->v3 * fabs(x - p->a);
    return v > 0.0 ? sqrt(v) : 0.0;
}

/* sigma(x) sigma'(x): kind 1 by the product rule; kind 2 as half the derivative
 * of sigma^2 (the sign of x - a for the absolute value; 0 where sigma^2 <= 0). */
static double ito_sigma_dsigma(const oracle_ito* p, double x)
{
    if (p->kind == 1) return ito_sigma(p, x) * (p->s1 + 2.0 * p->s2 * x);
    double v = p->v0 + p->v1 * x + p->v2 * x * x + p->v3 * fabs(x - p->a);
    if (v <= 0.0) return 0.0;
    double sg = (x > p->a) ? 1.0 : ((x < p->a) ? -1.0 : 0.0);
    return 0.5 * (p->v1 + 2.0 * p->v2 * x + p->v3 * sg);
}

double oracle_ito_step(const oracle_ito* p, double x, double dt, double dW, int32_t strat)
{
    double mu = p->m0 + p->m1 * x + p->m2 * x * x;
    if (strat) mu -= 0.5 * ito_sigma_dsigma(p, x);
    return x + mu * dt + ito_sigma(p, x) * dW;
}

/* Paths x [count][Nt+1] of one disturbance from increments dW [count][Nt]. */
void oracle_ito_paths(const oracle_ito* p, const double* dW, int64_t count, int32_t Nt, double dt, int32_t strat,
                      double* x)
{
    for (int64_t s = 0; s < count; ++s) {
        double v = p->x0;
        x[s * (Nt + 1)] = v;
        for (int32_t n = 0; n < Nt; ++n) {
            v = oracle_ito_step(p, v, dt, dW[s * Nt + n], strat);
            x[s * (Nt + 1) + n + 1] = v;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* The system (Eqs. state/algebra reduced to the classical model).            */
/* ------------------------------------------------------------------------- */
typedef struct oracle_system {
    int32_t n;           /* machines */
    int32_t d;           /* OU disturbances = Wiener processes */
    int32_t K;           /* KL terms per Wiener process */
    int32_t Nt;          /* time steps, T = Nt dt */
    double T;
    double dt;
    double omega_s;      /* synchronous speed, rad/s */
    int32_t has_inf_bus;
    int32_t integrator;  /* 0 = RK4, 1 = Heun */
    double Vinf;
    const double* G;     /* [n*n] Kron-reduced conductance */
    const double* B;     /* [n*n] Kron-reduced susceptance */
    const double* Ginf;  /* [n] machine-to-infinite-bus conductance (has_inf_bus) */
    const double* Binf;  /* [n] machine-to-infinite-bus susceptance */
    const double* H;     /* [n] inertia constants, s */
    const double* D;     /* [n] damping, p.u. power per p.u. speed */
    const double* E;     /* [n] internal EMFs */
    const double* Pm;    /* [n] mechanical power; Pm[0] is replaced by the balance
                            of machine 0 when there is no infinite bus */
    const double* theta; /* [d] OU mean-reversion rates, 1/s */
    const double* sigma; /* [d] OU diffusion, p.u./sqrt(s) */
    const double* inject;/* [n*d] how disturbance w enters machine i's power */
    const double* init_delta; /* [n] initial angles instead of the equilibrium, or NULL */
    int32_t basis;       /* 0: Brownian eigenbasis (sine), 1: Eq. (klb2) (cosine) */
    int32_t em;          /* 1: per-step normal increments (Eq. distito), not the KL expansion */
    uint64_t em_seed;    /* Philox key of those normals */
    int64_t em_k0;       /* index of the first simulated sample */
    /* an event in the style of the paper's generator trip (Section V-A): from grid
     * time t_{event_step} on, machine event_machine's mechanical power changes by
     * event_dpm (negative: generation lost); event_machine < 0: no event */
    int32_t event_machine;
    int32_t event_step;
    double event_dpm;
    /* [d] general disturbances, or NULL: all Ornstein-Uhlenbeck (theta, sigma).
     * The system is at equilibrium with every disturbance at its x0: the power
     * balance sees inject (x - x0).                                            */
    const oracle_ito* ito;
    /* 1: the disturbances follow the random ODE of Eq. (eqkl), driven by the
     * smooth forcing f(t) = sum_k zeta_k m_k(t) and integrated jointly with the
     * swing equations by the same RK4 or Heun stages (the swing stage j sees the
     * disturbance's own stage value); 0: Euler-Maruyama on the KL increments.
     * The smooth paths converge to the Stratonovich solution, so a general Ito
     * disturbance carries the drift mu - sigma sigma' / 2 (as the KL increments do). */
    int32_t smooth;
} oracle_system;

/* Electrical power, textbook pairwise form:
 *   Pe_i = sum_j E_i E_j (G_ij cos(delta_i - delta_j) + B_ij sin(delta_i - delta_j))
 * (form 0), or the same sum written with a_j = E_j cos delta_j, b_j = E_j sin delta_j
 * as Pe_i = a_i (G a - B b)_i + b_i (G b + B a)_i (form 1).                   */
void oracle_electrical_power(const oracle_system* s, const double* delta, double* pe, int32_t form)
{
    int n = s->n;
    if (form == 0) {
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int j = 0; j < n; ++j) {
                double dij = delta[i] - delta[j];
                acc += s->E[i] * s->E[j] * (s->G[i * n + j] * cos(dij) + s->B[i * n + j] * sin(dij));
            }
            if (s->has_inf_bus)
                acc += s->E[i] * s->Vinf * (s->Ginf[i] * cos(delta[i]) + s->Binf[i] * sin(delta[i]));
            pe[i] = acc;
        }
    } else {
        double* a = (double*)malloc(sizeof(double) * 2 * n);
        double* b = a + n;
        for (int j = 0; j < n; ++j) {
            a[j] = s->E[j] * cos(delta[j]);
            b[j] = s->E[j] * sin(delta[j]);
        }
        for (int i = 0; i < n; ++i) {
            double u = 0.0, v = 0.0;
            for (int j = 0; j < n; ++j) {
                u += s->G[i * n + j] * a[j] - s->B[i * n + j] * b[j];
                v += s->G[i * n + j] * b[j] + s->B[i * n + j] * a[j];
            }
            double acc = a[i] * u + b[i] * v;
            if (s->has_inf_bus)
                acc += s->Vinf * (s->Ginf[i] * a[i] + s->Binf[i] * b[i]);
            pe[i] = acc;
        }
        free(a);
    }
}

/* Dense linear solve A x = r by Gaussian elimination with partial pivoting.
 * A is m x m row-major and is overwritten.  Returns 0, or -1 if singular.       */
static int solve_dense(double* A, double* r, int m)
{
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int row = col + 1; row < m; ++row)
            if (fabs(A[row * m + col]) > fabs(A[piv * m + col])) piv = row;
        if (fabs(A[piv * m + col]) == 0.0) return -1;
        if (piv != col) {
            for (int j = 0; j < m; ++j) {
                double t = A[col * m + j]; A[col * m + j] = A[piv * m + j]; A[piv * m + j] = t;
            }
            double t = r[col]; r[col] = r[piv]; r[piv] = t;
        }
        for (int row = col + 1; row < m; ++row) {
            double f = A[row * m + col] / A[col * m + col];
            for (int j = col; j < m; ++j) A[row * m + j] -= f * A[col * m + j];
            r[row] -= f * r[col];
        }
    }
    for (int row = m - 1; row >= 0; --row) {
        double acc = r[row];
        for (int j = row + 1; j < m; ++j) acc -= A[row * m + j] * r[j];
        r[row] = acc / A[row * m + row];
    }
    return 0;
}

/* Equilibrium at t = 0 (Section V-A: "the system is assumed at equilibrium"):
 * Newton's method on Pm_i - Pe_i(delta) = 0 from a flat start delta = 0, with
 * the analytic Jacobian of the pairwise form.  With an infinite bus all n
 * angles are unknown.  Without one, delta_0 = 0 is the reference and machine 0
 * balances the power: equations i = 1..n-1 fix delta_1..delta_{n-1}, then
 * pm_eq[0] = Pe_0(delta).  Returns the iteration count, or -1 on failure.      */
int oracle_equilibrium(const oracle_system* s, double* delta0, double* pm_eq)
{
    int n = s->n;
    int first = s->has_inf_bus ? 0 : 1;
    int m = n - first;
    double* pe = (double*)malloc(sizeof(double) * n);
    double* J = (double*)malloc(sizeof(double) * (m > 0 ? m * m : 1));
    double* F = (double*)malloc(sizeof(double) * (m > 0 ? m : 1));
    for (int i = 0; i < n; ++i) { delta0[i] = 0.0; pm_eq[i] = s->Pm[i]; }
    int it = 0, ok = (m == 0);
    for (it = 0; it < 100 && m > 0; ++it) {
        oracle_electrical_power(s, delta0, pe, 0);
        double fmax = 0.0;
        for (int a = 0; a < m; ++a) {
            int i = a + first;
            F[a] = s->Pm[i] - pe[i];
            if (fabs(F[a]) > fmax) fmax = fabs(F[a]);
        }
        if (fmax < 1e-13) { ok = 1; break; }
        /* J[a][b] = d Pe_i / d delta_j, i = a+first, j = b+first */
        for (int a = 0; a < m; ++a) {
            int i = a + first;
            double diag = 0.0;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                double dij = delta0[i] - delta0[j];
                double dPe_ddj = s->E[i] * s->E[j] * (s->G[i * n + j] * sin(dij) - s->B[i * n + j] * cos(dij));
                diag -= dPe_ddj;
                if (j >= first) J[a * m + (j - first)] = dPe_ddj;
            }
            if (s->has_inf_bus)
                diag += s->E[i] * s->Vinf * (-s->Ginf[i] * sin(delta0[i]) + s->Binf[i] * cos(delta0[i]));
            J[a * m + a] = diag;
        }
        /* Newton: J ddelta = F (since F = Pm - Pe and dF/ddelta = -J) */
        if (solve_dense(J, F, m) != 0) break;
        for (int a = 0; a < m; ++a) delta0[a + first] += F[a];
    }
    if (ok && !s->has_inf_bus) {
        oracle_electrical_power(s, delta0, pe, 0);
        pm_eq[0] = pe[0];
    }
    free(pe); free(J); free(F);
    return ok ? it : -1;
}

/* ------------------------------------------------------------------------- */
/* The random ODE of Eq. (eqkl) for disturbance q: dx/dt = mu~(x) + sigma(x) f,   */
/* f the smooth forcing at the stage time; mu~ = -theta x for the OU disturbance, */
/* mu - sigma sigma' / 2 for a general one (see oracle_system.smooth).           */
/* ------------------------------------------------------------------------- */
static double smooth_rate(const oracle_system* s, int q, double x, double f)
{
    if (s->ito && s->ito[q].kind != 0) {
        const oracle_ito* p = &s->ito[q];
        double mu = p->m0 + p->m1 * x + p->m2 * x * x - 0.5 * ito_sigma_dsigma(p, x);
        return mu + ito_sigma(p, x) * f;
    }
    return -s->theta[q] * x + s->sigma[q] * f;
}

/* One step of the disturbance's random ODE from x at grid time t_n, with the
 * forcing f0 = f(t_n), fh = f(t_n + dt/2), f1 = f(t_{n+1}): the stage values
 * X[0..3] (RK4; Heun fills X[0..1]) and the new value.                        */
static double smooth_step(const oracle_system* s, int q, double x, double f0, double fh, double f1, double X[4])
{
    const double dt = s->dt;
    if (s->integrator == 0) {
        X[0] = x;
        double k1 = smooth_rate(s, q, X[0], f0);
        X[1] = x + 0.5 * dt * k1;
        double k2 = smooth_rate(s, q, X[1], fh);
        X[2] = x + 0.5 * dt * k2;
        double k3 = smooth_rate(s, q, X[2], fh);
        X[3] = x + dt * k3;
        double k4 = smooth_rate(s, q, X[3], f1);
        return x + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
    }
    X[0] = x;
    double k1 = smooth_rate(s, q, X[0], f0);
    X[1] = x + dt * k1;
    double k2 = smooth_rate(s, q, X[1], f1);
    X[2] = X[3] = X[1];
    return x + 0.5 * dt * (k1 + k2);
}

/* The disturbance q alone under the smooth forcing (the random ODE of
 * Eq. (eqkl)), by the system's integrator and the same step as the simulation:
 * x [count][Nt+1] for the coefficient rows zeta [count][d*K].                 */
int oracle_smooth_paths(const oracle_system* s, const double* zeta, int64_t count, int32_t q, double* x)
{
    const int Nt = s->Nt, K = s->K, d = s->d;
    if (q < 0 || q >= d || Nt < 1 || K < 1 || count < 1) return -1;
    const int64_t J = 2 * (int64_t)Nt + 1;
    double* mdot = (double*)malloc(sizeof(double) * (size_t)K * (size_t)J);
    double* f = (double*)malloc(sizeof(double) * (size_t)J);
    oracle_kl_forcing_basis_ex(s->basis, K, s->T, Nt, mdot);
    for (int64_t smp = 0; smp < count; ++smp) {
        const double* z = zeta + smp * (int64_t)d * K + (int64_t)q * K;
        for (int64_t j = 0; j < J; ++j) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc += z[k] * mdot[(int64_t)k * J + j];
            f[j] = acc;
        }
        double v = (s->ito && s->ito[q].kind != 0) ? s->ito[q].x0 : 0.0;
        double* row = x + smp * (int64_t)(Nt + 1);
        row[0] = v;
        for (int step = 0; step < Nt; ++step) {
            double X[4];
            v = smooth_step(s, q, v, f[2 * step], f[2 * step + 1], f[2 * step + 2], X);
            row[step + 1] = v;
        }
    }
    free(mdot);
    free(f);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1 step 3: the dynamic simulation of one sample.                   */
/* ------------------------------------------------------------------------- */
typedef struct sim_ws {
    double *delta, *omega, *pe, *force, *x, *xn, *xs;
    double *k1d, *k1w, *k2d, *k2w, *k3d, *k3w, *k4d, *k4w, *tmpd, *tmpw;
    double *dW;
    double *xst;  /* [4][d] stage values of the smooth form */
    double *f;    /* [d][2 Nt + 1] the smooth forcing of this sample */
} sim_ws;

static void ws_alloc(sim_ws* w, int n, int d, int Nt)
{
    double* buf = (double*)calloc((size_t)(16 * n + 7 * d) + (size_t)d * Nt + (size_t)d * (2 * Nt + 1),
                                  sizeof(double));
    w->delta = buf; w->omega = buf + n; w->pe = buf + 2 * n; w->force = buf + 3 * n;
    w->k1d = buf + 4 * n; w->k1w = buf + 5 * n; w->k2d = buf + 6 * n; w->k2w = buf + 7 * n;
    w->k3d = buf + 8 * n; w->k3w = buf + 9 * n; w->k4d = buf + 10 * n; w->k4w = buf + 11 * n;
    w->tmpd = buf + 12 * n; w->tmpw = buf + 13 * n;
    w->x = buf + 16 * n; w->xn = w->x + d; w->xs = w->xn + d;
    w->xst = w->xs + d;
    w->dW = w->xst + 4 * d;
    w->f = w->dW + (size_t)d * Nt;
}

/* Right-hand side of the swing equations at disturbance state xs. */
static void swing_rhs(const oracle_system* s, const double* pm_eq, const double* delta, const double* omega,
                      const double* xs, sim_ws* w, int32_t pe_form, int32_t event_on, double* ddelta, double* domega)
{
    int n = s->n, d = s->d;
    oracle_electrical_power(s, delta, w->pe, pe_form);
    for (int i = 0; i < n; ++i) {
        double force = pm_eq[i];
        if (event_on && i == s->event_machine) force += s->event_dpm;
        for (int q = 0; q < d; ++q) force += s->inject[i * d + q] * (xs[q] - (s->ito ? s->ito[q].x0 : 0.0));
        ddelta[i] = s->omega_s * omega[i];
        domega[i] = (force - w->pe[i] - s->D[i] * omega[i]) / (2.0 * s->H[i]);
    }
}

/* Test hook, off unless a pin test turns it on: plants a known mistake in the
 * disturbance values the swing stages see (increment form only), so that the
 * stage-forcing pin can show that it catches one.  1: x_n at every stage (the
 * forcing lags by half a step); 2: x_{n+1} at the two midpoint stages.  Not
 * thread-safe; tests set it around single-threaded calls.                    */
static int32_t g_stage_plant = 0;

void oracle_plant_stage_forcing(int32_t mode) { g_stage_plant = mode; }

/* Integrates one sample whose increments are dW[w][n]; writes the trajectory
 * traj[n][j] (j < n: delta_j, j >= n: domega_j) for n = 0..Nt.  An event (see
 * oracle_system) acts on whole steps from step event_step on.                 */
static void simulate_one(const oracle_system* s, const double* delta0, const double* pm_eq, sim_ws* w,
                         int32_t pe_form, double* traj)
{
    int n = s->n, d = s->d, Nt = s->Nt;
    double dt = s->dt;
    int32_t ev = 0;
    for (int i = 0; i < n; ++i) { w->delta[i] = delta0[i]; w->omega[i] = 0.0; }
    for (int q = 0; q < d; ++q) w->x[q] = s->ito ? s->ito[q].x0 : 0.0;
    for (int i = 0; i < n; ++i) { traj[i] = w->delta[i]; traj[n + i] = w->omega[i]; }
    for (int step = 0; step < Nt; ++step) {
        ev = (s->event_machine >= 0 && step >= s->event_step);
        /* the disturbance values the swing stages see: xa, xb, xc, xd (RK4) or
         * xa, xb (Heun) */
        const double *xa, *xb, *xc, *xd;
        if (s->smooth) {
            /* the random ODE of Eq. (eqkl), stage by stage with the swing equations */
            const int64_t J = 2 * (int64_t)Nt + 1;
            for (int q = 0; q < d; ++q) {
                const double* f = w->f + (int64_t)q * J + 2 * (int64_t)step;
                double X[4];
                w->xn[q] = smooth_step(s, q, w->x[q], f[0], f[1], f[2], X);
                for (int st = 0; st < 4; ++st) w->xst[st * d + q] = X[st];
            }
            xa = w->xst;
            xb = w->xst + d;
            xc = w->xst + 2 * d;
            xd = w->xst + 3 * d;
        } else {
            /* Euler-Maruyama for the OU disturbance (Eq. distito, Table I) */
            for (int q = 0; q < d; ++q)
                w->xn[q] = (s->ito && s->ito[q].kind != 0)
                               ? oracle_ito_step(&s->ito[q], w->x[q], dt, w->dW[(int64_t)q * Nt + step], !s->em)
                               : w->x[q] + (-s->theta[q] * w->x[q]) * dt + s->sigma[q] * w->dW[(int64_t)q * Nt + step];
            /* RK4 sees x at t_n, at the midpoint as the mean of the grid values, and
             * at t_{n+1}; Heun sees the grid values */
            for (int q = 0; q < d; ++q) w->xs[q] = 0.5 * (w->x[q] + w->xn[q]);
            xa = w->x;
            xb = (s->integrator == 0) ? w->xs : w->xn;
            xc = w->xs;
            xd = w->xn;
            if (g_stage_plant == 1) { xb = w->x; xc = w->x; xd = w->x; }
            if (g_stage_plant == 2 && s->integrator == 0) { xb = w->xn; xc = w->xn; }
        }
        if (s->integrator == 0) {
            /* classical RK4 */
            swing_rhs(s, pm_eq, w->delta, w->omega, xa, w, pe_form, ev, w->k1d, w->k1w);
            for (int i = 0; i < n; ++i) {
                w->tmpd[i] = w->delta[i] + 0.5 * dt * w->k1d[i];
                w->tmpw[i] = w->omega[i] + 0.5 * dt * w->k1w[i];
            }
            swing_rhs(s, pm_eq, w->tmpd, w->tmpw, xb, w, pe_form, ev, w->k2d, w->k2w);
            for (int i = 0; i < n; ++i) {
                w->tmpd[i] = w->delta[i] + 0.5 * dt * w->k2d[i];
                w->tmpw[i] = w->omega[i] + 0.5 * dt * w->k2w[i];
            }
            swing_rhs(s, pm_eq, w->tmpd, w->tmpw, xc, w, pe_form, ev, w->k3d, w->k3w);
            for (int i = 0; i < n; ++i) {
                w->tmpd[i] = w->delta[i] + dt * w->k3d[i];
                w->tmpw[i] = w->omega[i] + dt * w->k3w[i];
            }
            swing_rhs(s, pm_eq, w->tmpd, w->tmpw, xd, w, pe_form, ev, w->k4d, w->k4w);
            for (int i = 0; i < n; ++i) {
                w->delta[i] += dt / 6.0 * (w->k1d[i] + 2.0 * w->k2d[i] + 2.0 * w->k3d[i] + w->k4d[i]);
                w->omega[i] += dt / 6.0 * (w->k1w[i] + 2.0 * w->k2w[i] + 2.0 * w->k3w[i] + w->k4w[i]);
            }
        } else {
            /* Heun (explicit trapezoid) */
            swing_rhs(s, pm_eq, w->delta, w->omega, xa, w, pe_form, ev, w->k1d, w->k1w);
            for (int i = 0; i < n; ++i) {
                w->tmpd[i] = w->delta[i] + dt * w->k1d[i];
                w->tmpw[i] = w->omega[i] + dt * w->k1w[i];
            }
            swing_rhs(s, pm_eq, w->tmpd, w->tmpw, xb, w, pe_form, ev, w->k2d, w->k2w);
            for (int i = 0; i < n; ++i) {
                w->delta[i] += 0.5 * dt * (w->k1d[i] + w->k2d[i]);
                w->omega[i] += 0.5 * dt * (w->k1w[i] + w->k2w[i]);
            }
        }
        for (int q = 0; q < d; ++q) w->x[q] = w->xn[q];
        double* row = traj + (int64_t)(step + 1) * 2 * n;
        for (int i = 0; i < n; ++i) { row[i] = w->delta[i]; row[n + i] = w->omega[i]; }
    }
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1 steps 2-4 over `count` samples whose coefficients are the rows
 * of zeta [count x d*K].  Optional outputs: the increments dW [count x d x Nt],
 * the trajectories traj [count x (Nt+1) x 2n], and the moments mean, var
 * [(Nt+1) x 2n].  Moments use the shifted-sum identity
 *   mean = c + S1/N,  var = (S2 - S1^2/N)/(N-1),  S1 = sum(x-c), S2 = sum (x-c)^2,
 * with c the trajectory of the first sample (any c gives the same values in
 * exact arithmetic; a c near the data keeps the FP64 sums well conditioned).
 * Work is split over nthreads POSIX threads by contiguous sample blocks and the
 * per-thread sums are added in thread order.                                   */
/* ------------------------------------------------------------------------- */
/* The paper's response function (Section V-B): the RMS over the horizon of the
 * system frequency deviation, here the inertia-weighted (centre-of-inertia)
 * speed deviation omega_coi = sum_i H_i domega_i / sum_i H_i, on the grid:
 *   RRF = sqrt( (1/Nt) sum_{n=1..Nt} omega_coi(t_n)^2 )   (p.u. of speed).      */
static double rrf_of(const oracle_system* s, const double* traj)
{
    int n = s->n, Nt = s->Nt;
    double hs = 0.0;
    for (int i = 0; i < n; ++i) hs += s->H[i];
    double acc = 0.0;
    for (int step = 1; step <= Nt; ++step) {
        const double* row = traj + (int64_t)step * 2 * n;
        double c = 0.0;
        for (int i = 0; i < n; ++i) c += s->H[i] * row[n + i];
        c /= hs;
        acc += c * c;
    }
    return sqrt(acc / (double)Nt);
}

typedef struct sim_job {
    const oracle_system* s;
    const double* zeta;
    const double* phi;
    const double* mdot;  /* [K][2Nt+1] the forcing basis (smooth form) */
    const double* delta0;
    const double* pm_eq;
    const double* shift;
    int64_t s0, s1;
    int32_t pe_form;
    double* dW_out;
    double* traj_out;
    double* S1;
    double* S2;
    double* rrf_out;
} sim_job;

static void* sim_worker(void* arg)
{
    sim_job* job = (sim_job*)arg;
    const oracle_system* s = job->s;
    int n = s->n, d = s->d, K = s->K, Nt = s->Nt;
    int64_t cols = (int64_t)(Nt + 1) * 2 * n;
    sim_ws w;
    ws_alloc(&w, n, d, Nt);
    double* traj_local = (double*)malloc(sizeof(double) * cols);
    for (int64_t smp = job->s0; smp < job->s1; ++smp) {
        if (s->em) {
            oracle_em_increments(s->em_seed, s->em_k0 + smp, 1, d, Nt, s->dt, w.dW);
        } else {
            const double* z = job->zeta + smp * (int64_t)d * K;
            for (int q = 0; q < d; ++q)
                for (int step = 0; step < Nt; ++step) {
                    double acc = 0.0;
                    for (int k = 0; k < K; ++k) acc += z[q * K + k] * job->phi[(int64_t)k * Nt + step];
                    w.dW[(int64_t)q * Nt + step] = acc;
                }
        }
        if (s->smooth) {
            /* f[w][j] = sum_k zeta[w*K + k] m_k(j dt / 2) */
            const double* z = job->zeta + smp * (int64_t)d * K;
            const int64_t J = 2 * (int64_t)Nt + 1;
            for (int q = 0; q < d; ++q)
                for (int64_t j = 0; j < J; ++j) {
                    double acc = 0.0;
                    for (int k = 0; k < K; ++k) acc += z[q * K + k] * job->mdot[(int64_t)k * J + j];
                    w.f[(int64_t)q * J + j] = acc;
                }
        }
        if (job->dW_out) memcpy(job->dW_out + smp * (int64_t)d * Nt, w.dW, sizeof(double) * (size_t)d * Nt);
        double* traj = job->traj_out ? job->traj_out + smp * cols : traj_local;
        simulate_one(s, job->delta0, job->pm_eq, &w, job->pe_form, traj);
        if (job->rrf_out) job->rrf_out[smp] = rrf_of(s, traj);
        if (job->S1) {
            for (int64_t c = 0; c < cols; ++c) {
                double v = traj[c] - job->shift[c];
                job->S1[c] += v;
                job->S2[c] += v * v;
            }
        }
    }
    free(traj_local);
    free(w.delta);
    return NULL;
}

int oracle_simulate(const oracle_system* s, const double* zeta, int64_t count, int32_t pe_form, int32_t nthreads,
                    double* delta0_out, double* pm_eq_out, double* dW_out, double* traj_out, double* mean,
                    double* var, double* rrf)
{
    int n = s->n, Nt = s->Nt;
    if (n < 1 || s->d < 1 || s->K < 1 || Nt < 1 || count < 1 || s->dt <= 0.0) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > count) nthreads = (int32_t)count;
    int64_t cols = (int64_t)(Nt + 1) * 2 * n;
    if (s->smooth && s->em) return -1;  /* per-step normals have no smooth form */
    double* phi = (double*)malloc(sizeof(double) * (size_t)s->K * Nt);
    oracle_kl_increment_basis_ex(s->basis, s->K, s->T, Nt, phi);
    double* mdot = NULL;
    if (s->smooth) {
        mdot = (double*)malloc(sizeof(double) * (size_t)s->K * (2 * (size_t)Nt + 1));
        oracle_kl_forcing_basis_ex(s->basis, s->K, s->T, Nt, mdot);
    }
    double* delta0 = (double*)malloc(sizeof(double) * n);
    double* pm_eq = (double*)malloc(sizeof(double) * n);
    if (oracle_equilibrium(s, delta0, pm_eq) < 0) {
        free(phi); free(mdot); free(delta0); free(pm_eq);
        return -2;
    }
    /* a prescribed initial state (used to test the integrator off equilibrium) */
    if (s->init_delta)
        for (int i = 0; i < n; ++i) delta0[i] = s->init_delta[i];
    if (delta0_out) memcpy(delta0_out, delta0, sizeof(double) * n);
    if (pm_eq_out) memcpy(pm_eq_out, pm_eq, sizeof(double) * n);

    double* shift = NULL;
    double* S1 = NULL;
    double* S2 = NULL;
    int want_moments = (mean != NULL || var != NULL);
    if (want_moments) {
        /* shift = trajectory of the first sample, integrated once on its own */
        shift = (double*)malloc(sizeof(double) * cols);
        sim_job j0 = {s, zeta, phi, mdot, delta0, pm_eq, NULL, 0, 1, pe_form, NULL, shift, NULL, NULL, NULL};
        /* traj_out for sample 0 only points at `shift`; S1 == NULL disables sums */
        sim_worker(&j0);
        S1 = (double*)calloc((size_t)cols * nthreads, sizeof(double));
        S2 = (double*)calloc((size_t)cols * nthreads, sizeof(double));
    }
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
    sim_job* jobs = (sim_job*)malloc(sizeof(sim_job) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].s = s; jobs[t].zeta = zeta; jobs[t].phi = phi; jobs[t].mdot = mdot; jobs[t].delta0 = delta0;
        jobs[t].pm_eq = pm_eq; jobs[t].shift = shift;
        jobs[t].s0 = count * t / nthreads;
        jobs[t].s1 = count * (t + 1) / nthreads;
        jobs[t].pe_form = pe_form;
        jobs[t].dW_out = dW_out;
        jobs[t].traj_out = traj_out;
        jobs[t].S1 = want_moments ? S1 + (int64_t)t * cols : NULL;
        jobs[t].S2 = want_moments ? S2 + (int64_t)t * cols : NULL;
        jobs[t].rrf_out = rrf;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, sim_worker, &jobs[t]);
    sim_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    if (want_moments) {
        for (int64_t c = 0; c < cols; ++c) {
            double s1 = 0.0, s2 = 0.0;
            for (int t = 0; t < nthreads; ++t) { s1 += S1[(int64_t)t * cols + c]; s2 += S2[(int64_t)t * cols + c]; }
            double Nn = (double)count;
            if (mean) mean[c] = shift[c] + s1 / Nn;
            if (var) var[c] = (count > 1) ? (s2 - s1 * s1 / Nn) / (Nn - 1.0) : NAN;
        }
        free(shift); free(S1); free(S2);
    }
    free(th); free(jobs); free(phi); free(mdot); free(delta0); free(pm_eq);
    return 0;
}

/* Algorithm 1 step 4 on stored values: two-pass mean and unbiased variance of
 * x[N][C] over the N rows, column by column.                                  */
void oracle_moments_twopass(const double* x, int64_t N, int64_t C, double* mean, double* var)
{
    for (int64_t c = 0; c < C; ++c) {
        double s = 0.0;
        for (int64_t r = 0; r < N; ++r) s += x[r * C + c];
        double m = s / (double)N;
        double ss = 0.0;
        for (int64_t r = 0; r < N; ++r) {
            double e = x[r * C + c] - m;
            ss += e * e;
        }
        mean[c] = m;
        var[c] = (N > 1) ? ss / (double)(N - 1) : NAN;
    }
}
