// Initial equilibrium (Section V-A: the system is at equilibrium at t = 0),
// FP64 on the GPU: Newton's method on Pm_i - Pe_i(delta) = 0 from a flat start.
// Pe and its Jacobian use the product form
//   Pe_i = a_i u_i + b_i v_i,  a = E cos delta, b = E sin delta,
//   u = G a - B b, v = G b + B a  (+ Vinf (Ginf_i a_i + Binf_i b_i)),
//   dPe_i/d delta_j = G_ij (b_i a_j - a_i b_j) - B_ij (a_i a_j + b_i b_j)   (j != i)
//   dPe_i/d delta_i = a_i v_i - b_i u_i - B_ii (a_i^2 + b_i^2) + Vinf (Binf_i a_i - Ginf_i b_i).
// With an infinite bus every angle is unknown; otherwise delta_0 = 0 is the
// reference and machine 0 takes the power balance Pe_0(delta) as its Pm.
// One CTA; thread i owns machine i; the linear solve is Gaussian elimination
// with partial pivoting in shared memory.
#include "fmc_common.cuh"
#include "kernels.cuh"

namespace fmc {

constexpr int EQ_MAX = 64;

struct EqArgs {
    int n;
    int has_inf;
    double Vinf;
    const double* G;
    const double* B;
    const double* Ginf;
    const double* Binf;
    const double* E;
    const double* Pm;
};

// out: [0, n) delta0, [n, 2n) pm_eq, [2n, 4n) moment shift (delta0, then zeros),
// status[0] = iterations (>= 0) or -1 when Newton did not converge.
__global__ void __launch_bounds__(EQ_MAX) equilibrium_kernel(EqArgs a, double* __restrict__ out, int* __restrict__ status)
{
    __shared__ double delta[EQ_MAX], av[EQ_MAX], bv[EQ_MAX], F[EQ_MAX], J[EQ_MAX][EQ_MAX + 1];
    __shared__ double pe[EQ_MAX];
    __shared__ int piv_row;
    __shared__ int done;
    const int n = a.n;
    const int i = threadIdx.x;
    const int first = a.has_inf ? 0 : 1;
    const int m = n - first;
    if (i < n) delta[i] = 0.0;
    if (i == 0) done = (m == 0);
    __syncthreads();
    int it = 0;
    for (it = 0; it < 100 && !done; ++it) {
        if (i < n) {
            double s, c;
            sincos(delta[i], &s, &c);
            av[i] = a.E[i] * c;
            bv[i] = a.E[i] * s;
        }
        __syncthreads();
        if (i < n) {
            double u = 0.0, v = 0.0;
            for (int j = 0; j < n; ++j) {
                u += a.G[i * n + j] * av[j] - a.B[i * n + j] * bv[j];
                v += a.G[i * n + j] * bv[j] + a.B[i * n + j] * av[j];
            }
            double p = av[i] * u + bv[i] * v;
            double dii = av[i] * v - bv[i] * u - a.B[i * n + i] * (av[i] * av[i] + bv[i] * bv[i]);
            if (a.has_inf) {
                p += a.Vinf * (a.Ginf[i] * av[i] + a.Binf[i] * bv[i]);
                dii += a.Vinf * (a.Binf[i] * av[i] - a.Ginf[i] * bv[i]);
            }
            pe[i] = p;
            if (i >= first) {
                int r = i - first;
                F[r] = a.Pm[i] - p;
                for (int j = first; j < n; ++j) {
                    double v2 = (j == i) ? dii
                                         : a.G[i * n + j] * (bv[i] * av[j] - av[i] * bv[j]) -
                                               a.B[i * n + j] * (av[i] * av[j] + bv[i] * bv[j]);
                    J[r][j - first] = v2;
                }
            }
        }
        __syncthreads();
        if (i == 0) {
            double fmax = 0.0;
            for (int r = 0; r < m; ++r) fmax = fmax > fabs(F[r]) ? fmax : fabs(F[r]);
            done = (fmax < 1e-13);
        }
        __syncthreads();
        if (done) break;
        // J x = F by Gaussian elimination with partial pivoting
        for (int col = 0; col < m; ++col) {
            if (i == 0) {
                int p = col;
                for (int r = col + 1; r < m; ++r)
                    if (fabs(J[r][col]) > fabs(J[p][col])) p = r;
                piv_row = p;
            }
            __syncthreads();
            int p = piv_row;
            if (p != col) {
                for (int j = i; j < m; j += blockDim.x) {
                    double t = J[col][j];
                    J[col][j] = J[p][j];
                    J[p][j] = t;
                }
                if (i == 0) {
                    double t = F[col];
                    F[col] = F[p];
                    F[p] = t;
                }
            }
            __syncthreads();
            int r = col + 1 + i;
            double piv = J[col][col];
            if (r < m && piv != 0.0) {
                double f = J[r][col] / piv;
                for (int j = col; j < m; ++j) J[r][j] -= f * J[col][j];
                F[r] -= f * F[col];
            }
            __syncthreads();
        }
        if (i == 0) {
            for (int r = m - 1; r >= 0; --r) {
                double acc = F[r];
                for (int j = r + 1; j < m; ++j) acc -= J[r][j] * F[j];
                F[r] = (J[r][r] != 0.0) ? acc / J[r][r] : 0.0;
            }
        }
        __syncthreads();
        if (i >= first && i < n) delta[i] += F[i - first];
        __syncthreads();
    }
    // balance of the reference machine at the solution
    if (i < n) {
        double s, c;
        sincos(delta[i], &s, &c);
        av[i] = a.E[i] * c;
        bv[i] = a.E[i] * s;
    }
    __syncthreads();
    if (i < n) {
        double u = 0.0, v = 0.0;
        for (int j = 0; j < n; ++j) {
            u += a.G[i * n + j] * av[j] - a.B[i * n + j] * bv[j];
            v += a.G[i * n + j] * bv[j] + a.B[i * n + j] * av[j];
        }
        double p = av[i] * u + bv[i] * v;
        if (a.has_inf) p += a.Vinf * (a.Ginf[i] * av[i] + a.Binf[i] * bv[i]);
        out[i] = delta[i];
        out[n + i] = (i < first) ? p : a.Pm[i];
        out[2 * n + i] = delta[i];
        out[3 * n + i] = 0.0;
    }
    if (i == 0) status[0] = done ? it : -1;
}

cudaError_t launch_equilibrium(int n, int has_inf, double Vinf, const double* G, const double* B, const double* Ginf,
                               const double* Binf, const double* E, const double* Pm, double* out, int* status,
                               cudaStream_t st)
{
    if (n < 1 || n > EQ_MAX) return cudaErrorInvalidValue;
    EqArgs a{n, has_inf, Vinf, G, B, Ginf, Binf, E, Pm};
    equilibrium_kernel<<<1, EQ_MAX, 0, st>>>(a, out, status);
    return cudaGetLastError();
}

}  // namespace fmc
