/*
 * fastmc.h -- C ABI of the GB300 (sm_103a) implementation of the fast Monte
 * Carlo method of Qiu, Lin, Chen, Liu and Song, "Fast Monte Carlo Simulation of
 * Dynamic Power Systems Under Continuous Random Disturbances" (arXiv 2007.03847).
 *
 * The method (Algorithm 1, Section IV-C): the disturbance is an Ito process
 * (Eq. ito) driven by Wiener processes; each Wiener process is replaced by its
 * truncated Karhunen-Loeve expansion in K independent standard normals
 * (Eqs. kl, kle, eqkl); the M = d*K normals are drawn by Latin hypercube
 * sampling (Section IV-B); every sample's disturbance path drives a dynamic
 * simulation of the power system (Eqs. state, algebra); the expectation and
 * variance of the response are taken over the samples.
 *
 * This library computes that path on one GPU:
 *   fmc_lhs_sample, fmc_lhs_sample_split  -- Algorithm 1 step 1
 *   fmc_kl_basis, fmc_kle_reconstruct     -- Algorithm 1 step 2
 *   fmc_equilibrium                       -- the initial equilibrium (Section V-A)
 *   fmc_simulate                          -- Algorithm 1 steps 1-4 fused
 *   fmc_moments                           -- Algorithm 1 step 4 on given values
 *
 * Conventions for every entry point:
 *   - Return value: FMC_OK (0) or a positive FMC_E* code; fmc_last_error(ctx)
 *     then describes the failure.  No C++ exception crosses this boundary.
 *   - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *     library never frees them.  Host pointers are read during the call only.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     enqueued on it and the call returns without waiting, unless stated.
 *   - All arrays are dense row-major with the shapes given.
 *   - A context is not thread-safe: use one context per host thread.
 */
#ifndef FASTMC_H
#define FASTMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define FMC_OK 0
#define FMC_EINVAL 1        /* invalid argument (message in fmc_last_error) */
#define FMC_ENOMEM 2        /* device allocation failed or over budget */
#define FMC_ECUDA 3         /* a CUDA runtime/driver call failed */
#define FMC_ETIMEOUT 4      /* a bounded device-side wait gave up */
#define FMC_NOT_READY 5     /* asynchronous result not available yet */
#define FMC_EBUSY 6         /* resource in use */
#define FMC_ECANCELLED 7    /* request cancelled */
#define FMC_EUNSUPPORTED 8  /* valid request outside what the library handles */
#define FMC_ENOCONVERGE 9   /* equilibrium Newton iteration did not converge */

/* ---- sampling modes (Section IV-B) ---------------------------------------- */
#define FMC_LHS 0           /* Latin hypercube: stratum pi_i(k), uniform inside */
#define FMC_SRS 1           /* simple random sampling: p = u */
#define FMC_LHS_MIDPOINT 2  /* Latin hypercube at the stratum midpoint */
#define FMC_SRS_EM 3        /* the paper's traditional Monte Carlo (Section V-B): a fresh normal per
                               step and disturbance, dW = sqrt(dt) Phi^-1(u) with u from Philox
                               counter (k, n, 256, w/4) word w mod 4 -- Eq. (distito); no KL
                               expansion, K and the precision are not used */

/* ---- contraction precision of the KL reconstruction ------------------------- */
#define FMC_PREC_F32 0      /* FP32 SIMT (the plain form) */
#define FMC_PREC_BF16 1     /* BF16 operands on tcgen05 tensor cores, FP32 accumulate */
#define FMC_PREC_BF16X3 2   /* split BF16 hi+lo, three tcgen05 products: FP32-level accuracy */

/* ---- integrators for the swing equations --------------------------------- */
#define FMC_RK4 0
#define FMC_HEUN 1

/* ---- KL bases ------------------------------------------------------------ */
#define FMC_BASIS_SINE 0    /* eigenbasis of min(s,t): the Karhunen-Loeve expansion of W */
#define FMC_BASIS_COSINE 1  /* the paper's Eq. (klb2): constant + cosine white-noise modes */

/* ---- simulation paths --------------------------------------------------- */
#define FMC_PATH_FUSED 0    /* one kernel: contraction in TMEM -> integrator -> moment partials */
#define FMC_PATH_PLAIN 1    /* unfused FP32: increments and trajectories through HBM */

/* ---- limits of the library ------------------------------------------------ */
#define FMC_MAX_MACHINES 52        /* fused path (17..52 machines: four warps per sample) */
#define FMC_MAX_MACHINES_PLAIN 16  /* plain FP32 path */
#define FMC_MAX_DISTURBANCES 8

typedef struct fmc_ctx fmc_ctx;

/*
 * One uncertainty-evaluation problem.
 *
 * System: the Kron-reduced classical model of n machines (Eqs. state/algebra
 * reduced to the swing equations),
 *   d delta_i / dt  = omega_s * domega_i
 *   2 H_i d domega_i / dt = Pm_i + sum_w inject[i][w] x_w - Pe_i(delta) - D_i domega_i
 *   Pe_i = sum_j E_i E_j (G_ij cos(delta_i - delta_j) + B_ij sin(delta_i - delta_j))
 *          + E_i Vinf (Ginf_i cos delta_i + Binf_i sin delta_i)   [if has_inf_bus]
 * Disturbances: d Ornstein-Uhlenbeck processes dx_w = -theta_w x_w dt +
 * sigma_w dW_w (Eq. ito with Table I's Gaussian drift at rate theta_w),
 * advanced by Euler-Maruyama (Eq. distito) on the grid t_n = n dt, n < Nt,
 * T = Nt dt.  Each W_w is its K-term KL expansion with the Brownian eigenbasis
 *   W(t) = sum_k zeta_k sqrt(2T)/((k-1/2) pi) sin((k-1/2) pi t / T).
 * Sampling: N samples of the M = d*K coefficients, seeded by `seed`.
 * Initial state: the equilibrium (Section V-A) found by Newton's method; without
 * an infinite bus machine 0 is the angle reference and balances the power
 * (its Pm is replaced by the balance).
 * All arrays are host memory, read during the call.
 */
/*
 * A general one-dimensional Ito disturbance (Section II, Table I; the wind model
 * of Eq. windito):  d xi = mu(xi) dt + sigma(xi) dW,  xi(0) = x0,
 *   mu(x) = m[0] + m[1] x + m[2] x^2,
 *   kind FMC_ITO_POLY: sigma(x)   = s[0] + s[1] x + s[2] x^2,
 *   kind FMC_ITO_SQRT: sigma(x)^2 = v[0] + v[1] x + v[2] x^2 + v[3] |x - a|  (sigma = 0 where negative),
 *   kind FMC_ITO_OU:   the scenario's theta/sigma (mu = -theta x, sigma const, x0 = 0).
 * The system is at equilibrium with the disturbance at x0 (the power balance sees
 * inject * (xi - x0)).  Advanced by the scheme of Eq. (distito); with KL paths
 * (smooth, so converging to the Stratonovich solution) the drift carries
 * -sigma sigma'/2 so that the limit is the Ito process; with per-step normals
 * (FMC_SRS_EM) it does not.
 */
#define FMC_ITO_OU 0
#define FMC_ITO_POLY 1
#define FMC_ITO_SQRT 2
typedef struct fmc_ito {
    int32_t kind;
    int32_t reserved;
    double m[3];
    double s[3];
    double v[4];
    double a;
    double x0;
} fmc_ito;

#define FMC_FORCING_INCREMENTS 0
#define FMC_FORCING_SMOOTH 1

typedef struct fmc_scenario {
    int32_t n;              /* machines, 1..FMC_MAX_MACHINES (FMC_MAX_MACHINES_PLAIN on the plain path) */
    int32_t d;              /* disturbances = Wiener processes, 1..FMC_MAX_DISTURBANCES */
    int32_t K;              /* KL terms per Wiener process, >= 1 */
    int32_t sampling;       /* FMC_LHS, FMC_SRS or FMC_LHS_MIDPOINT */
    double T;               /* horizon, s; T/dt must be an integer to 1e-9 relative */
    double dt;              /* step, s */
    int64_t N;              /* samples, 1..2^31 */
    uint64_t seed;          /* Philox key of the design */
    int32_t precision;      /* FMC_PREC_* of the KL contraction */
    int32_t integrator;     /* FMC_RK4 or FMC_HEUN */
    int32_t has_inf_bus;    /* 0 or 1 */
    int32_t basis;          /* FMC_BASIS_SINE (default) or FMC_BASIS_COSINE */
    double omega_s;         /* synchronous speed, rad/s */
    double Vinf;            /* infinite-bus voltage */
    const double* G;        /* [n][n] conductance */
    const double* B;        /* [n][n] susceptance */
    const double* Ginf;     /* [n] or NULL without infinite bus */
    const double* Binf;     /* [n] or NULL without infinite bus */
    const double* H;        /* [n] inertia constants, s, > 0 */
    const double* D;        /* [n] damping */
    const double* E;        /* [n] internal EMF magnitudes */
    const double* Pm;       /* [n] mechanical powers */
    const double* theta;    /* [d] OU rates, 1/s */
    const double* sigma;    /* [d] OU diffusion coefficients */
    const double* inject;   /* [n][d] weight of disturbance w in machine i's power balance */
    /* An event in the style of the paper's generator trip (Section V-A): from grid
     * step round(event_time/dt) on, machine event_machine's mechanical power
     * changes by event_dpm p.u. (negative: generation lost), for whole steps.
     * event_machine < 0: none.  It takes a disturbance slot: d <= 7 with an event. */
    int32_t event_machine;
    /* How the KL path drives the disturbances: FMC_FORCING_INCREMENTS (default):
     * Euler-Maruyama (Eq. distito) on the path's increments over each step;
     * FMC_FORCING_SMOOTH: the random ODE of Eq. (eqkl), dx/dt = mu(x) +
     * sigma(x) sum_k zeta_k m_k(t) (m_k the time derivative of the KL basis
     * function; a general disturbance with the Stratonovich drift), stepped by
     * the same RK4/Heun stages as the swing equations.  The smooth form runs on
     * the plain path and on the per-sample fused kernel (up to 16 machines; the
     * forcing at the half steps is contracted on the tensor cores, and a chunk
     * takes two TMEM columns per step and disturbance); FMC_EUNSUPPORTED on the
     * large-system kernel, FMC_EINVAL with FMC_SRS_EM. */
    int32_t forcing;
    double event_time;      /* s */
    double event_dpm;       /* p.u. */
    const fmc_ito* ito;     /* [d] disturbance models, or NULL: all Ornstein-Uhlenbeck (theta, sigma) */
    /* Section IV-B step 2: FMC_CORR_NONE (default): the random permutations of the
     * design as they are; FMC_CORR_RANK: the permutation that minimises the
     * correlation between the design's columns (see fmc_lhs_decorrelate).  Needs
     * an LHS sampling mode and N > d K; the whole N-sample design is formed on
     * every call, also when a call simulates a block of it. */
    int32_t correlation;
    int32_t reserved;
} fmc_scenario;

#define FMC_CORR_NONE 0
#define FMC_CORR_RANK 1

/* ---- context ------------------------------------------------------------- */

/* Creates a context on CUDA device `device` (made current for the calling
 * thread).  `mem_budget_bytes` caps the library's own device workspace
 * (0 = no cap).  Returns FMC_OK and *out, or an error code. */
int fmc_create(fmc_ctx** out, int device, size_t mem_budget_bytes);

/* Synchronises the context's work, frees its workspace and the context. */
int fmc_destroy(fmc_ctx* ctx);

/* Message of the last failure on this context ("" if none).  Valid until the
 * next call on the context.  Accepts NULL (returns the message of the last
 * failed fmc_create on this thread). */
const char* fmc_last_error(const fmc_ctx* ctx);

/* Number of SMs and the device name of the context's GPU. */
int fmc_device_info(const fmc_ctx* ctx, int* sm_count, char* name, size_t name_len);

/* ---- Algorithm 1 step 1: Latin hypercube sampling (Section IV-B) ------------ */

/*
 * Rows k0 .. k0+count-1 of the N-sample design over M standard normal
 * coefficients.  For dimension i and sample k: stratum s = pi_i(k), where pi_i
 * is a keyed Feistel bijection of {0..N-1} (six rounds on 2h bits,
 * h = max(1, ceil(log2(N)/2)), round function Philox4x32-10 word 0 with
 * counter (R, i, 1 + round, 0), key = seed, restricted to [0, N) by cycle
 * walking); u = (r + 1/2) 2^-32 with r = Philox4x32-10(counter (k, i, 0, 0),
 * key = seed) word 0; p = (s + u)/N (LHS), (s + 1/2)/N (LHS_MIDPOINT) or u
 * (SRS); zeta = Phi^-1(p) in FP32.
 *   zeta_dev   [count][M] float, or NULL
 *   strata_dev [M][count] uint32 (s; k for SRS), or NULL
 * Errors: FMC_EINVAL if N < 1, N > 2^31, M < 1, k0 < 0, count < 0,
 * k0 + count > N, or both outputs NULL.
 */
int fmc_lhs_sample(fmc_ctx* ctx, uint64_t seed, int64_t N, int64_t k0, int64_t count, int32_t M,
                   int32_t mode, float* zeta_dev, uint32_t* strata_dev, void* stream);

/*
 * The same design written as split BF16 for the tensor-core contraction: the
 * M = d*K coefficients of a row are laid out as d groups of K_s =
 * round_up(K, 8) entries (entries K..K_s-1 are zero):
 *   hi_dev [count][d][K_s] bf16 (as uint16 bit patterns) = bf16(zeta)
 *   lo_dev [count][d][K_s] bf16 = bf16(zeta - hi), or NULL
 * Errors as fmc_lhs_sample; d or K < 1.
 */
int fmc_lhs_sample_split(fmc_ctx* ctx, uint64_t seed, int64_t N, int64_t k0, int64_t count, int32_t d,
                         int32_t K, int32_t mode, uint16_t* hi_dev, uint16_t* lo_dev, void* stream);

/* ---- Algorithm 1 step 2: KL reconstruction (Eqs. kl, kle, eqkl) --------------- */

/*
 * Increment basis of the truncated KL expansion on the grid t_n = n T/Nt,
 * k = 0..K-1 (0-based):
 *   FMC_BASIS_SINE   (Brownian eigenbasis): phi[k][n] = c_k (sin(a_k t_{n+1}) - sin(a_k t_n)),
 *                    a_k = (k+1/2) pi / T, c_k = sqrt(2T)/((k+1/2) pi);
 *   FMC_BASIS_COSINE (Eq. klb2, integrated): phi[0][n] = dt/sqrt(T), and for k >= 1
 *                    c_k (sin(a_k t_{n+1}) - sin(a_k t_n)), a_k = k pi / T, c_k = sqrt(2T)/(k pi).
 * Computed in FP64 on the GPU and rounded:  phi_dev [K][Nt] float.
 * Errors: FMC_EINVAL if K < 1, Nt < 1, T <= 0 or an unknown basis.
 */
int fmc_kl_basis(fmc_ctx* ctx, int32_t K, double T, int32_t Nt, int32_t basis, float* phi_dev, void* stream);

/*
 * Section IV-B step 2: the permutation of the N x M Latin hypercube design of
 * fmc_lhs_sample that minimises the correlation between its columns.  The
 * paper points to a Cholesky-based method without giving it; this is the rank
 * method of Iman and Conover (1982) with the identity as target correlation:
 * van der Waerden scores a(s) = Phi^-1((s + 1)/(N + 1)) paired by the design's
 * own permutations form R[k][i] = a(pi_i(k)); with corr(R) = Q Q^T (Cholesky),
 * R* = R Q^-T has uncorrelated columns, and sample k of dimension i takes as
 * its new stratum the rank of R*[k][i] in column i (ascending, ties by sample
 * index), keeping its own uniform inside the stratum.  Every stratum is still
 * hit once per dimension; the first dimension keeps its permutation.
 *   mode       FMC_LHS or FMC_LHS_MIDPOINT
 *   zeta_dev   [N][M] float (device), or NULL
 *   strata_dev [M][N] uint32 (device), or NULL: the new strata
 * Limits: 2 <= N, M < N, M <= 4096, N*M < 2^31.  Synchronises `stream` (the
 * call reads back whether the score correlation factorised).  Uses library
 * workspace (about 4 N M * 4 bytes).  Errors: FMC_EINVAL (sizes, mode, or a
 * score correlation that is not positive definite), FMC_ENOMEM, FMC_ECUDA.
 */
int fmc_lhs_decorrelate(fmc_ctx* ctx, uint64_t seed, int64_t N, int32_t M, int32_t mode, float* zeta_dev,
                        uint32_t* strata_dev, void* stream);

/*
 * Appendix (Eqs. likelihood, like, reprob, ident): identification of a scalar
 * Ito model dxi = mu(xi) dt + sigma(xi) dW from a record xi_dev [n] (device,
 * double) sampled every h seconds, by minimising
 *   L'(q) = 1/4 sum_j (dxi_j - h mu_j)^2 / D_j + 1/2 sum_j log D_j,
 *   D_j = h sigma(xi_j)^2 / 2,  dxi_j = xi_{j+1} - xi_j,
 * the negative log-likelihood of the Euler-Maruyama transition densities less
 * its constant.  Model (q[6], host): mu(x) = q0 + q1 x + q2 x^2 and
 *   kind FMC_IDENT_SIGMA:   sigma(x)   = q3 + q4 x + q5 x^2 (the form of Eq. windito),
 *   kind FMC_IDENT_SIGMA2:  sigma(x)^2 = q3 + q4 x + q5 x^2 (the forms of Table I).
 * fmc_ito_objective: L' (host *L; +infinity where some D_j <= 0) and, if grad /
 * hess are not NULL, its gradient [6] and Hessian [6][6] (host), summed on the
 * GPU in FP64.  fmc_ito_identify: Newton's method from q (overwritten by the
 * estimate) with the Hessian shifted by lambda I until positive definite and a
 * backtracking line search, until the step is below 1e-12 relative or the
 * predicted decrease g^T H^-1 g below 1e-12 max(1, |L'|) (the rounding of the
 * sums); *iterations (nullable) receives the count.  Both
 * synchronise `stream`.  Errors: FMC_EINVAL (kind, n < 8, h <= 0, a start with
 * some D_j <= 0), FMC_ENOCONVERGE (200 iterations or a failed line search).
 */
#define FMC_IDENT_SIGMA 1
#define FMC_IDENT_SIGMA2 2
int fmc_ito_objective(fmc_ctx* ctx, int32_t kind, const double* q, const double* xi_dev, int64_t n, double h,
                      double* L, double* grad, double* hess, void* stream);
int fmc_ito_identify(fmc_ctx* ctx, int32_t kind, const double* xi_dev, int64_t n, double h, double* q,
                     int32_t* iterations, void* stream);

/*
 * Increments of the reconstructed Wiener paths of `count` samples:
 *   dW[s][w][n] = sum_k zeta[s][w*K + k] phi[k][n],   T = Nt dt.
 *   zeta_dev [count][d*K] float (as written by fmc_lhs_sample)
 *   dW_dev   [count][d][Nt] float
 * precision: FMC_PREC_F32 (FP32 SIMT), FMC_PREC_BF16 or FMC_PREC_BF16X3
 * (tcgen05 tensor cores; zeta and phi split to BF16 inside the call, using
 * library workspace).
 * Errors: FMC_EINVAL on sizes < 1 or T/dt not an integer; FMC_ENOMEM.
 */
int fmc_kle_reconstruct(fmc_ctx* ctx, const float* zeta_dev, int64_t count, int32_t d, int32_t K, double T,
                        double dt, int32_t precision, float* dW_dev, void* stream);

/*
 * Allocation-free form of fmc_kle_reconstruct (the paper has no counterpart:
 * this is a service to callers that cannot allocate device memory).
 *
 * Some callers cannot call cudaMalloc: a process that has reserved the GPU's
 * memory for its own pool (so a fresh allocation would fail or fragment it), or
 * a loop with a hard latency budget (cudaMalloc and cudaFree may synchronise the
 * device).  This entry point allocates nothing.  Its working memory -- the split
 * BF16 coefficients and basis and an error word (or the FP32 basis) -- is a
 * fixed device array of FMC_NOALLOC_SCRATCH_BYTES bytes inside the library,
 * present on every GPU that loads the library until the process exits.  The
 * caller still passes the inputs and the output, with the same meaning, layout
 * and results as fmc_kle_reconstruct.
 *
 * Limits and behaviour:
 *   - A call needs 256 + 2*align256(count*d*round_up(K,8)*2) + 2*align256(Nt*round_up(K,32)*2)
 *     bytes (BF16/BF16X3) or 256 + align256(K*Nt*4) bytes (F32); a larger call
 *     returns FMC_EINVAL and says so in fmc_last_error.
 *   - The caller's current device must be the context's device (FMC_EINVAL
 *     otherwise): the kernels run on the current device and address its array.
 *   - The first call on a device looks up the array's device address with that
 *     device current; make that first call before any stream capture.
 *   - The array's first 256 bytes hold the call's device error word, cleared at
 *     the start of every call.  fmc_device_status reads it (after synchronising
 *     the device): FMC_ETIMEOUT if a bounded wait of the contraction gave up, in
 *     which case dW is not valid.  It reports the last call on the device.
 *   - All calls share the one array and it keeps the last call's contents: calls
 *     whose work overlaps on the GPU (different streams, or different host
 *     threads) race.  Serialise them on one stream.
 */
#define FMC_NOALLOC_SCRATCH_BYTES (16u << 20)
int fmc_kle_reconstruct_noalloc(fmc_ctx* ctx, const float* zeta_dev, int64_t count, int32_t d, int32_t K, double T,
                                double dt, int32_t precision, float* dW_dev, void* stream);

/* ---- equilibrium (Section V-A: "at equilibrium at t = 0") --------------------- */

/*
 * Newton's method in FP64 on the GPU for Pm_i = Pe_i(delta) from a flat start.
 * Writes delta0[n] and the balanced mechanical powers pm_eq[n] (host memory).
 * Synchronous.  Errors: FMC_EINVAL (scenario), FMC_ENOCONVERGE.
 */
int fmc_equilibrium(fmc_ctx* ctx, const fmc_scenario* scen, double* delta0, double* pm_eq);

/* ---- Algorithm 1 steps 1-4 ---------------------------------------------------- */

/*
 * Runs the whole path for one scenario: LHS -> KL reconstruction -> EM for the
 * OU disturbances -> integration of the swing equations for every sample ->
 * mean and unbiased variance (N-1; NaN for N = 1) over the N samples at every
 * grid time t_n, n = 0..Nt, for every state (delta_0..delta_{n-1},
 * domega_0..domega_{n-1}).
 *   mean_dev, var_dev [Nt+1][2n] double (device)
 *   traj_dev  [N][Nt+1][2n] float, or NULL: every sample's trajectory (for
 *             testing; N*(Nt+1)*2n*4 bytes)
 *   path      FMC_PATH_FUSED or FMC_PATH_PLAIN (FMC_PATH_PLAIN needs
 *             precision FMC_PREC_F32; FMC_PATH_FUSED needs BF16 or BF16X3)
 * The FP64 equilibrium is solved on the GPU first; the call then waits for the
 * stream once (to read the equilibrium angles, from which the integrator's
 * constants are formed) and enqueues the rest without waiting.
 * Errors: FMC_EINVAL, FMC_EUNSUPPORTED (n or d above the library's limits),
 * FMC_ENOMEM, FMC_ENOCONVERGE, FMC_ETIMEOUT (a bounded device wait gave up),
 * FMC_ECUDA.
 */
int fmc_simulate(fmc_ctx* ctx, const fmc_scenario* scen, int32_t path, double* mean_dev, double* var_dev,
                 float* traj_dev, void* stream);

/*
 * The same path for the block of samples k0 .. k0+count-1 of the N-sample
 * design (so that blocks on different GPUs form one design), returning the
 * per-time sums of shifted states instead of moments:
 *   S1_dev, S2_dev [Nt+1][2n] double: sum (x - c), sum (x - c)^2 over the block,
 *   shift_dev [2n] double: c (the equilibrium angles, then zeros; the sums use
 *   its FP32 rounding).  Sums of blocks add; fmc_moments_from_sums finishes.
 * Errors as fmc_simulate; FMC_EINVAL if the block is outside [0, N).
 */
int fmc_simulate_sums(fmc_ctx* ctx, const fmc_scenario* scen, int64_t k0, int64_t count, int32_t path,
                      double* S1_dev, double* S2_dev, double* shift_dev, float* traj_dev, void* stream);

/* ---- many scenarios ------------------------------------------------------- */

/*
 * A batch of independent scenarios of uneven size (machines, disturbances, K,
 * horizon, N), run concurrently on the GPU: every scenario's kernels go to one
 * of up to 16 library streams in turn, forked from and joined back to the
 * caller's stream, so that the CTAs of different scenarios share the SMs.
 * fmc_batch_create copies and checks every scenario (the caller's arrays may go
 * away afterwards), solves every equilibrium (waiting for the device), reserves
 * each scenario's workspace and, with use_graph = 1,
 * captures the whole batch into one CUDA graph; fmc_batch_launch then replays
 * it with a single graph launch on `stream` (or enqueues the kernels again
 * without a graph).  Results: mean_dev[i], var_dev[i] [Nt_i+1][2 n_i] double
 * (device, caller-owned, fixed at creation).  The fused path adds each
 * scenario's per-time sums with FP64 atomics (sums of FP32 partials over
 * 32-sample groups; summation order not fixed).
 */
typedef struct fmc_batch fmc_batch;
int fmc_batch_create(fmc_ctx* ctx, const fmc_scenario* scen, int32_t n_scen, int32_t path, double* const* mean_dev,
                     double* const* var_dev, int32_t use_graph, fmc_batch** out);
int fmc_batch_launch(fmc_batch* batch, void* stream);
int fmc_batch_destroy(fmc_batch* batch);

/* create + launch (without a graph) + wait + destroy. */
int fmc_simulate_batch(fmc_ctx* ctx, const fmc_scenario* scen, int32_t n_scen, int32_t path,
                       double* const* mean_dev, double* const* var_dev, void* stream);

/* ---- serving -------------------------------------------------------------- */

/*
 * A request server: requests (one scenario each, results to caller-owned
 * device buffers) wait in a FIFO queue and are admitted, head first, as soon as
 * one of `slots` worker slots is free and the request's device workspace fits
 * in what is left of the memory budget (0: 80% of the free device memory).
 * Each slot has its own stream, library context and workspace, so requests that
 * arrive while others run start at once and their kernels share the GPU.  The
 * fused path sums moments with FP64 atomics (no per-tile partial buffers).
 *   fmc_submit   queues a request (the scenario is copied); FMC_ENOMEM if it
 *                could never fit the budget.
 *   fmc_poll     non-blocking: FMC_NOT_READY, or FMC_OK and *out (once).
 *   fmc_wait     blocks up to timeout_us: FMC_ETIMEOUT, or FMC_OK and *out.
 *   fmc_cancel   removes a queued request (its result reports FMC_ECANCELLED);
 *                FMC_EBUSY if it is already running.
 * The server is thread-safe; results are reported once.
 */
typedef struct fmc_server fmc_server;
typedef struct fmc_result {
    int32_t status;         /* FMC_OK or the request's error code */
    int32_t replicates;     /* independent designs behind the moments (1 without a target) */
    double latency_us;      /* submit -> results complete on the device */
    double queue_us;        /* submit -> admitted */
    uint64_t device_bytes;  /* workspace charged against the budget */
    int64_t n_used;         /* samples simulated for the reported moments */
    double err_E;           /* estimated error of the expectations (targets only, else -1) */
    double err_Var;         /* estimated error of the variances (targets only, else -1) */
    int32_t target_met;     /* 1 if both targets were reached (targets only) */
    int32_t reserved;
    char message[256];      /* error text, "" on success */
} fmc_result;
int fmc_server_create(int device, int32_t slots, size_t mem_budget_bytes, fmc_server** out);
int fmc_server_destroy(fmc_server* srv);
int fmc_submit(fmc_server* srv, const fmc_scenario* scen, int32_t path, double* mean_dev, double* var_dev,
               uint64_t* handle);
/*
 * A request with a target error instead of a sample count.  The server runs
 * R = 4 independent Latin hypercube designs (seeds derived from the scenario's)
 * of n samples each, starting at n = scen->N, and estimates the error of the
 * pooled moments from the spread of the replicates:
 *   err_E   = max_{t,s} sd_r(E_r) / sqrt(R) / max_{t,s} sqrt(Var),
 *   err_Var = max_{t,s} sd_r(Var_r) / sqrt(R) / max_{t,s} Var
 * (the normalisation of the error the convergence study reports).  While a
 * target (> 0) is missed and 4 R n <= max_N, n grows fourfold and the designs
 * are drawn again.  The result holds the pooled moments (replicate averages) of
 * the last round, n_used = R n, the error estimates and target_met.  Only
 * Latin hypercube and simple random sampling take targets.
 */
int fmc_submit_target(fmc_server* srv, const fmc_scenario* scen, int32_t path, double tol_E, double tol_Var,
                      int64_t max_N, double* mean_dev, double* var_dev, uint64_t* handle);
int fmc_poll(fmc_server* srv, uint64_t handle, fmc_result* out);
int fmc_wait(fmc_server* srv, uint64_t handle, int64_t timeout_us, fmc_result* out);
int fmc_cancel(fmc_server* srv, uint64_t handle);
int fmc_server_stats(fmc_server* srv, int32_t* queued, int32_t* running, size_t* bytes_in_use);

/*
 * The paper's response function (Section V-B), per sample: the RMS over the
 * horizon of the system frequency deviation, taken as the centre-of-inertia
 * speed deviation omega_coi = sum_i H_i domega_i / sum_i H_i on the grid,
 *   RRF = sqrt( (1/Nt) sum_{n=1..Nt} omega_coi(t_n)^2 )   (p.u.),
 * and its expectation and unbiased variance over the N samples:
 *   rrf_dev [2] FP64 (device): E[RRF], Var[RRF].
 * Runs the whole scenario like fmc_simulate; mean_dev / var_dev [Nt+1][2n]
 * receive the moment trajectories too, or may be NULL.
 */
int fmc_simulate_rrf(fmc_ctx* ctx, const fmc_scenario* scen, int32_t path, double* rrf_dev, double* mean_dev,
                     double* var_dev, void* stream);

/* ---- Algorithm 1 step 4 --------------------------------------------------- */

/*
 * Moments from shifted sums over N samples (see fmc_simulate_sums):
 *   mean = c + S1/N, var = (S2 - S1^2/N)/(N - 1) (NaN for N = 1), c = FP32(shift).
 *   S1_dev, S2_dev, mean_dev, var_dev [rows][S] double; shift_dev [S] double.
 * mean_dev/var_dev may alias S1_dev/S2_dev.
 */
int fmc_moments_from_sums(fmc_ctx* ctx, const double* S1_dev, const double* S2_dev, const double* shift_dev,
                          int64_t N, int64_t rows, int32_t S, double* mean_dev, double* var_dev, void* stream);


/*
 * Column-wise mean and unbiased variance of x[N][C] over its N rows, combined
 * in FP64 from FP32 shifted partial sums (shift = row 0).
 *   x_dev [N][C] float; mean_dev, var_dev [C] double.  NaN variance for N = 1.
 * Errors: FMC_EINVAL if N < 1 or C < 1.
 */
int fmc_moments(fmc_ctx* ctx, const float* x_dev, int64_t N, int64_t C, double* mean_dev, double* var_dev,
                void* stream);

/* ---- diagnostics and measurement ------------------------------------------ */

/*
 * Waits for all work on the context's device, then reports the device-side
 * status words of the last simulation or tensor-core reconstruction:
 * *eq_iterations = Newton iterations of the last equilibrium (-1: did not
 * converge), *kernel_error = 0 or the code of a bounded wait that gave up.
 * Returns FMC_OK, FMC_ENOCONVERGE or FMC_ETIMEOUT accordingly.
 */
int fmc_device_status(fmc_ctx* ctx, int* eq_iterations, int* kernel_error);




/* ---- kernel choice of the fused path (no counterpart in the paper) -------- */
#define FMC_KERNEL_AUTO 0        /* per sample for n <= 16, split with the tensor-core network sum above */
#define FMC_KERNEL_PER_SAMPLE 1  /* one thread integrates a whole sample (n <= FMC_MAX_MACHINES_PLAIN) */
#define FMC_KERNEL_SPLIT 2       /* four warps share each sample's machines (any n up to FMC_MAX_MACHINES) */
#define FMC_KERNEL_SPLIT_TC 3    /* the split kernel with each RK stage's network sums over the CTA's 128
                                    samples as one tcgen05 TF32x3 product (13 <= n <= FMC_MAX_MACHINES) */

/*
 * Chooses the fused kernel for this context's later single-scenario calls
 * (fmc_simulate, fmc_simulate_sums).  AUTO takes the per-sample kernel up to 16
 * machines and the split kernel with the tensor-core network sum above (launch
 * rules, fmc_set_launch_rules, may choose otherwise per bucket); a system on an
 * infinite bus that fills every machine slot of the tensor-core layout
 * (n = 4 nmt: 20, 28, 40, 52 machines) takes the FP32 split kernel.  Batches and
 * the server always use AUTO's choice.  FMC_EINVAL for an unknown policy; a
 * per-sample request above 16 machines, or a SPLIT_TC request below 13 machines
 * or for such an infinite-bus system, fails at the call with FMC_EUNSUPPORTED.
 */
int fmc_set_kernel_policy(fmc_ctx* ctx, int32_t policy);

/*
 * Launch-shape rules of the fused path (no counterpart in the paper), as an
 * autotuner that measured the shapes writes them: the first rule whose ranges
 * hold a launch's machines n, disturbances d and samples N sets its kernel
 * (AUTO's choice only), the resident CTAs per SM and the time chunk; zero
 * fields keep the library's own choice.  Applies to the context's single-
 * scenario calls under FMC_KERNEL_AUTO and to its batches.  A chunk is cut to
 * what the TMEM share of max_ctas CTAs holds (and to 16 at least); the
 * large-system kernel keeps one CTA per SM.  The rules are copied; count 0
 * clears them.  FMC_EINVAL on a malformed rule (empty range, kernel not an
 * FMC_KERNEL_* value, max_ctas outside 0..4, TC not 0 or a power of two in
 * 16..256).
 */
typedef struct fmc_launch_rule {
    int32_t n_min, n_max;   /* machines */
    int32_t d_min, d_max;   /* disturbances */
    int64_t N_min, N_max;   /* samples of the launch */
    int32_t kernel;         /* FMC_KERNEL_* (AUTO: the library's choice) */
    int32_t max_ctas;       /* resident CTAs per SM, 1..4, or 0 */
    int32_t TC;             /* time chunk, 16..256 and a power of two, or 0 */
    int32_t reserved;
} fmc_launch_rule;
int fmc_set_launch_rules(fmc_ctx* ctx, const fmc_launch_rule* rules, int32_t count);

#ifdef __cplusplus
}
#endif

#endif /* FASTMC_H */
