/*
 * fastmc_diag.h -- diagnostics and test hooks of libfastmc (no counterpart in
 * the paper): the self-check of the bounded-wait failure path, kernel-phase
 * timing with CUDA events, the integrator's sin/cos against CUDA's sincosf, the
 * split kernel's tensor-core network matrix and layout choice, and the occupancy
 * of the last fused launch.  The method itself needs none of
 * them (fastmc.h); the same library exports them.
 */
#ifndef FASTMC_DIAG_H
#define FASTMC_DIAG_H

#include "fastmc.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Self-check of the failure-detection path (no counterpart in the paper).  Every
 * spin of the library's kernels on an mbarrier is bounded; when it runs out the
 * kernel records a timeout code in a device status word and returns, and
 * fmc_device_status reports FMC_ETIMEOUT.  This call exercises that path without
 * a fault: it clears the status word and launches one CTA whose thread waits, at
 * most poll_limit polls (1 .. 2^24), on an mbarrier that nothing arrives at,
 * with no bulk copy or MMA in flight, so the wait runs out and the timeout is
 * recorded.
 *   target 0: the context's status word (as fmc_simulate's kernels use it);
 *   target 1: the allocation-free reconstruction's word in its scratch array
 *             (same device rule as fmc_kle_reconstruct_noalloc).
 * Asynchronous on `stream`; a following fmc_device_status returns FMC_ETIMEOUT.
 * Errors: FMC_EINVAL (target, poll_limit, device), FMC_ENOMEM, FMC_ECUDA.
 */
int fmc_check_wait_path(fmc_ctx* ctx, int32_t target, int64_t poll_limit, void* stream);

/*
 * Kernel timing with CUDA events recorded on the launching stream around every
 * kernel phase of later calls (at most max_records phases; enable = 0 stops and
 * clears).  Phases: 0 LHS, 1 KL basis, 2 equilibrium, 3 fused simulation,
 * 4 fused moment reduce, 5 FP32 contraction, 6 plain integrator, 7 moments,
 * 8 a whole batch graph launch.
 */
int fmc_profile(fmc_ctx* ctx, int32_t enable, int64_t max_records);

/* Synchronises, then sums the recorded durations of one phase. */
int fmc_profile_read(fmc_ctx* ctx, int32_t phase, double* total_ms, int64_t* launches);

/*
 * Test hook (no counterpart in the paper): evaluates the integrator's own
 * sin/cos (Cody-Waite reduction + Taylor series, FP32) and CUDA's sincosf on
 * x_dev[n], writing s_dev, c_dev and s_ref_dev, c_ref_dev (device, float[n]).
 */
int fmc_test_sincos(fmc_ctx* ctx, const float* x_dev, int64_t n, float* s_dev, float* c_dev, float* s_ref_dev,
                    float* c_ref_dev, void* stream);

/*
 * The split kernel's tensor-core network matrix as the library builds it for a
 * launch (host only, no device): FP32 [2][NN][NN], Net_hi then Net_lo, with
 * NN = 2 KH H rounded up to a multiple of 16, KH = 2 nmt rounded up to a
 * multiple of 4, row and column of machine i at (i mod H) KH + 2 (i / H) (then
 * +1 for the v row and the eta column): Net = [[GE, -BE], [BE, GE]] with
 * GE = E_i E_j G_ij, BE = E_i E_j B_ij, zero diagonal and padding; with an
 * infinite bus its column E_i V (Ginf_i, Binf_i) sits in machine slot
 * H nmt - 1.  H is 2 or 4, n <= H nmt (< with an infinite bus).
 * Errors: FMC_EINVAL (arguments, out_floats < 2 NN^2).
 */
int fmc_diag_net_matrix(const fmc_scenario* scen, int32_t nmt, int32_t H, float* out, int64_t out_floats);

/*
 * The kernel and layout a single-scenario fused launch of `count` samples takes
 * under `policy` (FMC_KERNEL_*; no launch rules), as the library decides it
 * (host only, no device): out[0] the kernel (FMC_KERNEL_PER_SAMPLE, FMC_KERNEL_SPLIT
 * or FMC_KERNEL_SPLIT_TC), out[1] machine slots per thread of the split kernel
 * (0 for the per-sample kernel), out[2] its warps per sample, out[3] the
 * disturbance-slot bucket, out[4] 1 for the infinite-bus form.  Returns the
 * call's refusal (FMC_EUNSUPPORTED) where the launch would refuse.
 * Errors: FMC_EINVAL (arguments).
 */
int fmc_diag_kernel_choice(const fmc_scenario* scen, int32_t path, int32_t policy, int64_t count, int32_t* out);

/* CTAs per SM the last fused launch could keep resident (occupancy API). */
int fmc_last_fused_occupancy(const fmc_ctx* ctx, int* ctas_per_sm);

#ifdef __cplusplus
}
#endif

#endif /* FASTMC_DIAG_H */
