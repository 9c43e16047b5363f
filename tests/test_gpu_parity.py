"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances (stated once, derived from the arithmetic):
* LHS strata: bit-exact.
* zeta: 8 FP32 ulps plus the propagation of the FP32 probability argument,
  2^-21 min(p, 1-p) / phi(zeta) (FP32 relative error of p or 1-p times
  d zeta / dp = 1/phi).
* KL basis (FP64 on the GPU, rounded to FP32): 2 ulps of the largest entry.
* FP32 contraction: K * 2^-23 * sum_k |zeta_k phi_k| per entry.
* BF16x3 contraction: 2^-15 * sum_k |zeta_k phi_k| (dropped lo*lo term and the
  residuals of both splits, each below 2^-16 relative).
* BF16 contraction: 2^-7 * sum_k |zeta_k phi_k|.
* trajectories (FP32 integration, FP32 or BF16x3 contraction): normwise relative
  error <= 1e-4 on delta and on omega separately.
* moments (same samples): normwise relative error <= 1e-5 per moment array.
"""
import math

import numpy as np
import pytest
from scipy.special import ndtr

import fmc_synth as fs
from gpu_common import need_gpu, normwise_rel, traj_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fmc():
    return need_gpu()


@pytest.fixture(params=["per_sample", "split"])
def kernel(fmc, request):
    """Runs a test with each fused kernel forced, then restores the automatic choice."""
    fmc.set_kernel_policy(request.param)
    yield request.param
    fmc.set_kernel_policy("auto")


def _same_to_fp32(m, v, m1, v1):
    """Moments that differ only by FP32 rounding of spread-scale sums: means within
    1e-6 of the largest standard deviation of their state block, variances within
    2e-6 relative."""
    n = m.shape[1] // 2
    for sl in (slice(0, n), slice(n, 2 * n)):
        sd = float(np.sqrt(np.max(v1[:, sl])))
        assert np.max(np.abs(m[:, sl] - m1[:, sl])) <= 1e-6 * sd + 1e-15
        assert np.allclose(v[:, sl], v1[:, sl], rtol=2e-6, atol=1e-18)


def _batch_kernel(fmc, sc):
    # the kernel a batch (shared GPU) takes for this scenario
    fmc.set_kernel_policy("per_sample" if sc.n <= 16 else "split_tc")


def _zeta_tol(zref):
    z = np.asarray(zref, dtype=np.float64)
    ulp = np.spacing(np.abs(z).astype(np.float32)).astype(np.float64)
    p = ndtr(z)
    q = np.minimum(p, 1.0 - p)
    phi = np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)
    return 8 * ulp + 2.0**-21 * q / phi + 1e-30


# ----------------------------------------------------------------------------- a1 LHS


@pytest.mark.parametrize("N,M,k0,count", [(1, 5, 0, 1), (2, 7, 0, 2), (3, 4, 1, 2), (1000, 100, 0, 1000),
                                          (65537, 3, 0, 65537), (70000, 9, 12345, 777)])
def test_lhs_strata_bit_exact_and_values(fmc, orc, N, M, k0, count):
    import torch
    strata = torch.empty((M, count), dtype=torch.int32, device="cuda")
    zeta, _ = fmc.lhs_sample(17, N, M, mode=fmc.LHS, k0=k0, count=count, strata=strata)
    zg = zeta.cpu().numpy().astype(np.float64)
    sg = strata.cpu().numpy().view(np.uint32)
    zr, sr = orc.lhs_sample(17, N, M, mode=orc.LHS, k0=k0, count=count, with_strata=True)
    assert np.array_equal(sg, sr)
    assert np.all(np.abs(zg - zr) <= _zeta_tol(zr))


@pytest.mark.parametrize("mode", [1, 2])
def test_lhs_srs_and_midpoint(fmc, orc, mode):
    N, M = 513, 11
    zeta, _ = fmc.lhs_sample(5, N, M, mode=mode)
    zr = orc.lhs_sample(5, N, M, mode=mode)
    assert np.all(np.abs(zeta.cpu().numpy() - zr) <= _zeta_tol(zr))


def test_lhs_split_layout(fmc, orc):
    import torch
    N, d, K = 300, 3, 13
    hi, lo = fmc.lhs_sample_split(9, N, d, K)
    Ks = 16
    assert hi.shape == (N, d, Ks)
    h = hi.float().cpu().numpy()
    l = lo.float().cpu().numpy()
    assert np.all(h[:, :, K:] == 0) and np.all(l[:, :, K:] == 0)
    zr = orc.lhs_sample(9, N, d * K).reshape(N, d, K)
    # hi + lo carries the FP32 value to within 2^-16 relative
    assert np.all(np.abs(h[:, :, :K] + l[:, :, :K] - zr) <= 2.0**-15 * np.abs(zr) + _zeta_tol(zr))


# ----------------------------------------------------------------------------- a2 basis


@pytest.mark.parametrize("K,T,Nt", [(1, 1.0, 7), (100, 10.0, 1000), (200, 20.0, 4000), (37, 3.3, 333)])
@pytest.mark.parametrize("basis", [0, 1])
def test_kl_basis(fmc, orc, K, T, Nt, basis):
    phi = fmc.kl_basis(K, T, Nt, basis).cpu().numpy()
    ref = orc.kl_increment_basis(K, T, Nt, basis)
    assert np.max(np.abs(phi - ref)) <= 2 * np.spacing(np.float32(np.max(np.abs(ref))))


# ----------------------------------------------------------------------------- a3 contraction


@pytest.mark.parametrize("precision,factor", [("f32", None), ("bf16x3", 2.0**-15), ("bf16", 2.0**-7)])
@pytest.mark.parametrize("count,d,K,T,dt", [(300, 2, 50, 1.0, 0.01), (129, 3, 200, 2.0, 0.005),
                                            (1, 1, 1, 0.5, 0.01), (257, 1, 100, 10.0, 0.01)])
def test_kle_reconstruct(fmc, orc, precision, factor, count, d, K, T, dt):
    import torch
    Nt = int(round(T / dt))
    zeta, _ = fmc.lhs_sample(3, count, d * K)
    dW = fmc.kle_reconstruct(zeta, d, K, T, dt, precision=precision)
    fmc.device_status()
    got = dW.cpu().numpy().astype(np.float64)
    z64 = zeta.cpu().numpy().astype(np.float64)
    ref = orc.kle_reconstruct(z64, d, K, T, Nt)
    phi = orc.kl_increment_basis(K, T, Nt)
    absum = np.einsum("swk,kn->swn", np.abs(z64.reshape(count, d, K)), np.abs(phi))
    if factor is None:
        tol = K * 2.0**-23 * absum + 1e-12
    else:
        tol = factor * absum + 1e-12
    assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) / tol)


# ----------------------------------------------------------------------------- a7 equilibrium


@pytest.mark.parametrize("case", ["smib", "mm10", "mm16", "mm3"])
def test_equilibrium(fmc, orc, case):
    sc = {"smib": fs.smib_case(), "mm10": fs.multimachine_case(n=10), "mm16": fs.multimachine_case(n=16, seed=4),
          "mm3": fs.multimachine_case(n=3, d=1, seed=2)}[case]
    d0, pm = fmc.equilibrium(sc)
    rd0, rpm, _ = orc.equilibrium(sc)
    assert np.max(np.abs(d0 - rd0)) < 1e-11
    assert np.max(np.abs(pm - rpm)) < 1e-10


# ----------------------------------------------------------------------------- a4-a6 simulation


def _check_moments(m, v, rm, rv, n, tol=1e-5):
    """Means: error relative to the RMS size of the variable, max sqrt(mean^2 + var)
    (a mean of values each off by eps*scale is off by at most eps*scale; the mean
    of the speed deviation itself is near zero).  Variances: normwise relative."""
    for sl in (slice(0, n), slice(n, 2 * n)):
        scale = np.max(np.sqrt(rm[:, sl] ** 2 + rv[:, sl]))
        assert np.max(np.abs(m[:, sl] - rm[:, sl])) <= tol * scale
        assert normwise_rel(v[:, sl], rv[:, sl]) <= tol


def _small_cases():
    return {
        "smib": fs.smib_case(N=300, K=100, T=2.0, dt=0.01),
        "mm7_cosine": fs.multimachine_case(n=7, d=2, K=30, T=0.5, dt=0.005, N=150, seed=4).replace(
            basis=fs.BASIS_COSINE),
        "mm10": fs.multimachine_case(n=10, d=3, K=40, T=1.0, dt=0.005, N=200, seed=1),
        "mm5_ragged": fs.multimachine_case(n=5, d=2, K=23, T=0.333, dt=0.003, N=131, seed=2),
        "mm16_d8": fs.multimachine_case(n=16, d=8, K=16, T=0.2, dt=0.005, N=129, seed=3),
    }


@pytest.mark.parametrize("case", ["smib", "mm10", "mm5_ragged", "mm16_d8", "mm7_cosine"])
def test_simulate_trajectories_and_moments_plain(fmc, orc, case):
    _trajectories_and_moments(fmc, orc, "plain", "f32", case)


@pytest.mark.parametrize("case", ["smib", "mm10", "mm5_ragged", "mm16_d8", "mm7_cosine"])
def test_simulate_trajectories_and_moments_fused(fmc, orc, kernel, case):
    _trajectories_and_moments(fmc, orc, "fused", "bf16x3", case)


def _trajectories_and_moments(fmc, orc, path, precision, case):
    sc = _small_cases()[case]
    mean, var, traj = fmc.simulate(sc, path=path, precision=precision, want_traj=True)
    fmc.device_status()
    zr = orc.lhs_sample(sc.seed, sc.N, sc.M)
    ref = orc.simulate(sc, zr, want_traj=True, nthreads=8)
    ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
    assert ed <= 1e-4 and ew <= 1e-4, (ed, ew)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)


def test_simulate_bf16_error_is_stated(fmc, orc, kernel):
    # BF16 contraction: trajectories carry the 2^-9 rounding of zeta and phi
    sc = _small_cases()["mm10"]
    mean, var, traj = fmc.simulate(sc, path="fused", precision="bf16", want_traj=True)
    zr = orc.lhs_sample(sc.seed, sc.N, sc.M)
    ref = orc.simulate(sc, zr, want_traj=True, nthreads=8)
    ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
    assert ed <= 2e-2 and ew <= 2e-2, (ed, ew)


@pytest.mark.parametrize("tiles_per_sm", [1, 2, 3, 3.5])
@pytest.mark.parametrize("d", [1, 3, 6])
def test_chunk_length_follows_the_tiles(fmc, orc, tiles_per_sm, d):
    # The time chunk grows when few CTAs share an SM (one, two, or four per SM
    # give 512, 256 or 128 TMEM columns per CTA): sample counts just under each
    # boundary, a horizon that is not a multiple of any chunk length; 3.5 tiles
    # per SM leaves the SMs unevenly loaded (four CTAs on some, three on others).
    sms, _ = fmc.default_context().info()
    N = int(128 * sms * tiles_per_sm) - 37
    sc = fs.multimachine_case(n=4, d=d, K=24, T=0.305, dt=0.005, N=N, seed=40 + d)
    mean, var, traj = fmc.simulate(sc, path="fused", precision="bf16x3", want_traj=True)
    fmc.device_status()
    zr = orc.lhs_sample(sc.seed, sc.N, sc.M)
    ref = orc.simulate(sc, zr, want_traj=True, nthreads=8)
    ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
    assert ed <= 1e-4 and ew <= 1e-4, (ed, ew)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)


def test_heun_integrator(fmc, orc, kernel):
    sc = _small_cases()["mm10"].replace(integrator=fs.HEUN)
    mean, var, traj = fmc.simulate(sc, path="fused", precision="bf16x3", want_traj=True)
    zr = orc.lhs_sample(sc.seed, sc.N, sc.M)
    ref = orc.simulate(sc, zr, want_traj=True, nthreads=8)
    ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
    assert ed <= 1e-4 and ew <= 1e-4, (ed, ew)


def test_single_sample_variance_nan(fmc):
    sc = fs.smib_case(N=1, T=0.1)
    mean, var = fmc.simulate(sc, path="fused")
    v = var.cpu().numpy()
    assert np.all(np.isnan(v))


def test_sigma_zero_stays_at_equilibrium(fmc, orc, kernel):
    sc = fs.multimachine_case(n=10, d=3, K=50, T=1.0, dt=0.005, N=256).replace(sigma=np.zeros(3))
    mean, var = fmc.simulate(sc, path="fused")
    d0, _, _ = orc.equilibrium(sc)
    m = mean.cpu().numpy()
    assert np.max(np.abs(m[:, :10] - d0)) < 1e-5
    assert np.max(np.abs(m[:, 10:])) < 1e-6
    assert np.max(var.cpu().numpy()) < 1e-10


# ----------------------------------------------------------------------------- a6 moments kernel


@pytest.mark.parametrize("N,C", [(1, 3), (2, 5), (1000, 77), (4097, 300)])
def test_moments_kernel(fmc, orc, N, C):
    import torch
    rng = np.random.default_rng(N)
    x = (rng.standard_normal((N, C)) * 0.1 + rng.uniform(-2, 2, size=C)).astype(np.float32)
    mean, var = fmc.moments(torch.from_numpy(x).cuda())
    rm, rv = orc.moments_twopass(x.astype(np.float64))
    assert normwise_rel(mean.cpu().numpy(), rm) <= 1e-7
    if N > 1:
        assert normwise_rel(var.cpu().numpy(), rv) <= 1e-6
    else:
        assert np.all(np.isnan(var.cpu().numpy()))


# ----------------------------------------------------------------------------- full-size workload


def test_full_size_multimachine_sampled(fmc, orc):
    """The 10-machine, 3-disturbance, K = 200, T = 20 s, dt = 5 ms, N = 2^16 workload in
    the fused BF16x3 launch: sampled trajectories against the oracle sample by sample,
    the reducer against FP64 moments of the emitted trajectories, and LHS strata of
    sampled dimensions bit-exact."""
    import torch
    sc = fs.multimachine_case()
    mean, var, traj = fmc.simulate(sc, path="fused", precision="bf16x3", want_traj=True)
    fmc.device_status()
    n = sc.n
    picks = [0, 1, 4095, 32768, sc.N - 1]
    for k in picks:
        zk = orc.lhs_sample(sc.seed, sc.N, sc.M, k0=k, count=1)
        ref = orc.simulate(sc, zk, want_traj=True, want_moments=False)
        ed, ew = traj_errors(traj[k].cpu().numpy(), ref["traj"][0], n)
        assert ed <= 1e-4 and ew <= 1e-4, (k, ed, ew)
    # reducer vs FP64 moments of the same (FP32-rounded) trajectories, at times where
    # the spread is well above the FP32 rounding of the angles (~1e-7 rad)
    for t in [0, 1000, 2000, sc.Nt]:
        x = traj[:, t, :].double()
        assert normwise_rel(mean[t].cpu().numpy(), x.mean(0).cpu().numpy()) <= 1e-6
        if t > 0:
            assert normwise_rel(var[t].cpu().numpy(), x.var(0, unbiased=True).cpu().numpy()) <= 1e-5
    del traj
    torch.cuda.empty_cache()
    strata = torch.empty((sc.M, sc.N), dtype=torch.int32, device="cuda")
    fmc.lhs_sample(sc.seed, sc.N, sc.M, strata=strata)
    sg = strata.cpu().numpy().view(np.uint32)
    for i in [0, 199, 200, 599]:
        sr = np.array([orc.lhs_stratum(sc.seed, sc.N, i, k) for k in range(sc.N)], dtype=np.uint32)
        assert np.array_equal(sg[i], sr)


def test_integrator_sincos_accuracy(fmc):
    import torch
    x = torch.cat([torch.linspace(-100.0, 100.0, 200001), torch.linspace(-4.0, 4.0, 100001),
                   torch.tensor([0.0, 1e-30, -1e-30, math.pi / 4, math.pi / 2, math.pi, 3 * math.pi / 2])])
    x = x.float().cuda()
    s, c, sref, cref = fmc.test_sincos(x)
    xd = x.double().cpu().numpy()
    es = np.abs(s.double().cpu().numpy() - np.sin(xd))
    ec = np.abs(c.double().cpu().numpy() - np.cos(xd))
    er = max(np.abs(sref.double().cpu().numpy() - np.sin(xd)).max(), np.abs(cref.double().cpu().numpy() - np.cos(xd)).max())
    assert es.max() <= 1.2e-7 and ec.max() <= 1.2e-7, (es.max(), ec.max())
    assert max(es.max(), ec.max()) <= 2.0 * er + 1e-8


# ----------------------------------------------------------------------------- batches


def _mixed_batch():
    return [fs.multimachine_case(n=3, d=1, K=50, T=0.5, dt=0.005, N=300, seed=11),
            fs.multimachine_case(n=10, d=3, K=200, T=1.0, dt=0.005, N=1000, seed=12),
            fs.multimachine_case(n=16, d=8, K=37, T=0.25, dt=0.005, N=129, seed=13),
            fs.smib_case(N=777, T=1.0),
            fs.multimachine_case(n=7, d=5, K=120, T=0.8, dt=0.005, N=4096, seed=14)]


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_single_scenarios(fmc, use_graph):
    scs = _mixed_batch()
    b = fmc.Batch(scs, use_graph=use_graph)
    for rep in range(2):  # a replayed graph gives the same results
        means, vars_ = b.launch()
        fmc.device_status()
        for sc, m, v in zip(scs, means, vars_):
            _batch_kernel(fmc, sc)
            m1, v1 = fmc.simulate(sc, path="fused", precision="bf16x3")
            fmc.set_kernel_policy("auto")
            # same samples, kernel and per-tile arithmetic.  The batch adds the tiles'
            # (reference, deviation sum, M2) in FP64; a single call first merges
            # groups of eight tiles in FP32 about the group's reference, so the two
            # agree to FP32 rounding on the scale of the spread
            _same_to_fp32(m.cpu().numpy(), v.cpu().numpy(), m1.cpu().numpy(), v1.cpu().numpy())
    b.close()


def test_batch_moments_match_oracle(fmc, orc):
    scs = _mixed_batch()[:2]
    b = fmc.Batch(scs, use_graph=True)
    means, vars_ = b.launch()
    for sc, m, v in zip(scs, means, vars_):
        zr = orc.lhs_sample(sc.seed, sc.N, sc.M)
        ref = orc.simulate(sc, zr, nthreads=8)
        _check_moments(m.cpu().numpy(), v.cpu().numpy(), ref["mean"], ref["var"], sc.n)
    b.close()


# ----------------------------------------------------------------------------- the traditional Monte Carlo


@pytest.mark.parametrize("case", ["mm10", "mm16_d8", "smib"])
def test_srs_em_trajectories_and_moments(fmc, orc, kernel, case):
    # the paper's comparator (Section V-B): per-step normals drawn inside the
    # kernels from the same Philox counters as the oracle's
    sc = _small_cases()[case].replace(sampling=fs.SRS_EM)
    ref = orc.simulate_em(sc, want_traj=True, nthreads=8)
    for path, precision in (("fused", "bf16x3"), ("plain", "f32")):
        if path == "plain" and kernel == "split":
            continue
        mean, var, traj = fmc.simulate(sc, path=path, precision=precision, want_traj=True)
        fmc.device_status()
        ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
        assert ed <= 1e-4 and ew <= 1e-4, (path, ed, ew)
        _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)


def test_srs_em_sample_blocks(fmc, orc):
    # blocks of the design through the sums entry point draw the increments of
    # their own design indices
    sc = _small_cases()["mm10"].replace(sampling=fs.SRS_EM)
    ref = orc.simulate_em(sc, nthreads=8)
    a1, a2, shift = fmc.simulate_sums(sc, 0, 77)
    b1, b2, _ = fmc.simulate_sums(sc, 77, sc.N - 77)
    S1 = (a1 + b1).cpu().numpy()
    S2 = (a2 + b2).cpu().numpy()
    N = sc.N
    mean = shift.cpu().numpy()[None, :] + S1 / N
    var = (S2 - S1 * S1 / N) / (N - 1)
    _check_moments(mean, var, ref["mean"], ref["var"], sc.n)
