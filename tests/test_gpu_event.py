"""GPU parity of the event (a step in one machine's mechanical power, the paper's
generator-trip experiment in the classical model) and of the response function
(RMS centre-of-inertia speed deviation, Section V-B) against the FP64 oracle.

Tolerances as in the other parity tests: trajectories 1e-4 normwise, moments
1e-5; the response function's expectation within 1e-5 and its variance within
1e-4 relative (FP32 sums of 10^2..10^3 squared speeds per sample)."""
import numpy as np
import pytest

import fmc_synth as fs
from gpu_common import need_gpu, normwise_rel, traj_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fmc():
    return need_gpu()


def _check_moments(m, v, rm, rv, n, tol=1e-5):
    for sl in (slice(0, n), slice(n, 2 * n)):
        scale = np.max(np.sqrt(rm[:, sl] ** 2 + rv[:, sl]))
        assert np.max(np.abs(m[:, sl] - rm[:, sl])) <= tol * scale
        assert normwise_rel(v[:, sl], rv[:, sl]) <= tol


def _cases():
    return {
        "mm10_trip": fs.multimachine_case(n=10, d=3, K=40, T=1.0, dt=0.005, N=200, seed=51).replace(
            event_machine=2, event_time=0.3, event_dpm=-0.6),
        "mm7_d4_gain": fs.multimachine_case(n=7, d=4, K=30, T=0.6, dt=0.005, N=131, seed=52).replace(
            event_machine=6, event_time=0.1, event_dpm=0.4),
        "mm22_trip": fs.multimachine_case(n=22, d=2, K=30, T=0.5, dt=0.005, N=150, seed=53).replace(
            event_machine=5, event_time=0.2, event_dpm=-1.0),
        "smib_step": fs.smib_case(N=200, K=50, T=1.0, dt=0.01).replace(event_machine=0, event_time=0.5,
                                                                         event_dpm=-0.1),
    }


def _rrf_check(rrf, ref_rrf):
    """Mean within 1e-5 relative.  Variance: if every sample's response carries a
    relative error up to eps = 1e-5 (the moments' bound), the unbiased variance
    moves by at most 2 eps rms(r) std(r) (the covariance of the errors with the
    values), i.e. 2 eps rms(r)/std(r) relative -- larger than eps where the
    response's spread is small against its size."""
    e, v = rrf.cpu().numpy()
    eps = 1e-5
    assert abs(e - ref_rrf.mean()) <= eps * ref_rrf.mean()
    rms = float(np.sqrt(np.mean(ref_rrf ** 2)))
    sd = float(ref_rrf.std(ddof=1))
    assert abs(v - ref_rrf.var(ddof=1)) <= 2.0 * eps * rms * sd * len(ref_rrf) / (len(ref_rrf) - 1) + 1e-30


@pytest.mark.parametrize("kernel", ["per_sample", "split", "split_tc"])
@pytest.mark.parametrize("case", ["mm10_trip", "mm7_d4_gain", "mm22_trip", "smib_step"])
def test_event_fused(fmc, orc, kernel, case):
    sc = _cases()[case]
    if kernel.startswith("per_sample") and sc.n > 16:
        pytest.skip("the per-sample kernel takes up to 16 machines")
    if kernel == "split_tc" and sc.n < 13:
        pytest.skip("the tensor-core network sum takes 13 machines and more")
    fmc.set_kernel_policy(kernel)
    try:
        mean, var, traj = fmc.simulate(sc, path="fused", precision="bf16x3", want_traj=True)
        rrf, m2, v2 = fmc.simulate_rrf(sc, path="fused", precision="bf16x3")
    finally:
        fmc.set_kernel_policy("auto")
    fmc.device_status()
    zr = orc.lhs_sample(sc.seed, sc.N, sc.M)
    ref = orc.simulate(sc, zr, want_traj=True, nthreads=8)
    ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
    assert ed <= 1e-4 and ew <= 1e-4, (ed, ew)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)
    _check_moments(m2.cpu().numpy(), v2.cpu().numpy(), ref["mean"], ref["var"], sc.n)
    _rrf_check(rrf, ref["rrf"])


@pytest.mark.parametrize("case", ["mm10_trip", "smib_step"])
def test_event_plain(fmc, orc, case):
    sc = _cases()[case]
    rrf, mean, var = fmc.simulate_rrf(sc, path="plain", precision="f32")
    zr = orc.lhs_sample(sc.seed, sc.N, sc.M)
    ref = orc.simulate(sc, zr, nthreads=8)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)
    _rrf_check(rrf, ref["rrf"])


def test_event_with_the_traditional_monte_carlo(fmc, orc):
    sc = _cases()["mm10_trip"].replace(sampling=fs.SRS_EM)
    rrf, mean, var = fmc.simulate_rrf(sc, path="fused", precision="bf16x3")
    ref = orc.simulate_em(sc, nthreads=8)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)
    _rrf_check(rrf, ref["rrf"])


def test_no_event_leaves_the_results_unchanged(fmc):
    sc = fs.multimachine_case(n=10, d=3, K=40, T=0.5, dt=0.005, N=256, seed=54)
    m0, v0 = fmc.simulate(sc)
    rrf, m1, v1 = fmc.simulate_rrf(sc.replace(event_machine=None))
    assert np.array_equal(m0.cpu().numpy(), m1.cpu().numpy())
    assert np.array_equal(v0.cpu().numpy(), v1.cpu().numpy())
    assert rrf.cpu().numpy()[0] > 0


def test_event_needs_a_spare_disturbance_slot(fmc):
    sc = fs.multimachine_case(n=5, d=8, K=10, T=0.1, dt=0.005, N=64, seed=55).replace(
        event_machine=1, event_time=0.05, event_dpm=-0.2)
    with pytest.raises(fmc.FastMCError) as e:
        fmc.simulate(sc)
    assert e.value.code == fmc.EUNSUPPORTED
