"""GPU parity of the general Ito disturbances (Table I, the wind model of Eq.
windito) against the FP64 oracle: KL-driven paths with the Stratonovich drift
correction, and the traditional Monte Carlo's per-step normals without it.
Tolerances as the other simulation parity tests (trajectories 1e-4, moments 1e-5)."""
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


def _case(n, seed, N=160, T=0.6):
    sc = fs.multimachine_case(n=n, d=3, K=40, T=T, dt=0.005, N=N, seed=seed)
    # a wind farm (Eq. windito) on one machine, a Gamma and a Laplace process on others
    inj = np.zeros((n, 3))
    inj[1, 0] = 0.5
    inj[2, 1] = 0.3
    inj[n - 1, 2] = 0.4
    return sc.replace(inject=inj, ito=[fs.ito_wind(), fs.ito_gamma(2.0, 4.0), fs.ito_laplace(0.1, 0.05)])


@pytest.mark.parametrize("kernel", ["per_sample", "split"])
@pytest.mark.parametrize("sampling", [fs.LHS, fs.SRS_EM])
def test_general_disturbances(fmc, orc, kernel, sampling):
    sc = _case(8, 61).replace(sampling=sampling)
    fmc.set_kernel_policy(kernel)
    try:
        mean, var, traj = fmc.simulate(sc, path="fused", precision="bf16x3", want_traj=True)
    finally:
        fmc.set_kernel_policy("auto")
    fmc.device_status()
    if sampling == fs.SRS_EM:
        ref = orc.simulate_em(sc, want_traj=True, nthreads=8)
    else:
        ref = orc.simulate(sc, orc.lhs_sample(sc.seed, sc.N, sc.M), want_traj=True, nthreads=8)
    ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
    assert ed <= 1e-4 and ew <= 1e-4, (ed, ew)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)


def test_general_disturbances_plain_and_wide(fmc, orc):
    sc = _case(8, 62)
    m, v = fmc.simulate(sc, path="plain", precision="f32")
    ref = orc.simulate(sc, orc.lhs_sample(sc.seed, sc.N, sc.M), nthreads=8)
    _check_moments(m.cpu().numpy(), v.cpu().numpy(), ref["mean"], ref["var"], sc.n)
    sc = _case(24, 63, N=130, T=0.4)
    m, v = fmc.simulate(sc)
    ref = orc.simulate(sc, orc.lhs_sample(sc.seed, sc.N, sc.M), nthreads=8)
    _check_moments(m.cpu().numpy(), v.cpu().numpy(), ref["mean"], ref["var"], sc.n)


def test_ou_in_general_form_on_the_gpu(fmc):
    # an OU process written as a Table I Gaussian gives the built-in OU's moments
    sc = fs.multimachine_case(n=6, d=2, K=30, T=0.5, dt=0.005, N=256, seed=64).replace(theta=np.array([1.0, 1.0]))
    m0, v0 = fmc.simulate(sc)
    m1, v1 = fmc.simulate(sc.replace(ito=[fs.ito_gaussian(0.0, s**2 / 2.0) for s in sc.sigma]))
    _check_moments(m1.cpu().numpy(), v1.cpu().numpy(), m0.cpu().numpy(), v0.cpu().numpy(), sc.n, tol=1e-6)
