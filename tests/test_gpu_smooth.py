"""GPU parity of the smooth forcing (the random ODE of Eq. eqkl; FMC_FORCING_SMOOTH)
against the FP64 oracle, on the plain path and on the fused path (the forcing
contracted on the tensor cores at the half steps of each chunk, the stage values
formed in the step loop), with both fused kernels' chunk shapes (alone on the
GPU and in a batch).

Same tolerances as the other simulation parity tests: trajectories within 1e-4
normwise relative error on delta and on omega separately, moments within 1e-5.
"""
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
        "mm10": fs.multimachine_case(n=10, d=3, K=40, T=0.5, dt=0.005, N=200, seed=71),
        "mm6_heun_cosine": fs.multimachine_case(n=6, d=2, K=30, T=0.4, dt=0.005, N=150, seed=72).replace(
            integrator=fs.HEUN, basis=fs.BASIS_COSINE),
        "smib": fs.smib_case(N=300, K=50, T=1.0, dt=0.01),
        "mm5_trip": fs.multimachine_case(n=5, d=2, K=20, T=0.6, dt=0.005, N=129, seed=73).replace(
            event_machine=1, event_time=0.2, event_dpm=-0.5),
        "mm4_gamma": fs.multimachine_case(n=4, d=2, K=20, T=0.5, dt=0.005, N=160, seed=74).replace(
            ito=[fs.ito_gamma(2.0, 4.0), None]),
    }


@pytest.mark.parametrize("case", list(_cases()))
def test_smooth_plain_matches_the_oracle(fmc, orc, case):
    sc = _cases()[case].replace(forcing=fs.FORCING_SMOOTH)
    mean, var, traj = fmc.simulate(sc, path="plain", precision="f32", want_traj=True)
    fmc.device_status()
    zr = orc.lhs_sample(sc.seed, sc.N, sc.M)
    ref = orc.simulate(sc, zr, want_traj=True, nthreads=8)
    ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
    assert ed <= 1e-4 and ew <= 1e-4, (ed, ew)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)


def test_smooth_differs_from_the_increment_form(fmc, orc):
    # the two forms are different discretisations of the same truncated path
    sc = _cases()["mm10"]
    m0, _ = fmc.simulate(sc, path="plain", precision="f32")
    m1, _ = fmc.simulate(sc.replace(forcing=fs.FORCING_SMOOTH), path="plain", precision="f32")
    assert not np.array_equal(m0.cpu().numpy(), m1.cpu().numpy())


@pytest.mark.parametrize("case", list(_cases()))
def test_smooth_fused_matches_the_oracle(fmc, orc, case):
    sc = _cases()[case].replace(forcing=fs.FORCING_SMOOTH)
    mean, var, traj = fmc.simulate(sc, path="fused", precision="bf16x3", want_traj=True)
    fmc.device_status()
    zr = orc.lhs_sample(sc.seed, sc.N, sc.M)
    ref = orc.simulate(sc, zr, want_traj=True, nthreads=8)
    ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
    assert ed <= 1e-4 and ew <= 1e-4, (ed, ew)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)


def test_smooth_fused_in_a_batch_and_at_scale(fmc, orc):
    # a batch gives the kernel the shared-GPU chunk shape; the larger design runs
    # several waves with the horizon not a multiple of the chunk
    scs = [_cases()["mm10"].replace(forcing=fs.FORCING_SMOOTH),
           fs.multimachine_case(n=8, d=6, K=20, T=0.3, dt=0.005, N=300, seed=75).replace(forcing=fs.FORCING_SMOOTH)]
    b = fmc.Batch(scs, use_graph=True)
    means, vars_ = b.launch()
    fmc.device_status()
    for sc, m, v in zip(scs, means, vars_):
        ref = orc.simulate(sc, orc.lhs_sample(sc.seed, sc.N, sc.M), nthreads=8)
        _check_moments(m.cpu().numpy(), v.cpu().numpy(), ref["mean"], ref["var"], sc.n)
    b.close()
    sc = fs.multimachine_case(n=10, d=3, K=40, T=0.305, dt=0.005, N=60000, seed=76).replace(forcing=fs.FORCING_SMOOTH)
    mean, var = fmc.simulate(sc, path="fused", precision="bf16x3")
    ref = orc.simulate(sc, orc.lhs_sample(sc.seed, sc.N, sc.M), nthreads=16)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)


def test_smooth_forcing_on_the_split_kernel_is_refused(fmc):
    sc = fs.multimachine_case(n=20, d=2, K=20, T=0.1, dt=0.005, N=64, seed=77).replace(forcing=fs.FORCING_SMOOTH)
    with pytest.raises(fmc.FastMCError) as e:
        fmc.simulate(sc, path="fused")
    assert e.value.code == 8


def test_smooth_forcing_with_per_step_normals_is_refused(fmc):
    sc = _cases()["mm10"].replace(forcing=fs.FORCING_SMOOTH, sampling=fs.SRS_EM)
    with pytest.raises(fmc.FastMCError) as e:
        fmc.simulate(sc, path="plain", precision="f32")
    assert e.value.code == 1
