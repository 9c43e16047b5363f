"""GPU parity of the large-system fused kernel (17..52 machines, four warps per
sample group) against the FP64 oracle, with the network sums on the FP32 pipes
("split") and as the tensor-core TF32x3 product ("split_tc", the automatic choice).

Same tolerances as the other simulation parity tests: trajectories within 1e-4
normwise relative error on delta and on omega separately, moments within 1e-5.
Machine counts cover every slot bucket (n <= 20, 28, 40, 52) with full and
ragged last machine groups; sample counts leave a ragged last tile.
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


CASES = {
    "n17_d1": dict(n=17, d=1, K=30, T=0.5, dt=0.005, N=131, seed=21),
    "n22_d5": dict(n=22, d=5, K=30, T=0.4, dt=0.005, N=150, seed=28),
    "n24_d4": dict(n=24, d=4, K=40, T=0.5, dt=0.005, N=200, seed=27),
    "n28_d3": dict(n=28, d=3, K=40, T=0.5, dt=0.005, N=200, seed=22),
    "n37_d5": dict(n=37, d=5, K=23, T=0.333, dt=0.003, N=129, seed=23),
    "n50_d8": dict(n=50, d=8, K=16, T=0.2, dt=0.005, N=257, seed=24),
    "n52_d2": dict(n=52, d=2, K=50, T=0.3, dt=0.005, N=128, seed=25),
}


@pytest.mark.parametrize("kernel", ["split", "split_tc"])
@pytest.mark.parametrize("case", list(CASES))
def test_wide_trajectories_and_moments(fmc, orc, case, kernel):
    sc = fs.multimachine_case(**CASES[case])
    fmc.set_kernel_policy(kernel)
    try:
        mean, var, traj = fmc.simulate(sc, path="fused", precision="bf16x3", want_traj=True)
    finally:
        fmc.set_kernel_policy("auto")
    fmc.device_status()
    zr = orc.lhs_sample(sc.seed, sc.N, sc.M)
    ref = orc.simulate(sc, zr, want_traj=True, nthreads=8)
    ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
    assert ed <= 1e-4 and ew <= 1e-4, (ed, ew)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)


def test_wide_heun(fmc, orc):
    sc = fs.multimachine_case(**CASES["n28_d3"]).replace(integrator=fs.HEUN)
    mean, var, traj = fmc.simulate(sc, path="fused", precision="bf16x3", want_traj=True)
    zr = orc.lhs_sample(sc.seed, sc.N, sc.M)
    ref = orc.simulate(sc, zr, want_traj=True, nthreads=8)
    ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
    assert ed <= 1e-4 and ew <= 1e-4, (ed, ew)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)


def test_wide_sums_without_trajectories_match(fmc):
    # the moment path alone (no trajectory buffer) gives the same moments
    sc = fs.multimachine_case(**CASES["n37_d5"])
    m1, v1, _ = fmc.simulate(sc, path="fused", precision="bf16x3", want_traj=True)
    m2, v2 = fmc.simulate(sc, path="fused", precision="bf16x3")
    assert np.array_equal(m1.cpu().numpy(), m2.cpu().numpy())
    assert np.array_equal(v1.cpu().numpy(), v2.cpu().numpy())


def test_wide_sigma_zero_stays_at_equilibrium(fmc, orc):
    sc = fs.multimachine_case(n=40, d=4, K=50, T=1.0, dt=0.005, N=256, seed=5).replace(sigma=np.zeros(4))
    mean, var = fmc.simulate(sc, path="fused")
    d0, _, _ = orc.equilibrium(sc)
    m = mean.cpu().numpy()
    assert np.max(np.abs(m[:, :40] - d0)) < 1e-5
    assert np.max(np.abs(m[:, 40:])) < 1e-6
    assert np.max(var.cpu().numpy()) < 1e-10


def test_wide_sample_blocks_add_up(fmc, orc):
    # two blocks of the same design through the sums entry point = the whole design
    sc = fs.multimachine_case(**CASES["n50_d8"])
    zr = orc.lhs_sample(sc.seed, sc.N, sc.M)
    ref = orc.simulate(sc, zr, nthreads=8)
    a1, a2, shift = fmc.simulate_sums(sc, 0, 129)
    b1, b2, _ = fmc.simulate_sums(sc, 129, sc.N - 129)
    S1 = (a1 + b1).cpu().numpy()
    S2 = (a2 + b2).cpu().numpy()
    sh = shift.cpu().numpy()
    N = sc.N
    mean = sh[None, :] + S1 / N
    var = (S2 - S1 * S1 / N) / (N - 1)
    _check_moments(mean, var, ref["mean"], ref["var"], sc.n)


def test_per_sample_kernel_refuses_large_systems(fmc):
    sc = fs.multimachine_case(n=20, d=2, K=10, T=0.1, dt=0.005, N=64)
    fmc.set_kernel_policy("per_sample")
    try:
        with pytest.raises(fmc.FastMCError) as e:
            fmc.simulate(sc)
        assert e.value.code == 8
    finally:
        fmc.set_kernel_policy("auto")


def test_wide_plain_path_is_refused(fmc):
    sc = fs.multimachine_case(n=20, d=2, K=10, T=0.1, dt=0.005, N=64)
    with pytest.raises(fmc.FastMCError) as e:
        fmc.simulate(sc, path="plain")
    assert e.value.code == 8


def test_wide_in_a_batch(fmc):
    scs = [fs.multimachine_case(n=3, d=1, K=50, T=0.5, dt=0.005, N=300, seed=31),
           fs.multimachine_case(n=45, d=6, K=60, T=0.4, dt=0.005, N=1000, seed=32),
           fs.multimachine_case(n=10, d=3, K=200, T=0.5, dt=0.005, N=700, seed=33),
           fs.multimachine_case(n=21, d=8, K=20, T=0.25, dt=0.005, N=129, seed=34)]
    b = fmc.Batch(scs, use_graph=True)
    means, vars_ = b.launch()
    fmc.device_status()
    for sc, m, v in zip(scs, means, vars_):
        # the kernel the batch takes for this scenario on a shared GPU
        fmc.set_kernel_policy("per_sample" if sc.n <= 16 else "split_tc")
        m1, v1 = fmc.simulate(sc, path="fused", precision="bf16x3")
        fmc.set_kernel_policy("auto")
        # FP32 merge of tile groups in a single call, FP64 tile sums in the batch:
        # equal to FP32 rounding on the scale of the spread
        mm, vv, mm1, vv1 = m.cpu().numpy(), v.cpu().numpy(), m1.cpu().numpy(), v1.cpu().numpy()
        for sl in (slice(0, sc.n), slice(sc.n, 2 * sc.n)):
            sd = float(np.sqrt(np.max(vv1[:, sl])))
            assert np.max(np.abs(mm[:, sl] - mm1[:, sl])) <= 1e-6 * sd + 1e-15
            assert np.allclose(vv[:, sl], vv1[:, sl], rtol=2e-6, atol=1e-18)
    b.close()


@pytest.mark.parametrize("n,d", [(13, 2), (18, 3), (20, 3), (20, 8), (21, 7), (23, 2), (24, 6), (26, 4), (28, 3),
                                 (50, 3), (52, 8)])
def test_tensor_core_network_sum_matches_fp32_sum(fmc, n, d):
    # the TF32x3 product drops terms below 2^-21 of each product: the two forms of
    # the same design agree far inside the oracle tolerance
    sc = fs.multimachine_case(n=n, d=d, K=40, T=1.0, dt=0.005, N=300, seed=40 + n)
    out = {}
    for kernel in ("split", "split_tc"):
        fmc.set_kernel_policy(kernel)
        try:
            out[kernel] = fmc.simulate(sc, path="fused", precision="bf16x3", want_traj=True)
        finally:
            fmc.set_kernel_policy("auto")
        fmc.device_status()
    ed, ew = traj_errors(out["split_tc"][2].cpu().numpy(), out["split"][2].cpu().numpy().astype(np.float64), n)
    assert ed <= 1e-5 and ew <= 1e-5, (ed, ew)


def test_tensor_core_network_sum_refuses_small_systems(fmc):
    sc = fs.multimachine_case(n=12, d=2, K=10, T=0.1, dt=0.005, N=64)
    fmc.set_kernel_policy("split_tc")
    try:
        with pytest.raises(fmc.FastMCError) as e:
            fmc.simulate(sc)
        assert e.value.code == 8
    finally:
        fmc.set_kernel_policy("auto")


def _with_infinite_bus(sc, seed):
    """The system tied to an infinite bus (Binf = 2 at every machine), its mechanical
    powers those of a chosen equilibrium, so that no machine is the angle reference
    and the tensor-core kernel takes its deviations unshifted."""
    rng = np.random.default_rng(seed)
    n = sc.n
    d_t = rng.uniform(-0.2, 0.3, n)
    s2 = sc.replace(has_inf_bus=True, Ginf=np.zeros(n), Binf=np.full(n, 2.0), Vinf=1.0)
    V = s2.E * np.exp(1j * d_t)
    current = (s2.G + 1j * s2.B) @ V + (s2.Ginf + 1j * s2.Binf) * s2.Vinf
    return s2.replace(Pm=np.real(V * np.conj(current)))


def _tc_run(fmc, sc, **kw):
    fmc.set_kernel_policy("split_tc")
    try:
        out = fmc.simulate(sc, path="fused", precision="bf16x3", want_traj=True, **kw)
    finally:
        fmc.set_kernel_policy("auto")
    fmc.device_status()
    return out


@pytest.mark.parametrize("n,d,N", [(19, 3, 130), (44, 2, 129)])
def test_tensor_core_split_with_infinite_bus(fmc, orc, n, d, N):
    sc = _with_infinite_bus(fs.multimachine_case(n=n, d=d, K=30, T=0.4, dt=0.005, N=N, seed=60 + n), 70 + n)
    mean, var, traj = _tc_run(fmc, sc)
    ref = orc.simulate(sc, orc.lhs_sample(sc.seed, sc.N, sc.M), want_traj=True, nthreads=8)
    ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
    assert ed <= 1e-4 and ew <= 1e-4, (ed, ew)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)


@pytest.mark.parametrize("n,d", [(20, 2), (36, 5)])
def test_tensor_core_split_traditional_monte_carlo(fmc, orc, n, d):
    # per-step normals drawn in the chunk pass (Section V-B's comparator)
    sc = fs.multimachine_case(n=n, d=d, K=20, T=0.3, dt=0.005, N=140, seed=90 + n).replace(sampling=fs.SRS_EM)
    mean, var, traj = _tc_run(fmc, sc)
    ref = orc.simulate_em(sc, want_traj=True, nthreads=8)
    ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
    assert ed <= 1e-4 and ew <= 1e-4, (ed, ew)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)


def test_tensor_core_split_heun_two_warps_per_sample(fmc, orc):
    sc = fs.multimachine_case(n=19, d=4, K=30, T=0.4, dt=0.005, N=131, seed=95).replace(integrator=fs.HEUN)
    mean, var, traj = _tc_run(fmc, sc)
    ref = orc.simulate(sc, orc.lhs_sample(sc.seed, sc.N, sc.M), want_traj=True, nthreads=8)
    ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
    assert ed <= 1e-4 and ew <= 1e-4, (ed, ew)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)


def test_tensor_core_split_sample_blocks_add_up(fmc, orc):
    # two warps per sample (20 machines): blocks of the design through the sums
    # entry point give the whole design's moments
    sc = fs.multimachine_case(n=20, d=3, K=30, T=0.3, dt=0.005, N=300, seed=97)
    ref = orc.simulate(sc, orc.lhs_sample(sc.seed, sc.N, sc.M), nthreads=8)
    fmc.set_kernel_policy("split_tc")
    try:
        a1, a2, shift = fmc.simulate_sums(sc, 0, 131)
        b1, b2, _ = fmc.simulate_sums(sc, 131, sc.N - 131)
    finally:
        fmc.set_kernel_policy("auto")
    S1 = (a1 + b1).cpu().numpy()
    S2 = (a2 + b2).cpu().numpy()
    N = sc.N
    mean = shift.cpu().numpy()[None, :] + S1 / N
    var = (S2 - S1 * S1 / N) / (N - 1)
    _check_moments(mean, var, ref["mean"], ref["var"], sc.n)


def test_infinite_bus_without_a_free_slot(fmc, orc):
    # 20 machines fill every slot of both tensor-core layouts: the automatic choice
    # takes the FP32 split kernel, a forced tensor-core kernel is refused
    sc = _with_infinite_bus(fs.multimachine_case(n=20, d=2, K=30, T=0.3, dt=0.005, N=130, seed=98), 99)
    mean, var, traj = fmc.simulate(sc, path="fused", precision="bf16x3", want_traj=True)
    fmc.device_status()
    ref = orc.simulate(sc, orc.lhs_sample(sc.seed, sc.N, sc.M), want_traj=True, nthreads=8)
    ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
    assert ed <= 1e-4 and ew <= 1e-4, (ed, ew)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)
    fmc.set_kernel_policy("split_tc")
    try:
        with pytest.raises(fmc.FastMCError) as e:
            fmc.simulate(sc)
        assert e.value.code == 8
    finally:
        fmc.set_kernel_policy("auto")


def test_two_warps_per_sample_with_a_trip_event(fmc, orc):
    # 4 disturbances and a generator trip fill the 8-slot bucket, which the 13-slot
    # two-warp layout is not built for: the four-warp layout takes the system
    sc = fs.multimachine_case(n=25, d=4, K=20, T=0.3, dt=0.005, N=130, seed=99).replace(
        event_machine=3, event_time=0.1, event_dpm=-0.5)
    mean, var, traj = _tc_run(fmc, sc)
    ref = orc.simulate(sc, orc.lhs_sample(sc.seed, sc.N, sc.M), want_traj=True, nthreads=8)
    ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
    assert ed <= 1e-4 and ew <= 1e-4, (ed, ew)
    _check_moments(mean.cpu().numpy(), var.cpu().numpy(), ref["mean"], ref["var"], sc.n)
