"""Launch-shape rules (what the autotuner writes): any rule's shape -- kernel,
resident CTAs per SM, time chunk -- gives the oracle's trajectories and moments
within the usual tolerances, malformed rules are refused, and the rule table
is matched by machines, disturbances and samples."""
import numpy as np
import pytest

import fmc_synth as fs
from gpu_common import need_gpu, traj_errors

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kernel,max_ctas,TC", [(1, 1, 16), (1, 2, 32), (1, 4, 16), (2, 0, 16), (1, 0, 0)])
def test_rule_shapes_match_the_oracle(orc, kernel, max_ctas, TC):
    fmc = need_gpu()
    ctx = fmc.Context(0)
    try:
        sc = fs.multimachine_case(n=10, d=3, K=40, T=0.305, dt=0.005, N=300, seed=81)
        fmc.set_launch_rules([dict(n_min=5, n_max=12, d_min=2, d_max=4, kernel=kernel, max_ctas=max_ctas, TC=TC),
                              dict(kernel=2, TC=64)], ctx=ctx)
        mean, var, traj = fmc.simulate(sc, want_traj=True, ctx=ctx)
        fmc.device_status(ctx)
        ref = orc.simulate(sc, orc.lhs_sample(sc.seed, sc.N, sc.M), want_traj=True, nthreads=8)
        ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
        assert ed <= 1e-4 and ew <= 1e-4, (ed, ew)
        m, v = mean.cpu().numpy(), var.cpu().numpy()
        n = sc.n
        for sl in (slice(0, n), slice(n, 2 * n)):
            scale = np.max(np.sqrt(ref["mean"][:, sl] ** 2 + ref["var"][:, sl]))
            assert np.max(np.abs(m[:, sl] - ref["mean"][:, sl])) <= 1e-5 * scale
            assert np.max(np.abs(v[:, sl] - ref["var"][:, sl])) <= 1e-5 * np.max(np.abs(ref["var"][:, sl]))
    finally:
        ctx.close()


def test_malformed_rules_are_refused():
    fmc = need_gpu()
    ctx = fmc.Context(0)
    try:
        for bad in (dict(n_min=5, n_max=4), dict(kernel=4), dict(max_ctas=5), dict(TC=48), dict(TC=512)):
            with pytest.raises(fmc.FastMCError) as e:
                fmc.set_launch_rules([bad], ctx=ctx)
            assert e.value.code == fmc.EINVAL
        fmc.set_launch_rules([], ctx=ctx)
    finally:
        ctx.close()


def test_rule_kernel_that_cannot_take_the_system_is_ignored():
    # a bucket's rule is measured at its largest machine count: a tensor-core
    # split rule over 11..16 machines leaves 11 machines to the library's choice
    fmc = need_gpu()
    ctx = fmc.Context(0)
    try:
        sc = fs.multimachine_case(n=11, d=2, K=30, T=0.2, dt=0.005, N=200, seed=83)
        fmc.set_launch_rules([], ctx=ctx)
        m0, v0 = fmc.simulate(sc, ctx=ctx)
        fmc.set_launch_rules([dict(n_min=11, n_max=16, kernel=3)], ctx=ctx)
        m1, v1 = fmc.simulate(sc, ctx=ctx)
        fmc.device_status(ctx)
        assert np.array_equal(m0.cpu().numpy(), m1.cpu().numpy())
        assert np.array_equal(v0.cpu().numpy(), v1.cpu().numpy())
        # from 13 machines the rule's kernel takes the system
        sc = fs.multimachine_case(n=14, d=2, K=30, T=0.2, dt=0.005, N=200, seed=84)
        fmc.simulate(sc, ctx=ctx)
        fmc.device_status(ctx)
    finally:
        fmc.set_launch_rules([], ctx=ctx)
        ctx.close()
