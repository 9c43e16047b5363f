"""The device error path of the bounded waits, exercised without a fault.

Every spin of the library's kernels on an mbarrier has an iteration limit; when
it runs out the kernel records a timeout code in a device status word and
returns, and fmc_device_status turns the code into FMC_ETIMEOUT.  The self-check
entry point launches one CTA whose thread waits, with a short limit, on an
mbarrier that nothing arrives at (no bulk copy or MMA in flight), so that path
runs for real; the context stays usable afterwards.
"""
import numpy as np
import pytest

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def test_context_wait_timeout_maps_to_etimeout():
    fmc = need_gpu()
    ctx = fmc.Context(0)
    try:
        fmc.check_wait_path(target=0, poll_limit=1000, ctx=ctx)
        with pytest.raises(fmc.FastMCError) as e:
            fmc.device_status(ctx)
        assert e.value.code == fmc.ETIMEOUT
        # the context still works: a small simulation runs and reports clean
        import fmc_synth as fs
        sc = fs.smib_case(N=64, K=10, T=0.2, dt=0.01)
        m, v = fmc.simulate(sc, ctx=ctx)
        assert fmc.device_status(ctx)[1] == 0
        assert np.all(np.isfinite(m.cpu().numpy()))
    finally:
        ctx.close()


def test_wait_check_refuses_bad_arguments():
    fmc = need_gpu()
    with pytest.raises(fmc.FastMCError) as e:
        fmc.check_wait_path(target=2)
    assert e.value.code == fmc.EINVAL
    with pytest.raises(fmc.FastMCError) as e:
        fmc.check_wait_path(target=0, poll_limit=0)
    assert e.value.code == fmc.EINVAL
