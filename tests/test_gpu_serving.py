"""The request server on the GPU: results alone and in the mix, timeouts,
cancellation and memory admission.  Failures are made on the host (a wait that
runs out, a cancelled request, an over-budget request); nothing faults the GPU."""
import time

import numpy as np
import pytest

import fmc_synth as fs
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fmc():
    return need_gpu()


def _mix():
    return [fs.multimachine_case(n=10, d=3, K=200, T=2.0, dt=0.005, N=20000, seed=21),
            fs.multimachine_case(n=4, d=2, K=60, T=1.0, dt=0.005, N=3000, seed=22),
            fs.smib_case(N=1000, T=5.0),
            fs.multimachine_case(n=16, d=8, K=100, T=0.5, dt=0.005, N=5000, seed=23),
            fs.multimachine_case(n=7, d=1, K=250, T=1.5, dt=0.005, N=65536, seed=24),
            fs.multimachine_case(n=3, d=4, K=33, T=0.3, dt=0.005, N=129, seed=25)]


def _same_within_rounding(m, v, m0, v0, n):
    """Alone and in the mix: the same samples, kernel and per-sample arithmetic;
    only the width of the time chunk can differ (a launch that has the GPU alone
    sizes it from the free TMEM, a shared one does not), which may change the
    tensor cores' accumulation order of the contraction in the last FP32 bit.
    Means within 1e-6 of the variable's RMS size, variances within the stated
    moment tolerance (1e-5 normwise)."""
    for sl in (slice(0, n), slice(n, 2 * n)):
        scale = np.max(np.sqrt(m0[:, sl] ** 2 + v0[:, sl]))
        assert np.max(np.abs(m[:, sl] - m0[:, sl])) <= 1e-6 * scale
        assert np.max(np.abs(v[:, sl] - v0[:, sl])) <= 1e-5 * np.max(np.abs(v0[:, sl]))


def test_results_same_alone_and_in_the_mix(fmc):
    scs = _mix()
    # alone: the same kernel as the server's (a shared GPU takes the per-sample
    # kernel for these sizes)
    fmc.set_kernel_policy("per_sample")
    try:
        alone = [fmc.simulate(sc, path="fused", precision="bf16x3") for sc in scs]
    finally:
        fmc.set_kernel_policy("auto")
    srv = fmc.Server(slots=4)
    handles = [srv.submit(sc) for sc in scs + scs]  # two copies of each, all in flight together
    for i, h in enumerate(handles):
        res, m, v = srv.wait(h, timeout_s=120)
        assert res["status"] == 0, res
        m0, v0 = alone[i % len(scs)]
        _same_within_rounding(m.cpu().numpy(), v.cpu().numpy(), m0.cpu().numpy(), v0.cpu().numpy(),
                              scs[i % len(scs)].n)
        assert res["latency_us"] >= res["queue_us"] >= 0
    srv.close()


def test_wait_timeout_and_poll(fmc):
    srv = fmc.Server(slots=1)
    big = fs.multimachine_case(n=10, d=3, K=200, T=20.0, dt=0.005, N=1 << 16, seed=5)
    h = srv.submit(big)
    assert srv.wait(h, timeout_s=1e-6) is None          # FMC_ETIMEOUT: not done yet
    t0 = time.time()
    while srv.poll(h) is None:
        assert time.time() - t0 < 120
        time.sleep(0.01)
    srv.close()


def test_cancel_queued_request(fmc):
    srv = fmc.Server(slots=1)
    # the first request runs for about two seconds on one slot, so the second
    # is still queued when it is cancelled
    first = srv.submit(fs.multimachine_case(n=10, d=3, K=200, T=60.0, dt=0.005, N=1 << 20, seed=6))
    second = srv.submit(fs.smib_case(N=1000))
    time.sleep(0.05)
    assert srv.cancel(second) == fmc.OK
    res, _, _ = srv.wait(second, timeout_s=10)
    assert res["status"] == fmc.ECANCELLED
    res, _, _ = srv.wait(first, timeout_s=120)
    assert res["status"] == 0
    srv.close()


def test_memory_admission(fmc):
    sc = fs.multimachine_case(n=10, d=3, K=200, T=2.0, dt=0.005, N=1 << 15, seed=7)
    need = 2 * sc.N * sc.d * 200 * 2  # the split design alone
    srv = fmc.Server(slots=4, mem_budget_bytes=int(need * 1.5))
    with pytest.raises(fmc.FastMCError) as e:
        srv.submit(sc.replace(N=1 << 17))               # could never fit the budget
    assert e.value.code == fmc.ENOMEM
    hs = [srv.submit(sc) for _ in range(3)]             # fit one at a time
    peak = 0
    done = 0
    t0 = time.time()
    while done < 3:
        st = srv.stats()
        peak = max(peak, st["running"])
        for h in list(hs):
            r = srv.poll(h)
            if r is not None:
                assert r[0]["status"] == 0
                hs.remove(h)
                done += 1
        assert time.time() - t0 < 120
        time.sleep(0.002)
    assert peak <= 1
    srv.close()


def test_target_error_request(fmc):
    # four independent designs, growing until their spread meets the targets;
    # the pooled moments are then that close to a large independent reference
    sc = fs.multimachine_case(n=10, d=3, K=200, T=2.0, dt=0.005, N=64, seed=31)
    srv = fmc.Server(slots=2)
    tol_E, tol_Var = 2e-3, 2e-2
    h = srv.submit(sc, tol_E=tol_E, tol_Var=tol_Var, max_N=1 << 18)
    res, m, v = srv.wait(h, timeout_s=120)
    srv.close()
    assert res["status"] == 0, res
    assert res["target_met"] and res["replicates"] == 4
    assert res["err_E"] <= tol_E and res["err_Var"] <= tol_Var
    assert res["n_used"] % 4 == 0 and res["n_used"] >= 4 * 64
    mr, vr = fmc.simulate(sc.replace(N=1 << 17, seed=999), path="fused", precision="bf16x3")
    mr, vr, m, v = mr.cpu().numpy(), vr.cpu().numpy(), m.cpu().numpy(), v.cpu().numpy()
    # the replicate spread of four designs is itself uncertain: a factor 5
    assert np.max(np.abs(m - mr)) / np.sqrt(vr.max()) <= 5 * tol_E
    assert np.max(np.abs(v - vr)) / vr.max() <= 5 * tol_Var


def test_target_error_request_stops_at_max_n(fmc):
    sc = fs.multimachine_case(n=4, d=2, K=50, T=0.5, dt=0.005, N=64, seed=32)
    srv = fmc.Server(slots=1)
    h = srv.submit(sc, tol_E=1e-9, max_N=1024)      # unreachable: 64 -> 256 per design, then 4 x 4 x 256 > 1024
    res, m, v = srv.wait(h, timeout_s=60)
    assert res["status"] == 0 and not res["target_met"]
    assert res["n_used"] == 1024 and res["err_E"] > 1e-9
    assert np.all(np.isfinite(m.cpu().numpy())) and np.all(np.isfinite(v.cpu().numpy()))
    with pytest.raises(fmc.FastMCError) as e:
        srv.submit(sc, tol_E=1e-3, max_N=100)         # below four designs of N samples
    assert e.value.code == fmc.EINVAL
    srv.close()


def _mix64(x):
    """splitmix64's finaliser (the server's replicate seeds)."""
    m = (1 << 64) - 1
    x = (x + 0x9E3779B97F4A7C15) & m
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & m
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & m
    return x ^ (x >> 31)


@pytest.mark.parametrize("n", [10, 20])
def test_round_of_replicates_in_one_launch(fmc, n):
    # a round's four designs share one launch; its pooled moments are those of
    # the four designs run one by one (seed k: splitmix64 of seed ^ (k + 1) << 32)
    sc = fs.multimachine_case(n=n, d=3, K=50, T=0.5, dt=0.005, N=256, seed=41)
    srv = fmc.Server(slots=1)
    h = srv.submit(sc, tol_E=10.0, tol_Var=10.0, max_N=1 << 14)
    res, m, v = srv.wait(h, timeout_s=60)
    srv.close()
    assert res["status"] == 0 and res["target_met"] and res["n_used"] == 4 * 256
    ms, vs = [], []
    for k in range(4):
        mk, vk = fmc.simulate(sc.replace(seed=_mix64(sc.seed ^ ((k + 1) << 32))), path="fused", precision="bf16x3")
        ms.append(mk.cpu().numpy())
        vs.append(vk.cpu().numpy())
    m0 = ((ms[0] + ms[1]) + ms[2]) + ms[3]
    v0 = ((vs[0] + vs[1]) + vs[2]) + vs[3]
    _same_within_rounding(m.cpu().numpy(), v.cpu().numpy(), m0 / 4, v0 / 4, n)
