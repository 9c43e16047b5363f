"""Pins for the oracle's moments (Algorithm 1 step 4).

Fixed by numpy's mean/var(ddof=1) on brute-force small inputs, by the agreement
of the two-pass and shifted-sum forms, and by the N = 1 and offset cases.
"""
import numpy as np

import fmc_synth as fs


def test_brute_force_small(orc):
    rng = np.random.default_rng(0)
    for N in range(2, 9):
        x = rng.standard_normal((N, 5)) * 3 + 1
        m, v = orc.moments_twopass(x)
        assert np.allclose(m, x.mean(axis=0), rtol=1e-15, atol=1e-15)
        assert np.allclose(v, x.var(axis=0, ddof=1), rtol=1e-14)


def test_single_sample_variance_is_nan(orc):
    m, v = orc.moments_twopass(np.array([[1.0, 2.0]]))
    assert np.array_equal(m, [1.0, 2.0]) and np.all(np.isnan(v))


def test_large_offset_is_stable(orc):
    rng = np.random.default_rng(1)
    x = 1e8 + rng.standard_normal((1000, 3)) * 1e-3
    _, v = orc.moments_twopass(x)
    assert np.allclose(v, 1e-6, rtol=0.15)
    assert np.allclose(v, (x - 1e8).var(axis=0, ddof=1), rtol=1e-6)


def test_streaming_moments_match_two_pass(orc):
    sc = fs.multimachine_case(n=4, d=2, K=16, T=1.0, dt=0.01, N=64, seed=2)
    zeta = orc.lhs_sample(1, 64, sc.M)
    for threads in (1, 3):
        r = orc.simulate(sc, zeta, want_traj=True, nthreads=threads)
        m2, v2 = orc.moments_twopass(r["traj"])
        assert np.allclose(r["mean"], m2, rtol=1e-13, atol=1e-15)
        assert np.allclose(r["var"], v2, rtol=1e-9, atol=1e-20)
