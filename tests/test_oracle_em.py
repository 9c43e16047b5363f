"""Pins for the oracle's "traditional Monte Carlo" comparator (Section V-B): the
disturbance advanced by the scheme of Eq. (distito) with a fresh standard normal
per step, dW = sqrt(dt) zeta, the normals drawn from Philox4x32-10.

Fixed by definitions outside the oracle: the counter layout (Philox word
through scipy's ndtri, an independent inverse normal CDF); iid N(0, dt)
increments (moments and correlations within sampling error); the exact variance
of the EM recursion for the OU process, sigma^2 dt sum_m (1 - theta dt)^(2m).
"""
import numpy as np
import pytest
from scipy.special import ndtri

import fmc_synth as fs


@pytest.mark.parametrize("seed,k,w,n", [(0, 0, 0, 0), (7, 12345, 3, 999), (2**40 + 5, 65535, 5, 17),
                                        (123, 3, 7, 4000)])
def test_em_normal_is_philox_word_through_inverse_cdf(orc, seed, k, w, n):
    ctr = [k & 0xFFFFFFFF, n, 256, w // 4]
    key = [seed & 0xFFFFFFFF, seed >> 32]
    r = int(orc.philox4x32_10(ctr, key)[w % 4])
    u = (r + 0.5) / 2.0**32
    z = orc.em_normal(seed, k, w, n)
    assert abs(z - ndtri(u)) <= 1e-13 * max(1.0, abs(z))


def test_em_increments_are_iid_normal_with_variance_dt():
    import oracle as orc
    count, d, Nt, dt = 4000, 3, 64, 0.02
    dW = orc.em_increments(11, 0, count, d, Nt, dt)
    x = dW.reshape(count, -1) / np.sqrt(dt)
    m = x.size
    assert abs(x.mean()) < 5 / np.sqrt(m)
    assert abs(x.var() - 1.0) < 5 * np.sqrt(2.0 / m)
    # no correlation across disturbances, steps or samples
    c = np.corrcoef(x[:, :8].T)
    assert np.max(np.abs(c - np.eye(8))) < 5 / np.sqrt(count)
    assert abs(np.corrcoef(x[:-1, 0], x[1:, 0])[0, 1]) < 5 / np.sqrt(count)
    # sub-ranges are slices of the whole design
    part = orc.em_increments(11, 100, 50, d, Nt, dt)
    assert np.array_equal(part, dW[100:150])


def test_em_ou_variance_is_the_scheme_closed_form(orc):
    count, Nt, dt, theta, sigma = 20000, 200, 0.01, 1.0, 0.05
    dW = orc.em_increments(5, 0, count, 1, Nt, dt)[:, 0, :]
    x = orc.ou_em(dW, dt, theta, sigma)
    a = 1.0 - theta * dt
    n = np.arange(Nt + 1)
    exact = sigma**2 * dt * (1 - a ** (2 * n)) / (1 - a**2)
    v = x.var(axis=0, ddof=1)
    # sampling error of a variance estimate: sqrt(2/(N-1)) relative
    assert np.max(np.abs(v[1:] / exact[1:] - 1)) < 5 * np.sqrt(2.0 / (count - 1))
    assert np.max(np.abs(x.mean(axis=0)[1:]) / np.sqrt(exact[1:])) < 5 / np.sqrt(count)


def test_simulate_em_uses_those_increments(orc):
    sc = fs.multimachine_case(n=4, d=2, K=10, T=0.2, dt=0.005, N=64, seed=3)
    r = orc.simulate_em(sc, k0=10, count=20, want_dW=True, want_traj=True)
    assert np.array_equal(r["dW"], orc.em_increments(sc.seed, 10, 20, sc.d, sc.Nt, sc.dt))
    # the same increments through the KL entry point's integrator give the same paths:
    # sigma = 0 removes the noise, so both start and stay at the equilibrium
    z = orc.simulate_em(sc.replace(sigma=np.zeros(2)), count=4, want_traj=True)["traj"]
    d0, _, _ = orc.equilibrium(sc)
    assert np.max(np.abs(z[:, :, :4] - d0)) < 1e-12
