"""Pins for the oracle's general one-dimensional Ito disturbances (Section II,
Table I; the wind model of Eq. windito).

Fixed by the mathematics: with per-step normal increments the scheme samples the
Ito process, whose stationary laws are the densities Table I names (Gaussian,
Beta, Gamma, Laplace: their means and variances in closed form); paths driven by
the increments of a smooth (KL) expansion converge to the Stratonovich solution,
whose drift differs by sigma sigma'/2 (Wong-Zakai): with the correction term the
KL-driven Gamma process keeps the Ito mean a/b, without it the mean moves by
1/(2b); and an Ornstein-Uhlenbeck process written in the general form gives the
same system trajectories as the built-in one.
"""
import numpy as np
import pytest

import fmc_synth as fs


def _stationary(orc, spec, seed=0, S=20000, Nt=3000, dt=0.005, burn=1000):
    rng = np.random.default_rng(seed)
    dW = rng.standard_normal((S, Nt)) * np.sqrt(dt)
    x = orc.ito_paths(spec, dW, dt, stratonovich=False)[:, burn:]
    return x.mean(), x.var()


@pytest.mark.parametrize("name,spec,mean,var", [
    ("gaussian", fs.ito_gaussian(0.3, 0.02), 0.3, 0.02),
    ("beta", fs.ito_beta(2.0, 3.0), 2.0 / 5.0, 6.0 / (25.0 * 6.0)),
    ("gamma", fs.ito_gamma(2.0, 2.0), 1.0, 0.5),
    ("laplace", fs.ito_laplace(0.3, 0.2), 0.3, 2 * 0.2**2),
])
def test_stationary_law_of_table_one(orc, name, spec, mean, var):
    m, v = _stationary(orc, spec)
    # sampling (correlation time 1 s over 10 s, 2e4 paths) and O(dt) discretisation
    assert abs(m - mean) < 0.01 * np.sqrt(var) * 10
    assert abs(v / var - 1) < 0.03


def test_kl_paths_need_the_stratonovich_correction(orc):
    a, b = 2.0, 2.0
    spec = fs.ito_gamma(a, b)
    S, K, T, Nt = 1000, 300, 4.0, 2000
    dt = T / Nt
    z = orc.lhs_sample(5, S, K, mode=1)          # simple random sampling of the KL coefficients
    dW = orc.kle_reconstruct(z, 1, K, T, Nt)[:, 0, :]
    t0 = T / 8
    corr = orc.ito_paths(spec, dW, dt, stratonovich=True)[:, Nt // 8:].mean()
    raw = orc.ito_paths(spec, dW, dt, stratonovich=False)[:, Nt // 8:].mean()
    # corrected: started at the Ito mean, stays there
    assert abs(corr - a / b) < 0.05
    # uncorrected: the drift is higher by sigma sigma'/2 = 1/(2b) (constant for the
    # Gamma law), so the mean relaxes (unit rate) from a/b to a/b + 1/(2b); the
    # difference of the two time averages over [t0, T] on the same paths is
    shift = 1.0 / (2.0 * b) * (1.0 - (np.exp(-t0) - np.exp(-T)) / (T - t0))
    assert abs((raw - corr) - shift) < 0.01


def test_ou_in_general_form_matches_the_builtin_ou(orc):
    sc = fs.multimachine_case(n=5, d=2, K=30, T=0.5, dt=0.005, N=16, seed=4)
    sc = sc.replace(theta=np.array([1.0, 1.0]))
    specs = [fs.ito_gaussian(0.0, s**2 / 2.0) for s in sc.sigma]
    z = orc.lhs_sample(sc.seed, sc.N, sc.M)
    a = orc.simulate(sc, z, want_traj=True)["traj"]
    # the KL-driven general form subtracts sigma sigma'/2 = 0 for a constant sigma
    b = orc.simulate(sc.replace(ito=specs), z, want_traj=True)["traj"]
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_wind_model_start_is_the_stable_root(orc):
    w = fs.ito_wind()
    m0, m1, m2 = w["m"]
    x0 = w["x0"]
    assert abs(m0 + m1 * x0 + m2 * x0**2) < 1e-12
    assert m1 + 2 * m2 * x0 < 0
