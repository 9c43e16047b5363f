"""Pins of the oracle's smooth-forcing form: the disturbance as the random ODE of
Eq. (eqkl), dx/dt = mu(x) + sigma(x) sum_k zeta_k m_k(t), integrated jointly with
the swing equations by the same RK4 (or Heun) stages.

What fixes it independently of the oracle's own arithmetic:
* the forcing basis m_k is the time derivative of the KL basis: Simpson's rule
  over a step reproduces the increment basis (an independent routine) to O(dt^5);
* for the OU disturbance a single basis function drives a linear ODE whose
  solution is a closed form (sine basis; the paper's cosine basis, constant
  first function included);
* RK4 converges at order 4 and Heun at order 2 on it, and the coupled swing +
  disturbance system keeps order 4 (a stage fed the wrong disturbance value
  would drop it to 2);
* linearity: any coefficient vector gives the sum of the single-mode responses;
* the Euler-Maruyama form on the same path's increments converges to it at order 1
  (OU, and a general Ito disturbance with the Stratonovich drift on both sides).
"""
import math

import numpy as np
import pytest

import fmc_synth as fs
import oracle as orc


def _ou_case(T=10.0, dt=0.01, K=20, theta=1.0, sigma=0.05, basis=fs.BASIS_SINE, integrator=fs.RK4):
    return fs.smib_case(N=1, K=K, T=T, dt=dt, theta=theta, sigma=sigma).replace(
        forcing=fs.FORCING_SMOOTH, basis=basis, integrator=integrator)


def _mode(K, k):
    z = np.zeros((1, K))
    z[0, k] = 1.0
    return z


def _closed_form(t, theta, sigma, a, c):
    """x(t) of dx/dt = -theta x + sigma c cos(a t), x(0) = 0."""
    return sigma * c * (theta * np.cos(a * t) + a * np.sin(a * t) - theta * np.exp(-theta * t)) / (theta ** 2 + a ** 2)


@pytest.mark.parametrize("basis", [fs.BASIS_SINE, fs.BASIS_COSINE])
def test_forcing_basis_integrates_to_the_increment_basis(basis):
    K, T, Nt = 50, 10.0, 1000
    mdot = orc.kl_forcing_basis(K, T, Nt, basis)
    phi = orc.kl_increment_basis(K, T, Nt, basis)
    dt = T / Nt
    simpson = dt / 6.0 * (mdot[:, 0:-1:2] + 4.0 * mdot[:, 1::2] + mdot[:, 2::2])
    assert simpson.shape == phi.shape
    # Simpson's error dt^5 |m''''| / 2880 <= dt^5 a_K^4 sqrt(2/T) / 2880 (< 1e-9 here)
    assert np.max(np.abs(simpson - phi)) < 2e-9


@pytest.mark.parametrize("k", [0, 2, 7])
def test_single_sine_mode_matches_the_closed_form(k):
    sc = _ou_case()
    x = orc.smooth_paths(sc, _mode(sc.K, k))[0]
    t = np.arange(sc.Nt + 1) * sc.dt
    a = (k + 0.5) * math.pi / sc.T
    ref = _closed_form(t, 1.0, 0.05, a, math.sqrt(2.0 / sc.T))
    assert np.max(np.abs(x - ref)) <= 1e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("j", [0, 1, 5])
def test_single_cosine_mode_matches_the_closed_form(j):
    sc = _ou_case(basis=fs.BASIS_COSINE)
    x = orc.smooth_paths(sc, _mode(sc.K, j))[0]
    t = np.arange(sc.Nt + 1) * sc.dt
    if j == 0:
        ref = 0.05 / math.sqrt(sc.T) * (1.0 - np.exp(-t))   # m_1 = 1 / sqrt(T): a constant forcing
    else:
        ref = _closed_form(t, 1.0, 0.05, j * math.pi / sc.T, math.sqrt(2.0 / sc.T))
    assert np.max(np.abs(x - ref)) <= 1e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("integrator,order", [(fs.RK4, 4), (fs.HEUN, 2)])
def test_order_of_the_disturbance_step(integrator, order):
    k, T, theta = 4, 2.0, 1.0
    a = (k + 0.5) * math.pi / T
    errs = []
    for dt in (0.04, 0.02, 0.01):
        sc = _ou_case(T=T, dt=dt, K=8, integrator=integrator)
        x = orc.smooth_paths(sc, _mode(sc.K, k))[0]
        errs.append(abs(x[-1] - _closed_form(T, theta, 0.05, a, math.sqrt(2.0 / T))))
    for e0, e1 in zip(errs, errs[1:]):
        assert 2 ** order * 0.75 < e0 / e1 < 2 ** order * 1.25, errs


def test_linearity_in_the_coefficients():
    sc = _ou_case(K=12)
    rng = np.random.default_rng(3)
    z = rng.standard_normal((1, sc.K))
    x = orc.smooth_paths(sc, z)[0]
    modes = orc.smooth_paths(sc, np.eye(sc.K))
    ref = z[0] @ modes
    assert np.max(np.abs(x - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_the_increment_form_converges_to_it():
    # Euler-Maruyama on the increments of the same truncated path (order 1) against
    # the random ODE (order 4): the gap halves with dt
    gaps = []
    for dt in (0.02, 0.01, 0.005):
        sc = _ou_case(T=4.0, dt=dt, K=10)
        z = np.random.default_rng(5).standard_normal((1, sc.K))
        xs = orc.smooth_paths(sc, z)[0]
        dW = orc.kle_reconstruct(z, 1, sc.K, sc.T, sc.Nt)[:, 0, :]
        xe = orc.ou_em(dW, dt, 1.0, 0.05)[0]
        gaps.append(np.max(np.abs(xe - xs)))
    for g0, g1 in zip(gaps, gaps[1:]):
        assert 1.6 < g0 / g1 < 2.4, gaps


def test_general_ito_disturbance_agrees_with_the_increment_form():
    # a Gamma process of Table I: both forms carry the Stratonovich drift on a KL path
    spec = fs.ito_gamma(2.0, 4.0)
    gaps = []
    for dt in (0.02, 0.01, 0.005):
        sc = _ou_case(T=4.0, dt=dt, K=10).replace(ito=[spec])
        z = 0.5 * np.random.default_rng(7).standard_normal((1, sc.K))
        xs = orc.smooth_paths(sc, z)[0]
        dW = orc.kle_reconstruct(z, 1, sc.K, sc.T, sc.Nt)[:, 0, :]
        xe = orc.ito_paths(spec, dW, dt, stratonovich=True)[0]
        gaps.append(np.max(np.abs(xe - xs)))
    for g0, g1 in zip(gaps, gaps[1:]):
        assert 1.5 < g0 / g1 < 2.5, gaps


def test_coupled_system_keeps_rk4_order():
    # the swing stages see the disturbance's own RK4 stage values: delta(T) converges
    # at order 4 (Richardson ratio 16); midpoint averages instead would give order 2
    finals = []
    z = None
    for dt in (0.02, 0.01, 0.005, 0.0025):
        sc = fs.multimachine_case(n=3, d=2, K=6, T=1.0, dt=dt, N=1, seed=11).replace(
            forcing=fs.FORCING_SMOOTH, sigma=np.array([0.6, 0.8]))
        if z is None:
            z = np.random.default_rng(13).standard_normal((1, sc.d * sc.K))
        out = orc.simulate(sc, z, want_traj=True, want_moments=False)
        finals.append(out["traj"][0, -1, :])
    d = [np.max(np.abs(finals[i] - finals[i + 1])) for i in range(3)]
    assert 12.0 < d[0] / d[1] < 20.0 and 12.0 < d[1] / d[2] < 20.0, d


def test_smooth_form_refuses_per_step_normals():
    sc = fs.multimachine_case(n=3, d=1, K=4, T=0.1, dt=0.01, N=2, seed=1).replace(forcing=fs.FORCING_SMOOTH)
    with pytest.raises(RuntimeError):
        orc.simulate_em(sc)
