"""Pins for the oracle's disturbance and swing dynamics.

Fixed by closed forms and library routines, not by the oracle:
* OU (Table I, Gaussian row): Var x(t) = sigma^2/(2 theta) (1 - exp(-2 theta t)),
  approached by the EM scheme driven by KL increments as K grows and dt shrinks;
* electrical power: the real part of the complex power S = V conj(Y V);
* equilibrium: the SMIB closed form asin(Pm X / (E V)), a planted operating
  point, and scipy's root finder;
* an undisturbed equilibrium stays constant;
* RK4 is fourth order (against scipy's DOP853 at tight tolerance);
* linear regime: the differential Lyapunov equation (Van Loan, scipy expm) and
  the stationary algebraic Lyapunov equation of the linearised single machine
  plus OU state, against the exact variance of the oracle's scheme (its linear
  response to each KL coefficient) and against its Monte Carlo moments.
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.linalg import expm, solve_continuous_lyapunov
from scipy.optimize import fsolve

import fmc_synth as fs


def complex_power(sc, delta):
    """Pe_i = Re(V_i conj(I_i)), I = Y V, V_i = E_i exp(j delta_i) (+ infinite bus)."""
    Y = sc.G + 1j * sc.B
    V = sc.E * np.exp(1j * np.asarray(delta))
    I = Y @ V
    if sc.has_inf_bus:
        I = I + (sc.Ginf + 1j * sc.Binf) * sc.Vinf  # branch to the infinite bus at angle 0
    return np.real(V * np.conj(I))


# ----------------------------------------------------------------------------- OU


def test_ou_em_variance_tends_to_closed_form(orc):
    theta, sigma, T = 1.0, 0.05, 10.0
    exact = sigma**2 / (2 * theta) * (1 - np.exp(-2 * theta * T))
    errs = []
    for K, Nt in [(50, 500), (400, 4000), (1600, 16000)]:
        phi = orc.kl_increment_basis(K, T, Nt)
        # x is linear in zeta: the response to the unit coefficient k is the EM path
        # driven by phi[k]; Var x(T) = sum_k x_k(T)^2 for iid unit coefficients
        x = orc.ou_em(phi, T / Nt, theta, sigma)
        errs.append(abs(np.sum(x[:, -1] ** 2) / exact - 1))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 5e-3


def test_ou_mean_reverts_without_noise(orc):
    # sigma = 0: x stays 0; with a unit increment then silence x decays as (1-theta dt)^n
    dW = np.zeros((1, 100))
    dW[0, 0] = 1.0
    x = orc.ou_em(dW, 0.01, 2.0, 1.0)
    assert np.allclose(x[0, 1:], (1 - 0.02) ** np.arange(100), rtol=1e-14)


# ----------------------------------------------------------------------------- Pe


@pytest.mark.parametrize("case", ["smib", "mm10", "mm4"])
def test_electrical_power_is_complex_power(orc, case):
    sc = {"smib": fs.smib_case(), "mm10": fs.multimachine_case(), "mm4": fs.multimachine_case(n=4, seed=3)}[case]
    rng = np.random.default_rng(1)
    for _ in range(5):
        delta = rng.uniform(-1.5, 1.5, size=sc.n)
        ref = complex_power(sc, delta)
        assert np.allclose(orc.electrical_power(sc, delta, orc.PE_PAIRWISE), ref, rtol=1e-13, atol=1e-12)
        assert np.allclose(orc.electrical_power(sc, delta, orc.PE_PRODUCT), ref, rtol=1e-13, atol=1e-12)


# ----------------------------------------------------------------------------- equilibrium


def test_smib_equilibrium_closed_form(orc):
    sc = fs.smib_case()
    delta0, pm_eq, it = orc.equilibrium(sc)
    assert abs(delta0[0] - math.asin(0.8 * 0.5 / (1.1 * 1.0))) < 1e-14
    assert pm_eq[0] == 0.8


def test_multimachine_equilibrium_residual_and_planted_point(orc):
    sc = fs.multimachine_case(n=10, seed=5)
    delta0, pm_eq, it = orc.equilibrium(sc)
    assert delta0[0] == 0.0 and np.array_equal(pm_eq[1:], sc.Pm[1:])
    assert np.max(np.abs(complex_power(sc, delta0) - pm_eq)) < 1e-12
    # planted operating point: Pm := Pe(delta*) must be recovered from a flat start
    rng = np.random.default_rng(2)
    planted = np.concatenate([[0.0], rng.uniform(-0.5, 0.5, size=sc.n - 1)])
    sc2 = sc.replace(Pm=complex_power(sc, planted))
    d2, p2, _ = orc.equilibrium(sc2)
    assert np.max(np.abs(d2 - planted)) < 1e-10
    assert abs(p2[0] - sc2.Pm[0]) < 1e-10


def test_equilibrium_matches_scipy_root(orc):
    sc = fs.multimachine_case(n=7, seed=8)
    delta0, pm_eq, _ = orc.equilibrium(sc)

    def F(x):
        delta = np.concatenate([[0.0], x])
        return (sc.Pm - complex_power(sc, delta))[1:]

    x = fsolve(F, np.zeros(sc.n - 1), xtol=1e-12)
    assert np.max(np.abs(x - delta0[1:])) < 1e-9


@pytest.mark.parametrize("case", ["smib", "mm"])
def test_undisturbed_equilibrium_stays_constant(orc, case):
    if case == "smib":
        sc = fs.smib_case(N=4)
    else:
        sc = fs.multimachine_case(n=10, d=3, K=20, T=2.0, dt=0.005, N=4)
    sc = sc.replace(sigma=np.zeros(sc.d))
    zeta = orc.lhs_sample(0, 4, sc.M)
    r = orc.simulate(sc, zeta, want_traj=True, want_moments=False)
    traj = r["traj"]
    assert np.max(np.abs(traj[:, :, : sc.n] - r["delta0"])) < 1e-12
    assert np.max(np.abs(traj[:, :, sc.n:])) < 1e-12


# ----------------------------------------------------------------------------- integrator order


def _smib_free_swing(orc, dt, integrator, T=2.0, kick=0.2):
    sc = fs.smib_case(N=1, T=T, dt=dt, K=1).replace(sigma=np.zeros(1))
    d0 = math.asin(0.8 * 0.5 / 1.1)
    r = orc.simulate(sc, np.zeros((1, 1)), want_traj=True, want_moments=False, integrator=integrator,
                     init_delta=[d0 + kick])
    return r["traj"][0, -1]


def _smib_reference(T=2.0, kick=0.2):
    H, D, Pm, Pmax, ws = 5.0, 1.0, 0.8, 1.1 / 0.5, 2 * math.pi * 50
    d0 = math.asin(Pm / Pmax)

    def rhs(t, y):
        return [ws * y[1], (Pm - Pmax * math.sin(y[0]) - D * y[1]) / (2 * H)]

    sol = solve_ivp(rhs, (0, T), [d0 + kick, 0.0], method="DOP853", rtol=1e-13, atol=1e-14)
    return sol.y[:, -1]


@pytest.mark.parametrize("integrator,order", [(0, 4), (1, 2)])
def test_integrator_order(orc, integrator, order):
    ref = _smib_reference()
    errs = []
    for dt in [0.04, 0.02, 0.01]:
        y = _smib_free_swing(orc, dt, integrator)
        errs.append(np.max(np.abs(y - ref) / np.array([1.0, 1e-2])))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 0.7 * 2**order < r1 < 1.4 * 2**order
    assert 0.7 * 2**order < r2 < 1.4 * 2**order


def test_multimachine_rk4_self_convergence(orc):
    sc = fs.multimachine_case(n=5, d=2, K=1, T=1.0, dt=0.01, N=1, seed=4).replace(sigma=np.zeros(2))
    delta0, _, _ = orc.equilibrium(sc)
    init = delta0 + np.linspace(0.05, -0.05, sc.n)
    ends = []
    for dt in [0.01, 0.005, 0.0025, 0.00125]:
        r = orc.simulate(sc.replace(dt=dt), np.zeros((1, sc.M)), want_traj=True, want_moments=False,
                         init_delta=init)
        ends.append(r["traj"][0, -1])
    e1 = np.max(np.abs(ends[0] - ends[1]))
    e2 = np.max(np.abs(ends[1] - ends[2]))
    e3 = np.max(np.abs(ends[2] - ends[3]))
    assert 11 < e1 / e2 < 22 and 11 < e2 / e3 < 22


# ----------------------------------------------------------------------------- linear regime / Lyapunov


def _smib_linear_matrices(H=5.0, D=1.0, E=1.1, V=1.0, X=0.5, Pm=0.8, theta=1.0, sigma=1.0):
    ws = 2 * math.pi * 50
    Pmax = E * V / X
    Ks = Pmax * math.cos(math.asin(Pm / Pmax))
    A = np.array([[0.0, ws, 0.0],
                  [-Ks / (2 * H), -D / (2 * H), 1.0 / (2 * H)],
                  [0.0, 0.0, -theta]])
    Bn = np.array([[0.0], [0.0], [sigma]])
    return A, Bn


def _lyapunov_at(A, Bn, T):
    """P(T) of dP/dt = A P + P A^T + B B^T, P(0) = 0, by Van Loan's matrix exponential."""
    n = A.shape[0]
    M = np.zeros((2 * n, 2 * n))
    M[:n, :n] = -A
    M[:n, n:] = Bn @ Bn.T
    M[n:, n:] = A.T
    E = expm(M * T)
    F22 = E[n:, n:]
    F12 = E[:n, n:]
    return F22.T @ F12


def _scheme_variance(orc, sc, eps):
    """Exact variance of the oracle's scheme in the linear regime: the response to
    each unit KL coefficient (scaled by eps) gives one column of the linear map."""
    K = sc.K
    zeta = np.eye(K) * eps
    r = orc.simulate(sc.replace(N=K), zeta, want_traj=True, want_moments=False, nthreads=8)
    resp = (r["traj"] - np.concatenate([r["delta0"], np.zeros(sc.n)])) / eps
    return np.sum(resp**2, axis=0)  # [Nt+1, 2n]


def test_lyapunov_transient_variance(orc):
    sigma_small = 1e-3
    sc = fs.smib_case(K=400, T=10.0, dt=0.005, sigma=sigma_small)
    var = _scheme_variance(orc, sc, eps=1.0)
    A, Bn = _smib_linear_matrices(sigma=sigma_small)
    P = _lyapunov_at(A, Bn, 10.0)
    assert abs(var[-1, 0] / P[0, 0] - 1) < 0.02
    assert abs(var[-1, 1] / P[1, 1] - 1) < 0.02
    # a truncation below the swing mode (a_K = 3 rad/s < 8 rad/s) is far off (Proposition 1)
    var10 = _scheme_variance(orc, sc.replace(K=10), eps=1.0)
    assert abs(var10[-1, 0] / P[0, 0] - 1) > 5 * abs(var[-1, 0] / P[0, 0] - 1)


def test_lyapunov_stationary_variance(orc):
    sigma_small, D = 1e-3, 10.0
    sc = fs.smib_case(K=400, T=20.0, dt=0.005, sigma=sigma_small, D=D)
    var = _scheme_variance(orc, sc, eps=1.0)
    A, Bn = _smib_linear_matrices(sigma=sigma_small, D=D)
    Pinf = solve_continuous_lyapunov(A, -Bn @ Bn.T)
    assert abs(var[-1, 0] / Pinf[0, 0] - 1) < 0.02
    assert abs(var[-1, 1] / Pinf[1, 1] - 1) < 0.02


def test_monte_carlo_moments_match_exact_scheme_variance(orc):
    sc = fs.smib_case(K=50, T=5.0, dt=0.01, sigma=1e-3)
    var_exact = _scheme_variance(orc, sc, eps=1.0)
    N = 4096
    zeta = orc.lhs_sample(0, N, sc.M)
    r = orc.simulate(sc, zeta, nthreads=8)
    sel = slice(100, None)
    rel = np.abs(r["var"][sel] / var_exact[sel] - 1)
    assert np.max(rel) < 5 * np.sqrt(2.0 / N)
    # the mean stays at the equilibrium to within the standard error
    se = np.sqrt(var_exact[sel, 0] / N)
    assert np.max(np.abs(r["mean"][sel, 0] - r["delta0"][0]) / se) < 5
