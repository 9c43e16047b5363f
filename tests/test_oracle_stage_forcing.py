"""Pin of the disturbance value each RK stage sees in the increment form (reading R8).

With the KL increments, the disturbance is known only on the time grid, x_n at
t_n.  RK4 feeds the swing equations x_n, (x_n + x_{n+1})/2 twice and x_{n+1};
Heun feeds x_n and x_{n+1}.  Those are exactly the values, at the stage times
t_n, t_n + dt/2 and t_n + dt, of the piecewise-linear interpolant of the grid
values.  So the oracle's trajectory must be RK4 (or Heun) applied to the swing
ODE driven by that interpolant, and must converge to the ODE's exact solution at
order 4 (or 2).

What fixes this independently of the oracle's own arithmetic:
* the disturbance is made deterministic and smooth: theta = 0 and a single KL
  coefficient, so x_n = sigma c_k sin(a_k t_n) telescoped from the increments;
* the exact solution of the interpolant-driven ODE comes from scipy's DOP853,
  restarted at every grid node (the interpolant has a kink there), with the
  electrical power from the complex power V conj(Y V);
* the error ratio between dt and dt/2 must be 2^4 (RK4) or 2^2 (Heun).  Planted
  mistakes in the oracle's stage values -- x_n at every stage, or x_{n+1} at
  the midpoint stages -- lag or lead the forcing by half a step, which leaves an
  O(dt) error, and the same check rejects them.
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import fmc_synth as fs
import oracle as orc


def _grid_disturbance(sc, k, sigma):
    """x_n = sigma c_k sin(a_k t_n) on the grid (theta = 0, one KL mode)."""
    t = np.arange(sc.Nt + 1) * sc.dt
    a = (k + 0.5) * math.pi / sc.T
    c = math.sqrt(2.0 * sc.T) / ((k + 0.5) * math.pi)
    return sigma * c * np.sin(a * t)


def _pe_complex(sc, delta):
    """Electrical power as Re(V conj(Y V)), V = E e^{j delta} (+ the infinite bus)."""
    V = sc.E * np.exp(1j * delta)
    Y = sc.G + 1j * sc.B
    pe = np.real(V * np.conj(Y @ V))
    if sc.has_inf_bus:
        # the machines' coupling to the infinite bus (voltage Vinf at angle 0), in the
        # same mutual-admittance convention as the network
        pe = pe + np.real(V * np.conj((sc.Ginf + 1j * sc.Binf) * sc.Vinf))
    return pe


def _exact(sc, x, delta0, pm_eq):
    """The swing ODE driven by the piecewise-linear interpolant of x, solved to
    DOP853's tight tolerance interval by interval; returns the state at T."""
    n, dt = sc.n, sc.dt
    H, D, ws, inj = sc.H, sc.D, sc.omega_s, sc.inject[:, 0]

    def rhs(t, y, t0, x0, x1):
        delta, om = y[:n], y[n:]
        xt = x0 + (t - t0) / dt * (x1 - x0)
        force = pm_eq + inj * xt
        return np.concatenate([ws * om, (force - _pe_complex(sc, delta) - D * om) / (2.0 * H)])

    y = np.concatenate([delta0, np.zeros(n)])
    for m in range(sc.Nt):
        t0 = m * dt
        sol = solve_ivp(rhs, (t0, t0 + dt), y, method="DOP853", rtol=1e-13, atol=1e-15,
                        args=(t0, x[m], x[m + 1]))
        y = sol.y[:, -1]
    return y


def _case(kind, dt, integrator):
    if kind == "smib":
        sc = fs.smib_case(N=1, K=6, T=2.0, dt=dt, theta=0.0, sigma=0.2)
    else:
        sc = fs.multimachine_case(n=3, d=1, K=6, T=1.0, dt=dt, N=1, seed=21)
        sc = sc.replace(theta=np.array([0.0]), sigma=np.array([0.6]))
    return sc.replace(integrator=integrator)


def _errors(kind, integrator, k=2):
    # steps inside each system's asymptotic range (the three-machine network's
    # fastest swing mode is several times the single machine's)
    dts = (0.04, 0.02, 0.01) if kind == "smib" else (0.01, 0.005, 0.0025)
    errs = []
    for dt in dts:
        sc = _case(kind, dt, integrator)
        z = np.zeros((1, sc.K))
        z[0, k] = 1.0
        out = orc.simulate(sc, z, want_traj=True, want_moments=False)
        got = out["traj"][0, -1, :]
        x = _grid_disturbance(sc, k, float(sc.sigma[0]))
        ref = _exact(sc, x, out["delta0"], out["pm_eq"])
        errs.append(np.max(np.abs(got - ref)))
    return errs


def _orders(errs):
    return [math.log2(e0 / e1) for e0, e1 in zip(errs, errs[1:])]


def test_grid_disturbance_is_the_telescoped_increments():
    # the deterministic disturbance the pin relies on: theta = 0 and one KL mode
    # make x_n the mode itself on the grid
    sc = _case("smib", 0.02, fs.RK4)
    z = np.zeros((1, sc.K))
    z[0, 2] = 1.0
    dW = orc.kle_reconstruct(z, 1, sc.K, sc.T, sc.Nt)[:, 0, :]
    x = orc.ou_em(dW, sc.dt, 0.0, float(sc.sigma[0]))[0]
    assert np.max(np.abs(x - _grid_disturbance(sc, 2, float(sc.sigma[0])))) < 1e-14


@pytest.mark.parametrize("kind", ["smib", "three_machines"])
@pytest.mark.parametrize("integrator,order", [(fs.RK4, 4), (fs.HEUN, 2)])
def test_stage_forcing_is_the_interpolant(kind, integrator, order):
    errs = _errors(kind, integrator)
    for p in _orders(errs):
        assert abs(p - order) < 0.3, (errs, _orders(errs))


@pytest.mark.parametrize("plant", [1, 2])
def test_planted_stage_mistakes_are_caught(plant):
    orc.plant_stage_forcing(plant)
    try:
        errs = _errors("three_machines", fs.RK4)
    finally:
        orc.plant_stage_forcing(0)
    orders = _orders(errs)
    # a half-step lag or lead of the forcing: first order, far from 4
    assert all(p < 2.0 for p in orders), (errs, orders)
