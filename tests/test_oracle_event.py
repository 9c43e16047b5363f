"""Pins for the oracle's event (a step in one machine's mechanical power, in the
style of the paper's generator trip, Section V-A) and for its response function
(RMS of the centre-of-inertia speed deviation over the horizon, Section V-B).

Fixed by the mathematics: in a lossless system (G = 0) the electrical powers sum
to zero for any angles, so with damping proportional to inertia (D_i = 2 c H_i)
the centre-of-inertia speed obeys the scalar equation
    y' = dP / (2 sum H) - c y,
and RK4 (Heun), being linear, maps it exactly by the scalar recursion
    y_{n+1} = y_inf + R(-c dt) (y_n - y_inf),  R the method's stability polynomial;
the response function is then a closed-form sum of that sequence.  The RRF of
every sample also equals a numpy evaluation on its trajectory.
"""
import numpy as np
import pytest

import fmc_synth as fs


def _lossless(n=5, c=0.4, seed=3):
    sc = fs.multimachine_case(n=n, d=1, K=10, T=4.0, dt=0.01, N=4, seed=seed)
    G = np.zeros((n, n))
    D = 2.0 * c * sc.H
    # a balanced operating point without conductances: Pm summing to zero
    Pm = sc.Pm - sc.Pm.mean()
    return sc.replace(G=G, D=D, Pm=Pm, sigma=np.zeros(1))


@pytest.mark.parametrize("integrator,R", [(fs.RK4, lambda z: 1 + z + z**2 / 2 + z**3 / 6 + z**4 / 24),
                                          (fs.HEUN, lambda z: 1 + z + z**2 / 2)])
def test_coi_speed_after_the_event_is_the_scalar_recursion(orc, integrator, R):
    c, dP, k_ev, t_ev = 0.4, -0.3, 2, 1.0
    sc = _lossless(c=c).replace(integrator=integrator, event_machine=k_ev, event_time=t_ev, event_dpm=dP)
    r = orc.simulate(sc, np.zeros((1, sc.d * sc.K)), want_traj=True)
    traj = r["traj"][0]
    n, H = sc.n, sc.H
    y = (traj[:, n:] * H).sum(axis=1) / H.sum()
    n_ev = int(round(t_ev / sc.dt))
    yinf = dP / (2.0 * H.sum()) / c
    expect = np.zeros(sc.Nt + 1)
    for m in range(n_ev, sc.Nt):
        expect[m + 1] = yinf + R(-c * sc.dt) * (expect[m] - yinf)
    assert np.max(np.abs(y - expect)) < 1e-12 * abs(yinf)
    assert np.max(np.abs(y[: n_ev + 1])) < 1e-15
    rrf = np.sqrt(np.mean(expect[1:] ** 2))
    assert abs(r["rrf"][0] - rrf) < 1e-12 * rrf


def test_rrf_is_the_rms_of_the_coi_speed_of_each_sample(orc):
    sc = fs.multimachine_case(n=6, d=2, K=20, T=1.0, dt=0.005, N=50, seed=9).replace(
        event_machine=1, event_time=0.25, event_dpm=-0.5)
    z = orc.lhs_sample(sc.seed, sc.N, sc.M)
    r = orc.simulate(sc, z, want_traj=True)
    n = sc.n
    coi = (r["traj"][:, 1:, n:] * sc.H).sum(axis=2) / sc.H.sum()
    assert np.allclose(r["rrf"], np.sqrt(np.mean(coi**2, axis=1)), rtol=1e-13, atol=0)


def test_event_changes_nothing_before_its_step(orc):
    sc = fs.multimachine_case(n=4, d=1, K=20, T=0.5, dt=0.005, N=8, seed=2)
    z = orc.lhs_sample(sc.seed, sc.N, sc.M)
    a = orc.simulate(sc, z, want_traj=True)["traj"]
    b = orc.simulate(sc.replace(event_machine=3, event_time=0.2, event_dpm=0.7), z, want_traj=True)["traj"]
    n_ev = 40
    assert np.array_equal(a[:, : n_ev + 1], b[:, : n_ev + 1])
    assert np.max(np.abs(a[:, n_ev + 2:] - b[:, n_ev + 2:])) > 1e-6
