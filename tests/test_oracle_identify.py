"""Pins of the oracle's identification of an Ito model from a record (Appendix,
Eqs. likelihood, like, reprob, ident).

What fixes it independently of the oracle's own arithmetic:
* the objective equals minus the log-likelihood of the Euler-Maruyama
  transition densities, written here with scipy's normal log-density, less the
  constant the paper drops, (n/2) log(4 pi);
* its gradient and Hessian agree with central differences of the objective;
* planted models -- the OU process, a Gamma process of Table I and the wind
  model of Eq. (windito) -- are recovered from long synthetic records drawn by
  Euler-Maruyama with known normals, each coefficient within four standard
  errors given by the inverse Hessian (the observed Fisher information).
"""
import numpy as np
import pytest
from scipy.stats import norm

import fmc_synth as fs
import oracle as orc

H_STEP = 0.01


def _record(spec, n, seed):
    dW = np.sqrt(H_STEP) * np.random.default_rng(seed).standard_normal((1, n))
    return orc.ito_paths(spec, dW, H_STEP, stratonovich=False)[0]


def _cases():
    w = fs.ito_wind()
    return {
        "ou": (2, fs.ito_gaussian(0.0, 0.045), np.array([0.0, -1.0, 0.0, 0.09, 0.0, 0.0])),
        "gamma": (2, fs.ito_gamma(8.0, 4.0), np.array([2.0, -1.0, 0.0, 0.0, 0.5, 0.0])),
        "wind": (1, w, np.array(list(w["m"]) + list(w["s"]))),
    }


@pytest.mark.parametrize("case", ["ou", "gamma", "wind"])
def test_objective_is_the_transition_likelihood(case):
    kind, spec, q = _cases()[case]
    xi = _record(spec, 3000, 1)
    x, dx = xi[:-1], np.diff(xi)
    mu = q[0] + q[1] * x + q[2] * x * x
    sp = q[3] + q[4] * x + q[5] * x * x
    var = H_STEP * (sp * sp if kind == 1 else sp)
    loglik = norm.logpdf(dx, loc=H_STEP * mu, scale=np.sqrt(var)).sum()
    # -loglik = sum 1/2 log(2 pi var) + r^2 / (2 var) with var = 2 D, so
    # L' = 1/4 sum r^2/D + 1/2 sum log D = -loglik - (n/2) log(4 pi)
    n = dx.size
    expect = -loglik - 0.5 * n * np.log(4 * np.pi)
    assert abs(orc.ito_objective(kind, q, xi, H_STEP) - expect) <= 1e-9 * abs(expect)


@pytest.mark.parametrize("case", ["ou", "gamma", "wind"])
def test_derivatives_match_differences(case):
    kind, spec, q = _cases()[case]
    xi = _record(spec, 4000, 2)
    q0 = q * 1.05 + 0.002
    L, g, H = orc.ito_objective(kind, q0, xi, H_STEP, derivatives=True)
    eps = 1e-6
    for a in range(6):
        e = np.zeros(6)
        e[a] = eps
        Lp, gp, _ = orc.ito_objective(kind, q0 + e, xi, H_STEP, derivatives=True)
        Lm, gm, _ = orc.ito_objective(kind, q0 - e, xi, H_STEP, derivatives=True)
        assert abs((Lp - Lm) / (2 * eps) - g[a]) <= 1e-5 * (abs(g[a]) + np.max(np.abs(g)))
        col = (gp - gm) / (2 * eps)
        assert np.max(np.abs(col - H[:, a])) <= 1e-5 * np.max(np.abs(H))


@pytest.mark.parametrize("case", ["ou", "gamma", "wind"])
def test_planted_model_recovered(case):
    kind, spec, q = _cases()[case]
    xi = _record(spec, 200000, 3)
    est, it = orc.ito_identify(kind, xi, H_STEP, q * 1.1 + 0.01)
    L, g, H = orc.ito_objective(kind, est, xi, H_STEP, derivatives=True)
    assert np.all(np.linalg.eigvalsh(H) > 0)
    se = np.sqrt(np.diag(np.linalg.inv(H)))
    assert np.all(np.abs(est - q) <= 4.0 * se), ((est - q) / se)
    # the estimate is a minimum: no lower value at the planted coefficients
    assert L <= orc.ito_objective(kind, q, xi, H_STEP)
