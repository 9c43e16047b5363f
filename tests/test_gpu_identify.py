"""GPU parity of the Appendix's identification (Eqs. likelihood, like, reprob,
ident) against the FP64 oracle: the objective, its gradient and Hessian summed
on the GPU in FP64 agree with the oracle's to summation rounding, and Newton's
method reaches the oracle's estimate (to a small fraction of its standard
error), on records drawn from the OU process, a
Gamma process of Table I and the wind model of Eq. (windito)."""
import numpy as np
import pytest

import fmc_synth as fs
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

H_STEP = 0.01


def _cases():
    w = fs.ito_wind()
    return {
        "ou": (2, fs.ito_gaussian(0.0, 0.045), np.array([0.0, -1.0, 0.0, 0.09, 0.0, 0.0])),
        "gamma": (2, fs.ito_gamma(8.0, 4.0), np.array([2.0, -1.0, 0.0, 0.0, 0.5, 0.0])),
        "wind": (1, w, np.array(list(w["m"]) + list(w["s"]))),
    }


def _record(orc, spec, n, seed):
    dW = np.sqrt(H_STEP) * np.random.default_rng(seed).standard_normal((1, n))
    return orc.ito_paths(spec, dW, H_STEP, stratonovich=False)[0]


@pytest.mark.parametrize("case", ["ou", "gamma", "wind"])
def test_objective_and_estimate_match_oracle(orc, case):
    fmc = need_gpu()
    import torch
    kind, spec, q = _cases()[case]
    xi = _record(orc, spec, 200000, 3)
    xd = torch.from_numpy(xi).cuda()
    q0 = q * 1.1 + 0.01
    L, g, H = fmc.ito_objective(kind, q0, xd, H_STEP, derivatives=True)
    Lr, gr, Hr = orc.ito_objective(kind, q0, xi, H_STEP, derivatives=True)
    assert abs(L - Lr) <= 1e-10 * abs(Lr)
    assert np.max(np.abs(g - gr)) <= 1e-9 * np.max(np.abs(gr))
    assert np.max(np.abs(H - Hr)) <= 1e-9 * np.max(np.abs(Hr))
    est, it = fmc.ito_identify(kind, xd, H_STEP, q0)
    ref, _ = orc.ito_identify(kind, xi, H_STEP, q0)
    _, _, Hf = orc.ito_objective(kind, ref, xi, H_STEP, derivatives=True)
    se = np.sqrt(np.diag(np.linalg.inv(Hf)))
    # both stop where the remaining decrease is at the rounding of the sums; the
    # estimates then differ by a few thousandths of a standard error at most
    assert np.all(np.abs(est - ref) <= 2e-3 * se), (est - ref) / se


def test_identification_refusals():
    fmc = need_gpu()
    import torch
    xd = torch.linspace(0.5, 1.5, 100, dtype=torch.float64, device="cuda")
    with pytest.raises(fmc.FastMCError) as e:
        fmc.ito_identify(3, xd, 0.01, np.zeros(6))
    assert e.value.code == fmc.EINVAL
    with pytest.raises(fmc.FastMCError) as e:   # sigma = 0 everywhere: no positive diffusion
        fmc.ito_identify(1, xd, 0.01, np.zeros(6))
    assert e.value.code == fmc.EINVAL
    assert fmc.ito_objective(2, np.array([0, 0, 0, -1.0, 0, 0]), xd, 0.01) == float("inf")
