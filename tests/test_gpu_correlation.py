"""GPU parity of the correlation-reducing permutation (Section IV-B step 2, the
rank method of Iman and Conover) against the FP64 oracle.

The new strata are ranks of the decorrelated scores R*, which the GPU forms in
FP32 (Gram matrix, Cholesky factor, inverse, GEMM) and the oracle in FP64, so
two samples whose R* values nearly tie may swap ranks.  What is unique is
compared exactly: every column is a permutation, the first column is the
design's own, and every sample whose oracle value is separated from its
neighbours in rank order by more than the FP32 error bound takes the oracle's
stratum; swapped samples must be such near-ties and stay rare.  Where the
strata agree the design values follow the LHS tolerance of the plain design.
A simulation with the permutation switched on matches the oracle run on the
oracle's decorrelated design.
"""
import math

import numpy as np
import pytest
from scipy.special import ndtr

import fmc_synth as fs
from gpu_common import need_gpu, traj_errors

pytestmark = pytest.mark.gpu


def _zeta_tol(zref):
    z = np.asarray(zref, dtype=np.float64)
    ulp = np.spacing(np.abs(z).astype(np.float32)).astype(np.float64)
    p = ndtr(z)
    q = np.minimum(p, 1.0 - p)
    phi = np.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)
    return 8 * ulp + 2.0**-21 * q / phi + 1e-30


@pytest.mark.parametrize("N,M,seed", [(500, 20, 1), (2000, 50, 2), (4097, 30, 3)])
def test_decorrelated_design_matches_oracle(orc, N, M, seed):
    fmc = need_gpu()
    zeta, strata = fmc.lhs_decorrelate(seed, N, M)
    zg = zeta.cpu().numpy().astype(np.float64)
    sg = strata.cpu().numpy().view(np.uint32).astype(np.int64)
    zr, sr, rstar = orc.lhs_decorrelate(seed, N, M, want_rstar=True)
    sr = sr.astype(np.int64)
    for i in range(M):
        assert np.array_equal(np.sort(sg[i]), np.arange(N))
    assert np.array_equal(sg[0], sr[0])
    eps = 1e-4 * np.max(np.abs(rstar))
    swapped = 0
    for i in range(M):
        bad = np.nonzero(sg[i] != sr[i])[0]
        swapped += bad.size
        if bad.size == 0:
            continue
        order = np.argsort(rstar[:, i], kind="stable")
        v = rstar[order, i]
        gap = np.full(N, np.inf)
        gap[:-1] = np.minimum(gap[:-1], np.diff(v))
        gap[1:] = np.minimum(gap[1:], np.diff(v))
        gap_of = np.empty(N)
        gap_of[order] = gap
        assert np.all(gap_of[bad] < eps), (i, bad, gap_of[bad])
    assert swapped <= 0.01 * N * M, swapped
    same = sg.T == sr.T
    assert np.all(np.abs(zg - zr)[same] <= _zeta_tol(zr)[same])


def test_simulation_with_the_permutation(orc):
    fmc = need_gpu()
    sc = fs.multimachine_case(n=10, d=3, K=40, T=0.5, dt=0.005, N=200, seed=1).replace(correlation=fs.CORR_RANK)
    _, strata = fmc.lhs_decorrelate(sc.seed, sc.N, sc.M)
    zr, sr = orc.lhs_decorrelate(sc.seed, sc.N, sc.M)
    assert np.array_equal(strata.cpu().numpy().view(np.uint32), sr)
    ref = orc.simulate(sc, zr, want_traj=True, nthreads=8)
    for path, precision in (("fused", "bf16x3"), ("plain", "f32")):
        mean, var, traj = fmc.simulate(sc, path=path, precision=precision, want_traj=True)
        fmc.device_status()
        ed, ew = traj_errors(traj.cpu().numpy(), ref["traj"], sc.n)
        assert ed <= 1e-4 and ew <= 1e-4, (path, ed, ew)
        m, v = mean.cpu().numpy(), var.cpu().numpy()
        n = sc.n
        for sl in (slice(0, n), slice(n, 2 * n)):
            scale = np.max(np.sqrt(ref["mean"][:, sl] ** 2 + ref["var"][:, sl]))
            assert np.max(np.abs(m[:, sl] - ref["mean"][:, sl])) <= 1e-5 * scale
            assert np.max(np.abs(v[:, sl] - ref["var"][:, sl])) <= 1e-5 * np.max(np.abs(ref["var"][:, sl]))


def test_refusals():
    fmc = need_gpu()
    for N, M, mode in [(10, 10, fmc.LHS), (100, 5, fmc.SRS), (1, 1, fmc.LHS)]:
        with pytest.raises(fmc.FastMCError) as e:
            fmc.lhs_decorrelate(3, N, M, mode=mode)
        assert e.value.code == fmc.EINVAL
    sc = fs.multimachine_case(n=4, d=2, K=50, T=0.1, dt=0.005, N=64, seed=2).replace(correlation=fs.CORR_RANK)
    with pytest.raises(fmc.FastMCError) as e:
        fmc.simulate(sc)
    assert e.value.code == fmc.EINVAL
