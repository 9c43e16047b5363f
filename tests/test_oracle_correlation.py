"""Pins of the oracle's correlation-reducing permutation (Section IV-B step 2),
the rank method of Iman and Conover (1982) with the identity as target.

What fixes it independently of the oracle's own arithmetic:
* the result is still a Latin hypercube: every stratum hit exactly once per
  dimension, read back through scipy's normal CDF, and each sample keeps its
  position inside its stratum (the uniform of the unreordered design);
* the first dimension is never reordered (the Cholesky factor's first column is
  a scaling), while the others are;
* the decorrelated scores R* have the identity as their sample correlation
  (numpy's corrcoef), and the strata are exactly their ranks (numpy argsort);
* scipy's Spearman rank correlation between columns falls well below that of
  the plain design's random pairing, and a design of one dimension, or with
  N <= M, is left alone or refused.
"""
import numpy as np
import pytest
from scipy.special import ndtr
from scipy.stats import spearmanr

import oracle as orc


def _offdiag(m):
    M = m.shape[0]
    r = m - np.eye(M)
    return np.abs(r).max(), np.sqrt((r ** 2).sum() / (M * (M - 1)))


@pytest.mark.parametrize("N,M", [(17, 3), (500, 20), (2000, 50)])
def test_still_a_latin_hypercube(N, M):
    z, strata = orc.lhs_decorrelate(7, N, M)
    p = ndtr(z)
    st = np.floor(N * p).astype(np.int64)
    for i in range(M):
        assert np.array_equal(np.sort(st[:, i]), np.arange(N))
        assert np.array_equal(st[:, i], strata[i].astype(np.int64))
    # each sample keeps its own uniform inside the new stratum
    u = np.array([[orc.lhs_uniform(7, i, k) for i in range(M)] for k in range(N)])
    assert np.max(np.abs(N * p - st - u)) < 1e-6


def test_first_dimension_kept_and_others_reordered():
    N, M = 500, 20
    _, strata = orc.lhs_decorrelate(3, N, M)
    plain = np.array([[orc.lhs_stratum(3, N, i, k) for k in range(N)] for i in range(M)], dtype=np.uint32)
    assert np.array_equal(strata[0], plain[0])
    assert all(not np.array_equal(strata[i], plain[i]) for i in range(1, M))


@pytest.mark.parametrize("N,M", [(300, 10), (2000, 50)])
def test_scores_are_decorrelated_and_ranked(N, M):
    _, strata, rstar = orc.lhs_decorrelate(11, N, M, want_rstar=True)
    c = np.corrcoef(rstar, rowvar=False)
    assert np.max(np.abs(c - np.eye(M))) < 1e-12
    for i in range(M):
        ranks = np.empty(N, dtype=np.int64)
        ranks[np.argsort(rstar[:, i], kind="stable")] = np.arange(N)
        assert np.array_equal(ranks, strata[i].astype(np.int64))


@pytest.mark.parametrize("N,M,seed", [(500, 20, 1), (2000, 50, 2), (4000, 30, 3)])
def test_rank_correlation_falls(N, M, seed):
    plain = orc.lhs_sample(seed, N, M)
    z, _ = orc.lhs_decorrelate(seed, N, M)
    pmax, prms = _offdiag(spearmanr(plain).correlation)
    dmax, drms = _offdiag(spearmanr(z).correlation)
    # the random pairing leaves correlations of order 1/sqrt(N); the rank method
    # removes most of them
    assert drms < 0.4 * prms and dmax < 0.6 * pmax, (prms, drms, pmax, dmax)


def test_degenerate_designs():
    N = 64
    z1, s1 = orc.lhs_decorrelate(5, N, 1)
    assert np.array_equal(s1[0], np.array([orc.lhs_stratum(5, N, 0, k) for k in range(N)], dtype=np.uint32))
    with pytest.raises(ValueError):
        orc.lhs_decorrelate(5, 10, 10)
    with pytest.raises(ValueError):
        orc.lhs_decorrelate(5, 100, 3, mode=orc.SRS)
    zm, sm = orc.lhs_decorrelate(5, 100, 4, mode=orc.LHS_MIDPOINT)
    assert np.allclose(ndtr(zm) * 100 - sm.T, 0.5, atol=1e-9)
