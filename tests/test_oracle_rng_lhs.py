"""Pins for the oracle's random numbers and Latin hypercube design (Section IV-B).

What fixes the values here is not the oracle itself:
* Philox4x32-10 against the published known-answer vectors of its definition;
* the LHS design against the defining property of Latin hypercube sampling --
  every one of the N equal-probability strata of every dimension holds exactly
  one sample -- checked through scipy's normal CDF, plus the uniform placement
  inside each stratum and the independence of the per-dimension permutations.
"""
import os

import numpy as np
import pytest
from scipy.special import ndtr
from scipy.stats import chisquare

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(orc, ctr, key, expect):
    assert list(orc.philox4x32_10(ctr, key)) == expect


def test_philox_avalanche(orc):
    # one flipped counter bit changes about half of the 128 output bits
    base = orc.philox4x32_10([1, 2, 3, 4], [5, 6])
    flips = []
    for bit in range(32):
        o = orc.philox4x32_10([1 ^ (1 << bit), 2, 3, 4], [5, 6])
        flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, o)))
    assert 48 < np.mean(flips) < 80


@pytest.mark.parametrize("N", [1, 2, 3, 17, 1000, 1 << 16, (1 << 16) + 1])
def test_every_stratum_hit_once(orc, N):
    M = 3 if N > 5000 else 8
    zeta, strata = orc.lhs_sample(11, N, M, with_strata=True)
    assert zeta.shape == (N, M) and strata.shape == (M, N)
    for i in range(M):
        assert np.array_equal(np.sort(strata[i]), np.arange(N)), f"dimension {i} is not a permutation"
    # the value of sample k in dimension i lies in stratum pi_i(k): N*Phi(zeta) - s in (0, 1)
    pos = N * ndtr(zeta.T) - strata
    assert pos.min() > -1e-9 and pos.max() < 1 + 1e-9


def test_uniform_within_stratum(orc):
    N, M = 4096, 16
    zeta, strata = orc.lhs_sample(3, N, M, with_strata=True)
    pos = (N * ndtr(zeta.T) - strata).ravel()
    # u ~ U(0,1): mean 1/2, variance 1/12; decile counts flat
    assert abs(pos.mean() - 0.5) < 4 * np.sqrt(1 / 12 / pos.size)
    counts, _ = np.histogram(pos, bins=10, range=(0, 1))
    assert chisquare(counts).pvalue > 1e-4


def test_midpoint_and_srs_modes(orc):
    N, M = 100, 5
    zm, sm = orc.lhs_sample(5, N, M, mode=orc.LHS_MIDPOINT, with_strata=True)
    assert np.allclose(N * ndtr(zm.T) - sm, 0.5, atol=1e-9)
    zl, sl = orc.lhs_sample(5, N, M, mode=orc.LHS, with_strata=True)
    assert np.array_equal(sm, sl)  # same permutation, only the in-stratum point differs
    zs = orc.lhs_sample(5, N, M, mode=orc.SRS)
    # SRS: Phi(zeta) is the raw uniform of (k, i)
    u = np.array([[orc.lhs_uniform(5, i, k) for i in range(M)] for k in range(N)])
    assert np.allclose(ndtr(zs), u, rtol=1e-13, atol=0)


def test_subrange_is_slice_of_design(orc):
    N, M = 777, 6
    full, sf = orc.lhs_sample(9, N, M, with_strata=True)
    part, sp = orc.lhs_sample(9, N, M, k0=100, count=77, with_strata=True)
    assert np.array_equal(part, full[100:177])
    assert np.array_equal(sp, sf[:, 100:177])


def test_permutations_independent_across_dimensions(orc):
    N, M = 2000, 6
    _, st = orc.lhs_sample(21, N, M, with_strata=True)
    for i in range(M):
        for j in range(i + 1, M):
            rho = np.corrcoef(st[i].astype(float), st[j].astype(float))[0, 1]
            assert abs(rho) < 5 / np.sqrt(N)


def test_permutation_position_uniform_small_domain(orc):
    # the stratum given to sample 0 is uniform over {0..4} across many dimensions
    N, M = 5, 20000
    _, st = orc.lhs_sample(1, N, M, with_strata=True)
    counts = np.bincount(st[:, 0], minlength=N)
    assert chisquare(counts).pvalue > 1e-4


def test_lhs_mean_much_tighter_than_srs(orc):
    N, M = 1000, 50
    zl = orc.lhs_sample(2, N, M)
    zs = orc.lhs_sample(2, N, M, mode=orc.SRS)
    # LHS: every stratum filled once, so the per-dimension sample mean is O(1/N)
    assert np.abs(zl.mean(axis=0)).max() < 5.0 / N
    # SRS: O(1/sqrt(N))
    assert np.abs(zs.mean(axis=0)).std() > 0.3 / np.sqrt(N)
    assert abs(zl.var(axis=0, ddof=1).mean() - 1.0) < 0.02
