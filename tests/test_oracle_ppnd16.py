"""Pins for the oracle's inverse normal CDF (Wichura AS 241, PPND16).

Fixed by: the normal CDF of scipy (Phi(Phi^-1(p)) = p), the symmetry of the
normal law, tabulated percentage points, and monotonicity.
"""
import os

import numpy as np
from scipy.special import ndtr, ndtri

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_round_trip_lower_tail(orc):
    # a relative error e in z shows as about e z^2 relative error in Phi(z) in the tail,
    # so the implied error in z is compared against a few FP64 ulps
    for p in np.concatenate([np.logspace(-300, -1, 200), np.linspace(0.1, 0.5, 101)]):
        z = orc.ppnd16(p)
        assert abs(ndtr(z) / p - 1.0) / max(1.0, z * z) < 2e-15, p


def test_round_trip_upper_tail(orc):
    for q in np.logspace(-15, np.log10(0.5), 120):
        p = 1.0 - q
        z = orc.ppnd16(p)
        # 1 - p is exact for these p; compare the tail mass
        assert abs(ndtr(-z) / (1.0 - p) - 1.0) / max(1.0, z * z) < 2e-15, p


def test_symmetry(orc):
    for k in range(1, 1024):
        p = k / 1024.0
        assert orc.ppnd16(1.0 - p) == -orc.ppnd16(p)


def test_tabulated_quantiles(orc):
    with open(os.path.join(GOLDEN, "normal_quantiles.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p, z = map(float, line.split())
            assert abs(orc.ppnd16(p) - z) < 1e-9


def test_against_library_and_monotone(orc):
    ps = np.linspace(1e-6, 1 - 1e-6, 20001)
    zs = np.array([orc.ppnd16(p) for p in ps])
    assert np.all(np.diff(zs) > 0)
    assert np.max(np.abs(zs - ndtri(ps)) / np.maximum(1.0, np.abs(zs))) < 1e-14
    assert orc.ppnd16(0.0) == -np.inf and orc.ppnd16(1.0) == np.inf
