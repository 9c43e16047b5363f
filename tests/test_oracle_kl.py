"""Pins for the oracle's Karhunen-Loeve reconstruction (Eqs. kl, kle, eqkl).

Fixed by the mathematics of the Brownian motion, not by the oracle:
* Var W(T) = T, and the truncation remainder at t = T has the closed form
  (2T/pi^2) psi_1(K + 1/2) (trigamma, scipy);
* Cov(W(s), W(t)) = min(s, t), approached within the truncation bound;
* increments telescope to W, and are nearly orthogonal with Var ~ dt;
* the reconstruction is the matrix product zeta . phi (numpy on tiny inputs);
* the empirical covariance of LHS-reconstructed increments matches the
  truncated closed form within sampling error.
"""
import numpy as np
import pytest
from scipy.special import polygamma


@pytest.mark.parametrize("K,T", [(1, 1.0), (6, 60.0), (100, 10.0), (200, 20.0), (300, 5.0)])
def test_variance_at_horizon_with_closed_form_remainder(orc, K, T):
    Nt = 16
    psi = orc.kl_path_basis(K, T, Nt)
    var_trunc = np.sum(psi[:, Nt] ** 2)
    remainder = 2.0 * T / np.pi**2 * polygamma(1, K + 0.5)
    assert abs(var_trunc + remainder - T) < 1e-12 * T


def test_covariance_tends_to_min(orc):
    K, T, Nt = 20000, 10.0, 20
    psi = orc.kl_path_basis(K, T, Nt)
    t = np.linspace(0, T, Nt + 1)
    cov = psi.T @ psi
    bound = 2.0 * T / np.pi**2 * polygamma(1, K + 0.5)
    assert np.max(np.abs(cov - np.minimum.outer(t, t))) <= bound + 1e-12


def test_increments_telescope(orc):
    K, T, Nt = 50, 7.0, 333
    phi = orc.kl_increment_basis(K, T, Nt)
    psi = orc.kl_path_basis(K, T, Nt)
    assert np.allclose(phi, np.diff(psi, axis=1), rtol=0, atol=1e-14)
    assert np.allclose(phi.sum(axis=1), psi[:, -1], rtol=0, atol=1e-13)
    assert np.all(psi[:, 0] == 0.0)


def test_increments_nearly_orthonormal(orc):
    K, T, Nt = 10, 10.0, 20000
    dt = T / Nt
    phi = orc.kl_increment_basis(K, T, Nt)
    gram = phi @ phi.T / dt
    assert np.max(np.abs(gram - np.eye(K))) < 1e-4


def test_reconstruct_is_matrix_product(orc):
    rng = np.random.default_rng(0)
    count, d, K, T, Nt = 3, 2, 4, 1.5, 5
    zeta = rng.standard_normal((count, d * K))
    dW = orc.kle_reconstruct(zeta, d, K, T, Nt)
    phi = orc.kl_increment_basis(K, T, Nt)
    ref = np.einsum("swk,kn->swn", zeta.reshape(count, d, K), phi)
    assert np.allclose(dW, ref, rtol=1e-14, atol=1e-15)


def test_empirical_increment_covariance(orc):
    N, d, K, T, Nt = 8192, 1, 20, 10.0, 50
    zeta = orc.lhs_sample(4, N, d * K)
    dW = orc.kle_reconstruct(zeta, d, K, T, Nt)[:, 0, :]
    phi = orc.kl_increment_basis(K, T, Nt)
    cov_true = phi.T @ phi  # truncated closed form: zeta iid unit normals
    cov_emp = np.cov(dW.T)
    scale = np.sqrt(np.outer(np.diag(cov_true), np.diag(cov_true)))
    assert np.max(np.abs(cov_emp - cov_true) / scale) < 6 * np.sqrt(2.0 / N)
    # and the variance of each increment approaches dt as K grows (Proposition 1)
    v20 = np.sum(orc.kl_increment_basis(20, T, Nt) ** 2, axis=0).mean()
    v400 = np.sum(orc.kl_increment_basis(400, T, Nt) ** 2, axis=0).mean()
    assert abs(v400 - T / Nt) < abs(v20 - T / Nt)
    # the missing part is the tail sum_{k>K} c_k^2 (sin a_k t_{n+1} - sin a_k t_n)^2, whose
    # time average is about the closed-form remainder (2T/pi^2) psi_1(K + 1/2)
    rem = 2.0 * T / np.pi**2 * polygamma(1, 400 + 0.5)
    assert 0.5 * rem < (T / Nt - v400) < 1.5 * rem


# ----------------------------------------------------------------------------- the paper's cosine basis
# Eq. (klb2): m_1 = 1/sqrt(T), m_j = sqrt(2/T) cos((j-1) pi t / T).  Integrated,
# the first term is t/sqrt(T) and the others are the Karhunen-Loeve expansion of
# the Brownian bridge, whose variance is t (1 - t/T); so W_K(T) is exact for
# every K, Var W_K(t) -> t from below, and the bridge tail after K - 1 terms is
# at most (2T/pi^2) psi_1(K) (trigamma).


@pytest.mark.parametrize("K,T", [(1, 1.0), (2, 3.0), (6, 60.0), (100, 10.0)])
def test_cosine_basis_exact_at_horizon(orc, K, T):
    Nt = 24
    psi = orc.kl_path_basis(K, T, Nt, orc.BASIS_COSINE)
    assert abs(np.sum(psi[:, Nt] ** 2) - T) < 1e-12 * T
    assert abs(psi[0, Nt] - np.sqrt(T)) < 1e-14 * np.sqrt(T)


@pytest.mark.parametrize("K", [1, 2, 17, 300])
def test_cosine_basis_variance_below_t_within_bridge_tail(orc, K):
    T, Nt = 10.0, 400
    psi = orc.kl_path_basis(K, T, Nt, orc.BASIS_COSINE)
    t = np.linspace(0.0, T, Nt + 1)
    rem = t - np.sum(psi**2, axis=0)
    assert rem.min() > -1e-12
    assert rem.max() <= 2.0 * T / np.pi**2 * polygamma(1, K) + 1e-12
    if K == 1:  # only the linear term: the bridge variance is missing entirely
        assert np.allclose(rem, t * (1 - t / T), rtol=0, atol=1e-12)


def test_cosine_basis_covariance_tends_to_min(orc):
    K, T, Nt = 20000, 10.0, 20
    psi = orc.kl_path_basis(K, T, Nt, orc.BASIS_COSINE)
    t = np.linspace(0, T, Nt + 1)
    cov = psi.T @ psi
    assert np.max(np.abs(cov - np.minimum.outer(t, t))) <= 2.0 * T / np.pi**2 * polygamma(1, K) + 1e-12


def test_cosine_basis_increments(orc):
    K, T, Nt = 40, 5.0, 250
    phi = orc.kl_increment_basis(K, T, Nt, orc.BASIS_COSINE)
    psi = orc.kl_path_basis(K, T, Nt, orc.BASIS_COSINE)
    assert np.allclose(phi, np.diff(psi, axis=1), rtol=0, atol=1e-14)
    # the constant white-noise mode contributes dt/sqrt(T) per step; every
    # oscillating mode integrates to zero over [0, T]
    # (a difference of two values up to sqrt(T): a few ulps of sqrt(T) absolute)
    assert np.allclose(phi[0], (T / Nt) / np.sqrt(T), rtol=0, atol=8 * np.finfo(float).eps * np.sqrt(T))
    assert np.max(np.abs(phi[1:].sum(axis=1))) < 1e-13
    # differs from the Brownian eigenbasis
    assert np.max(np.abs(phi - orc.kl_increment_basis(K, T, Nt))) > 1e-3
