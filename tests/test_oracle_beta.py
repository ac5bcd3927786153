"""Pins of the oracle's beta draw (CPU only).

Eq. 12: beta | - ~ N(Sigma X^T z, Sigma) with Sigma = (X^T X + tau^{-2}
Lambda^{-2})^{-1}.  With lambda, tau and z frozen, many draws over distinct
sweep counters must have that mean and covariance, computed here with
numpy's LU solve and inverse (not the Cholesky route the oracle takes).  The
test also shows that the literal reading of the paper's garbled transposes
(solving L v = s with the lower Cholesky factor L) gives the wrong covariance.
"""
import numpy as np
import scipy.linalg
from scipy import stats

from oracle import philox, sweep


def _problem(p=4, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(12, p)) @ np.diag(np.linspace(0.5, 2.0, p)) + 0.6 * rng.normal(size=(12, 1))
    G = X.T @ X
    lam = rng.exponential(size=p) + 0.2
    tau = 0.9
    xtz = rng.normal(size=p) * 3
    return G, lam, tau, xtz


def _draws(G, lam, tau, xtz, n, literal=False):
    out = np.empty((n, G.shape[0]))
    for k in range(1, n + 1):
        if not literal:
            out[k - 1] = sweep.draw_beta(G, lam, tau, xtz, 31, k)[0]
        else:
            A = G + tau * np.diag(lam)
            L = np.linalg.cholesky(A)
            u, uc, _, _ = philox.uniforms(31, np.arange(G.shape[0]), k, philox.BETA)
            s = sweep.std_normal_from_uniform(u, uc)
            mean = scipy.linalg.solve_triangular(L.T, scipy.linalg.solve_triangular(L, xtz, lower=True), lower=False)
            out[k - 1] = mean + scipy.linalg.solve_triangular(L, s, lower=True)
    return out


def _check(draws, G, lam, tau, xtz):
    A = G + tau * np.diag(lam)
    mu = np.linalg.solve(A, xtz)
    Sigma = np.linalg.inv(A)
    n, p = draws.shape
    d = draws.mean(0) - mu
    t2 = n * d @ np.linalg.solve(Sigma, d)
    p_mean = stats.chi2(p).sf(t2)
    S = np.cov(draws.T)
    # Bartlett-type test of the covariance: n * (tr(Sigma^-1 S) - log det(Sigma^-1 S) - p) ~ chi2(p(p+1)/2)
    M = np.linalg.solve(Sigma, S)
    stat = (n - 1) * (np.trace(M) - np.log(np.linalg.det(M)) - p)
    p_cov = stats.chi2(p * (p + 1) // 2).sf(stat)
    return p_mean, p_cov


def test_beta_conditional_is_the_closed_form_gaussian():
    G, lam, tau, xtz = _problem()
    draws = _draws(G, lam, tau, xtz, 6000)
    p_mean, p_cov = _check(draws, G, lam, tau, xtz)
    assert p_mean > 1e-3 and p_cov > 1e-3


def test_literal_transpose_reading_is_detected():
    """Planted mistake: v = L^{-1} s has covariance (L^T L)^{-1} != Sigma."""
    G, lam, tau, xtz = _problem()
    draws = _draws(G, lam, tau, xtz, 6000, literal=True)
    _, p_cov = _check(draws, G, lam, tau, xtz)
    assert p_cov < 1e-6


def test_beta_noise_term_equals_triangular_solve():
    """beta - A^{-1} X^T z = L^{-T} s, with L L^T = A, for the oracle's own s."""
    G, lam, tau, xtz = _problem(p=6, seed=3)
    beta, L, s = sweep.draw_beta(G, lam, tau, xtz, 8, 5)
    A = G + tau * np.diag(lam)
    np.testing.assert_allclose(L @ L.T, A, rtol=1e-13, atol=1e-13 * np.abs(A).max())
    resid = beta - np.linalg.solve(A, xtz)
    np.testing.assert_allclose(L.T @ resid, s, rtol=1e-10, atol=1e-10)
