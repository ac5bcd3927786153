"""Flat-prior special case of the oracle's z and beta steps.

With the shrinkage term tau^{-2} Lambda^{-2} set to zero, the two steps of
the sweep that remain (z | beta by Eq. 12's truncated normal, beta | z from
N(G^{-1} X^T z, G^{-1})) are Albert and Chib's (1993) data-augmentation Gibbs
sampler for probit regression with a flat prior, whose target is the probit
likelihood itself.  For N >> p its posterior mean is within O(1/N) of the
maximum-likelihood estimate, computed here independently of the oracle by
Newton's method on log Phi.  A dropped term or a wrong sign in either step
moves the chain's mean far outside Monte Carlo error.
"""
import numpy as np
from scipy import special

from oracle import sweep as osw


def _probit_mle(X, y, iters=50):
    s = 2.0 * y - 1.0
    b = np.zeros(X.shape[1])
    for _ in range(iters):
        m = s * (X @ b)
        lam = np.exp(-0.5 * m * m - 0.5 * np.log(2 * np.pi) - special.log_ndtr(m))  # phi(m) / Phi(m)
        grad = X.T @ (s * lam)
        w = lam * (lam + m)
        H = (X * w[:, None]).T @ X
        step = np.linalg.solve(H, grad)
        b = b + step
        if np.abs(step).max() < 1e-13:
            break
    return b


def test_flat_prior_chain_mean_matches_probit_mle():
    rng = np.random.default_rng(7)
    N, p = 3000, 3
    X = rng.normal(size=(N, p))
    beta_true = np.array([0.8, -0.5, 0.3])
    y = (X @ beta_true + rng.normal(size=N) > 0).astype(np.uint8)
    G = X.T @ X
    zero = np.zeros(p)
    beta = np.zeros(p)
    draws = []
    seed, n, burn = 11, 3000, 200
    for k in range(1, n + 1):
        z, _ = osw.draw_z(beta, X, y, seed, k)
        beta, _, _ = osw.draw_beta(G, zero, 0.0, X.T @ z, seed, k)
        if k > burn:
            draws.append(beta.copy())
    draws = np.array(draws)
    mean = draws.mean(0)
    # batch-means standard error of the chain's mean
    nb = 20
    bm = draws[: len(draws) // nb * nb].reshape(nb, -1, p).mean(1)
    se = bm.std(0, ddof=1) / np.sqrt(nb)
    mle = _probit_mle(X, y)
    assert np.all(np.abs(mean - mle) <= 5 * se + 2.0 / N), (mean, mle, se)
    # the posterior spread matches the likelihood's curvature (inverse observed information)
    s = 2.0 * y - 1.0
    m = s * (X @ mle)
    lam = np.exp(-0.5 * m * m - 0.5 * np.log(2 * np.pi) - special.log_ndtr(m))
    info = (X * (lam * (lam + m))[:, None]).T @ X
    sd_mle = np.sqrt(np.diag(np.linalg.inv(info)))
    np.testing.assert_allclose(draws.std(0), sd_mle, rtol=0.15)


def test_a_planted_sign_error_in_the_beta_mean_is_detected():
    """The same check on a chain whose beta step uses -X^T z: its mean lands
    far from the MLE, so the test above can fail."""
    rng = np.random.default_rng(8)
    N, p = 2000, 2
    X = rng.normal(size=(N, p))
    y = (X @ np.array([0.7, -0.4]) + rng.normal(size=N) > 0).astype(np.uint8)
    G = X.T @ X
    beta = np.zeros(p)
    draws = []
    for k in range(1, 801):
        z, _ = osw.draw_z(beta, X, y, 3, k)
        beta, _, _ = osw.draw_beta(G, np.zeros(p), 0.0, -(X.T @ z), 3, k)
        if k > 100:
            draws.append(beta.copy())
    assert np.abs(np.mean(draws, 0) - _probit_mle(X, y)).max() > 0.2
