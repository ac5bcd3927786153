"""Truncated-normal latent draw (oracle side).

Eq. 12 (first line) gives z_i ~ TN(x_i beta, 1, y_i): N(x_i beta, 1) truncated
to R+ if y_i = 1 and to R- if y_i = 0 (Sect. 5, definition after Eq. 12).
The paper folds the sign with y*_i = 2 y_i - 1 and mu*_i = y*_i x_i beta, draws
z+ from N(mu*, 1) truncated to R+, and returns z_i = y*_i z+ (Sect. 5, z
update, step a).

Transition used here (the CUDA library computes the same map): z+ is the
inverse-CDF image of the uniform u,
    P(Z > z+ | Z > 0) = u  for Z ~ N(mu*, 1),  i.e.  Phi(mu* - z+) = u Phi(mu*),
    z+ = mu* - Phi^{-1}(u Phi(mu*)).
Phi^{-1} is evaluated on the smaller of q = u Phi(mu*) and
1 - q = (1 - u) + u Phi(-mu*) (both exact algebra; 1 - u is exact), and where
q would leave the normal float64 range the same equation is solved in log
space, log Phi(mu* - z) - log Phi(mu*) = log u, by bracketed root finding.
z+ is floored at the smallest normal float64 so that y*_i z_i > 0 always.

``tn_positive_rejection`` is the paper's own two-arm rejection sampler
(Sect. 5, z update, steps b and c): Gaussian proposals when mu* > 0.47,
otherwise Robert (1995) exponential proposals z+ ~ Exp(theta) with
theta = (-mu* + sqrt(mu*^2 + 4)) / 2 and acceptance
rho = exp(-(z+ - mu* - theta)^2 / 2).  The paper does not print theta and rho;
they are Robert's optimal rate and acceptance for N(0,1) truncated to
(a, inf) with a = -mu*, shifted back by mu*.  It draws from its own numpy
generator and is compared with the inverse-CDF map in distribution only.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq
from scipy.special import log_ndtr, ndtr, ndtri

TINY = np.finfo(np.float64).tiny
LOG_NORMAL_FLOOR = -700.0     # exp(-700) ~ 1e-304: q stays a normal float64


def tn_positive(mu, u, uc):
    """z+ with Phi(mu - z+) = u Phi(mu); ``uc`` must be 1 - u exactly."""
    mu = np.asarray(mu, dtype=np.float64)
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), mu.shape)
    uc = np.broadcast_to(np.asarray(uc, dtype=np.float64), mu.shape)
    out = np.empty(mu.shape)
    log_pm = log_ndtr(mu)
    main = (np.log(u) + log_pm) > LOG_NORMAL_FLOOR
    m, um, ucm = mu[main], u[main], uc[main]
    q = um * ndtr(m)
    qc = ucm + um * ndtr(-m)
    w = np.where(q <= qc, ndtri(np.minimum(q, 0.5)), -ndtri(np.minimum(qc, 0.5)))
    out[main] = m - w
    for idx in zip(*np.nonzero(~main)):
        out[idx] = _tail_root(float(mu[idx]), float(u[idx]), float(log_pm[idx]))
    return np.maximum(out, TINY)


def _tail_root(mu, u, log_pm):
    target = np.log(u)

    def f(z):
        return float(log_ndtr(mu - z)) - log_pm - target

    hi = 2.0 * (-target) / max(-mu, 1.0) + 1.0
    while f(hi) > 0.0:
        hi *= 2.0
    return brentq(f, 0.0, hi, xtol=1e-300, rtol=4.0 * np.finfo(float).eps, maxiter=500)


def tn_signed(ystar, eta, u, uc):
    """z_i = y*_i z+_i with mu*_i = y*_i eta_i."""
    ystar = np.asarray(ystar, dtype=np.float64)
    return ystar * tn_positive(ystar * np.asarray(eta, dtype=np.float64), u, uc)


def tn_positive_rejection(mu, rng: np.random.Generator, switch: float = 0.47):
    """The paper's two-arm rejection sampler; returns (z+, proposals used)."""
    mu = np.atleast_1d(np.asarray(mu, dtype=np.float64))
    out = np.empty(mu.shape)
    tries = np.zeros(mu.shape, dtype=np.int64)
    for i, m in enumerate(mu):
        if m > switch:
            while True:
                tries[i] += 1
                z = rng.standard_normal() + m
                if z > 0.0:
                    out[i] = z
                    break
        else:
            theta = (-m + np.sqrt(m * m + 4.0)) / 2.0
            while True:
                tries[i] += 1
                z = -np.log(rng.random()) / theta
                rho = np.exp(-0.5 * (z - m - theta) ** 2)
                if rng.random() < rho:
                    out[i] = z
                    break
    return out, tries
