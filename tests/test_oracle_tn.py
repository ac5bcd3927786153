"""Pins of the oracle's truncated-normal draw (CPU only).

The draw is z+ = mu - Phi^{-1}(u Phi(mu)) (the inverse-CDF map of the
truncated normal of Eq. 12, first line).  It is pinned to a 50-digit mpmath
evaluation of the same closed form, to scipy's truncnorm in distribution,
and to the sign rule of Sect. 5 (z update, step a); the paper's own rejection
sampler is pinned to its stated acceptance near mu* = 0.47.
"""
import mpmath as mp
import numpy as np
import pytest
from scipy import stats

from oracle import philox, tn
from tests.golden import claims


def _z_true(mu, u):
    mp.mp.dps = 60
    mu_m, u_m = mp.mpf(mu), mp.mpf(u)
    target = mp.log(u_m) + mp.log(mp.ncdf(mu_m))
    w0 = mu - 1.0 if mu < 0 else -1.0
    from scipy.special import log_ndtr, ndtri
    try:
        guess = float(ndtri(float(u) * float(mp.ncdf(mu_m)))) if float(target) > -700 else None
    except Exception:
        guess = None
    if guess is None or not np.isfinite(guess):
        guess = mu - (-float(mp.log(u_m))) / max(-mu, 1.0)
    w = mp.findroot(lambda x: mp.log(mp.ncdf(x)) - target, mp.mpf(guess), tol=mp.mpf(10) ** -50)
    return float(mu_m - w)


MUS = [-60.0, -40.0, -36.0, -30.0, -10.0, -3.0, -0.5, 0.0, 0.47, 2.0, 8.0, 30.0]
US = [2.0 ** -53, 1e-9, 0.01, 0.3, 0.5, 0.9, 1 - 2.0 ** -30, 1 - 2.0 ** -53]


@pytest.mark.parametrize("mu", MUS)
def test_tn_matches_high_precision_closed_form(mu):
    u = np.array(US)
    uc = np.array([1.0 - x for x in US])       # exact for these values
    z = tn.tn_positive(np.full(len(US), mu), u, uc)
    for zi, ui in zip(z, US):
        zt = _z_true(mu, ui)
        assert zi > 0.0
        assert abs(zi - zt) <= 1e-12 * max(1.0, abs(zt)), (mu, ui, zi, zt)


def test_tn_sign_rule():
    rng = np.random.default_rng(3)
    n = 5000
    y = rng.integers(0, 2, n)
    eta = rng.normal(0, 20, n)
    u, uc, _, _ = philox.uniforms(9, np.arange(n), 1, philox.Z)
    z = tn.tn_signed(2.0 * y - 1.0, eta, u, uc)
    assert np.all((z > 0) == (y == 1)) and np.all(z != 0)


@pytest.mark.parametrize("mu", [-3.0, 0.0, 0.47, 2.0])
def test_tn_inverse_cdf_distribution(mu):
    n = 20000
    u, uc, _, _ = philox.uniforms(5, np.arange(n), 7, philox.Z)
    z = tn.tn_positive(np.full(n, mu), u, uc)
    ref = stats.truncnorm(a=-mu, b=np.inf, loc=mu, scale=1.0)
    assert stats.kstest(z, ref.cdf).pvalue > 1e-3


@pytest.mark.parametrize("mu", [-1.0, 0.3, 0.47, 0.6, 2.0])
def test_paper_rejection_sampler_distribution(mu):
    rng = np.random.default_rng(11)
    z, _ = tn.tn_positive_rejection(np.full(8000, mu), rng)
    ref = stats.truncnorm(a=-mu, b=np.inf, loc=mu, scale=1.0)
    assert stats.kstest(z, ref.cdf).pvalue > 1e-3


def test_paper_rejection_acceptance_near_switch():
    """Worst-case acceptance about 2/3 for mu* near 0.47 (Sect. 5, remark on warp divergence)."""
    c = claims.load()
    switch = float(c["tn_rejection_switch"])
    worst = float(c["tn_rejection_worst_acceptance"])
    rng = np.random.default_rng(12)
    n = 40000
    for mu in (switch - 0.01, switch + 0.01):
        _, tries = tn.tn_positive_rejection(np.full(n, mu), rng)
        acc = n / tries.sum()
        assert abs(acc - worst) < 0.03, (mu, acc)
    # away from the switch the acceptance is higher
    _, tries = tn.tn_positive_rejection(np.full(n, 2.5), rng)
    assert n / tries.sum() > 0.95
