"""Pins of the oracle's Gamma (Cheng GB) and Exponential draws (CPU only)."""
import numpy as np
import pytest
from scipy import stats

from oracle import gamma, philox, sweep
from tests.golden import claims


def _draws(a, n, seed=21):
    return np.array([gamma.gamma_first_accepted(a, seed, k)[0] for k in range(1, n + 1)])


@pytest.mark.parametrize("a", [1.0, 1.5, 5.5, 50.5, 500.5])
def test_cheng_gb_gamma_distribution(a):
    g = _draws(a, 3000)
    assert stats.kstest(g, stats.gamma(a).cdf).pvalue > 1e-3
    assert abs(g.mean() - a) < 5 * np.sqrt(a / len(g))


def test_cheng_per_proposal_acceptance_matches_paper():
    """Each of the 32 proposals accepts with probability about 0.88 (Sect. 5, tau update, step c)."""
    c = claims.load()
    n = 200_000
    u1, uc1, u2, _ = philox.uniforms(3, np.arange(n), 1, philox.TAU)
    for a in (50.5, 500.5):
        _, acc = gamma.cheng_gb_propose(a, u1, uc1, u2)
        assert abs(acc.mean() - float(c["cheng_per_proposal_acceptance"])) < 0.01
    # the paper's combined failure probability is (1 - 0.88)^32
    assert np.isclose((1 - float(c["cheng_per_proposal_acceptance"])) ** 32,
                      float(c["cheng_all_reject_probability"]), rtol=0.05)


def test_cheng_first_accepted_rule():
    """The returned proposal is the smallest accepted lane of the first round with an acceptance."""
    seen_later_lane = False
    for k in range(1, 400):
        G, r, m = gamma.gamma_first_accepted(1.0, 77, k)
        idx = r * 32 + np.arange(32)
        u1, uc1, u2, _ = philox.uniforms(77, idx, k, philox.TAU)
        X, acc = gamma.cheng_gb_propose(1.0, u1, uc1, u2)
        assert acc[m] and not acc[:m].any() and X[m] == G
        seen_later_lane |= m > 0
    assert seen_later_lane


def test_tau_draw_moments():
    """tau^{-2} | - ~ Gamma(shape (p+1)/2, rate xi^{-1} + sum lambda^{-2} beta^2 / 2) (Eq. 12)."""
    p = 9
    rng = np.random.default_rng(1)
    beta = rng.normal(size=p)
    lam = rng.exponential(size=p)
    xi = 0.7
    shape = (p + 1) / 2
    rate = xi + 0.5 * np.sum(lam * beta ** 2)
    t = np.array([sweep.draw_tau(beta, lam, xi, 5, k)[0] for k in range(1, 4001)])
    assert stats.kstest(t, stats.gamma(shape, scale=1 / rate).cdf).pvalue > 1e-3


def test_exponential_draws_by_inversion():
    """Eq. 11 and the inversion -ln(u)/theta: lambda^{-2}, nu^{-1}, xi^{-1} are Exp(rate)."""
    p = 50_000
    rng = np.random.default_rng(2)
    st = sweep.init_state(p)
    st.beta = rng.normal(size=p)
    st.nu_inv = rng.exponential(size=p) + 0.1
    st.tau_inv2 = 0.8
    lam = sweep.draw_lambda(st, 9, 1)
    rate = st.nu_inv + st.tau_inv2 * st.beta ** 2 / 2
    # lambda^{-2} * rate is Exp(1)
    assert stats.kstest(lam * rate, "expon").pvalue > 1e-3
    u, _, _, _ = philox.uniforms(9, np.arange(p), 1, philox.LAMBDA)
    np.testing.assert_allclose(lam, -np.log(u) / rate, rtol=1e-15)
    nu = sweep.draw_nu(lam, 9, 1)
    assert stats.kstest(nu * (1 + lam), "expon").pvalue > 1e-3
    xis = np.array([sweep.draw_xi(0.5, 9, k) for k in range(1, 3001)])
    assert stats.kstest(xis * 1.5, "expon").pvalue > 1e-3
