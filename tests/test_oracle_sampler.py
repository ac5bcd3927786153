"""Whole-sampler pins of the oracle (CPU only).

1. p = 1: the posterior mean and second moment of beta from a long oracle
   chain agree, within batch-means Monte Carlo error, with brute-force
   quadrature of pi(beta | y) proportional to prod_i Phi(y*_i x_i beta) p_HS(beta)
   (Eq. 9 and Eq. 10).  p_HS integrates N(beta; 0, s^2) over s = lambda tau,
   whose density for two independent C+(0,1) factors is
   (4/pi^2) ln(s) / (s^2 - 1).
2. Geweke (2004) joint-distribution test: alternating one Gibbs sweep with a
   fresh y ~ Ber(Phi(X beta)) leaves the prior of (beta, lambda, tau)
   invariant, so functionals of the chain match direct prior draws.
3. The paper's qualitative claim (Sect. 6.1): on synthetic data the posterior
   identifies every nonzero coefficient and shrinks the others.
Each test is also run once with a planted mistake to show it would fail.
"""
import numpy as np
import pytest
from scipy import integrate
from scipy.special import log_ndtr

import oracle.sweep as osw
from oracle import gamma, philox, sweep

import hs_synth


def _g_s(s):
    return np.where(np.abs(s - 1) < 1e-9, 2 / np.pi ** 2, 4 / np.pi ** 2 * np.log(s) / (s * s - 1))


def _hs_prior(b):
    def f(t):
        return np.exp(-0.5 * (b * np.exp(-t)) ** 2) / np.sqrt(2 * np.pi) * _g_s(np.exp(t))
    c = np.log(abs(b))
    return integrate.quad(f, -50, c, limit=200)[0] + integrate.quad(f, c, 50, limit=200)[0]


def _p1_data():
    rng = np.random.default_rng(5)
    N = 12
    x = rng.normal(size=(N, 1))
    y = (x[:, 0] + rng.normal(size=N) > 0).astype(np.uint8)
    ys = 2.0 * y - 1
    assert (ys * x[:, 0] > 0).any() and (ys * x[:, 0] < 0).any()   # not separable
    return x, y, ys


def _quadrature_moments(x, ys):
    def post(b, k):
        return b ** k * np.exp(np.sum(log_ndtr(ys * x[:, 0] * b))) * _hs_prior(b)
    m = [sum(integrate.quad(post, a, c, args=(k,), limit=400)[0] for a, c in ((-40, 0), (0, 40)))
         for k in (0, 1, 2)]
    return m[1] / m[0], m[2] / m[0]


def _bm(v, f, nb=40):
    vals = np.array([f(c) for c in np.array_split(v, nb)])
    return vals.mean(0), vals.std(0, ddof=1) / np.sqrt(nb)


def _p1_chain_z(n=16000, burn=1000):
    x, y, ys = _p1_data()
    m1, m2 = _quadrature_moments(x, ys)
    G = x.T @ x
    _, B, _, _ = sweep.run(sweep.init_state(1), x, y, G, 123, n)
    b = B[burn:, 0]
    mean, se = _bm(b, lambda v: np.array([v.mean(), (v ** 2).mean()]))
    return (mean - np.array([m1, m2])) / se


def test_p1_posterior_matches_quadrature():
    z = _p1_chain_z()
    assert np.all(np.abs(z) < 4.5), z


def _prior_stats(v):
    v = np.abs(v)
    return np.array([np.mean(v < 0.1), np.mean(v < 1), np.mean(v < 10), np.mean(np.arctan(v))])


def _geweke_z(C=12, T=1500, p=3, N=10, seed=0):
    """z-scores of prior functionals over C independent successive-conditional
    chains, each started from a draw of the prior (its stationary law), so the
    between-chain spread is an honest standard error."""
    r = np.random.default_rng(seed)
    X = r.normal(size=(N, p))
    G = X.T @ X
    per = []
    for c in range(C):
        lam = np.abs(r.standard_cauchy(p))
        tau = abs(r.standard_cauchy())
        nu = 1 / r.gamma(0.5, 1.0, size=p)          # nu ~ IG(1/2, 1)
        xi = 1 / r.gamma(0.5, 1.0)
        st = sweep.State(lam * tau * r.normal(size=p), lam ** -2, 1 / nu, tau ** -2, 1 / xi, 0)
        vals = np.empty((T, 2 * p + 1))
        for it in range(T):
            y = (X @ st.beta + r.normal(size=N) > 0).astype(np.uint8)
            st = sweep.sweep_once(st, X, y, G, 1000 * seed + c + 1)
            vals[it] = np.concatenate([st.beta, st.lam_inv2 ** -0.5, [st.tau_inv2 ** -0.5]])
        per.append(np.concatenate([_prior_stats(vals[:, j]) for j in range(vals.shape[1])]))
    per = np.array(per)
    rr = np.random.default_rng(1)
    M = 1_000_000
    pb = np.abs(rr.standard_cauchy(M)) * np.abs(rr.standard_cauchy(M)) * rr.normal(size=M)
    pc = np.abs(rr.standard_cauchy(M))
    ref = np.concatenate([_prior_stats(pb)] * p + [_prior_stats(pc)] * (p + 1))
    return (per.mean(0) - ref) / (per.std(0, ddof=1) / np.sqrt(C))


def test_geweke_joint_distribution():
    z = _geweke_z()
    assert np.all(np.abs(z) < 5.5), np.round(z, 2)


def _bad_tau(beta_prev, lam, xi, seed, k, chain=0, problem=0):
    rate = xi + float(np.sum(lam * beta_prev ** 2))                   # planted: 1/2 dropped
    g, r, m = gamma.gamma_first_accepted((beta_prev.size + 1) / 2.0, seed, k, chain, problem)
    return g / rate, (r, m)


def _bad_lambda(st, seed, k, chain=0, problem=0):
    u, _, _, _ = philox.uniforms(seed, np.arange(st.beta.size), k, philox.LAMBDA, chain, problem)
    return -np.log(u) / (st.nu_inv + st.tau_inv2 * st.beta ** 2)       # planted: 1/2 dropped


def test_planted_tau_mistake_fails_geweke(monkeypatch):
    monkeypatch.setattr(osw, "draw_tau", _bad_tau)
    z = _geweke_z(C=6, T=600)
    assert np.any(np.abs(z) > 5.5)


def test_planted_lambda_mistake_fails_quadrature(monkeypatch):
    monkeypatch.setattr(osw, "draw_lambda", _bad_lambda)
    z = _p1_chain_z()
    assert np.any(np.abs(z) > 4.5)


def test_paper_claim_identifies_nonzeros():
    """Sect. 6.1: the posterior identifies all nonzero coefficients and shrinks the rest."""
    d = hs_synth.make_problem(3000, 30, 5, "f64", seed=1)
    X, y = d["X"], d["y"]
    _, B, _, _ = sweep.run(sweep.init_state(30), X, y, sweep.gram(X), 0, 800)
    post = B[300:]
    lo, hi = np.quantile(post, [0.05, 0.95], axis=0)
    nz = d["beta_true"] != 0
    assert np.all((lo[nz] > 0) | (hi[nz] < 0))               # 90% intervals exclude 0
    assert np.all(np.abs(post.mean(0)[~nz]) < 0.1)
