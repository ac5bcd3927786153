"""One Gibbs sweep of the Horseshoe-probit sampler (oracle side, float64).

Model (Sect. 5): Eq. 9 (probit likelihood through latent z), Eq. 10
(horseshoe prior), Eq. 11 (kappa ~ IG(1, theta) <=> 1/kappa ~ Exp(theta)) and
the full conditionals of Eq. 12, with Sigma = (X^T X + tau^{-2} Lambda^{-2})^{-1}.
State: beta, lambda^{-2} (``lam_inv2``), nu^{-1} (``nu_inv``), tau^{-2},
xi^{-1} and the number k of sweeps done.  z is not part of the state: it is
drawn afresh from beta at the start of every sweep.

Update schedule (Sect. 5, steps (i) and (ii) after Eq. 12):
 (i)  z and lambda^{-2} in parallel (both from the previous state), then
      tau^{-2} (from the new lambda^{-2} and the previous beta and xi^{-1});
 (ii) beta, nu^{-1} and xi^{-1} in parallel.
Exponential draws use inversion, -ln(u) / theta (Sect. 5, lambda/nu/xi
update, step ii); the Exp parameter is a rate.

beta (Sect. 5, beta update, steps i to viii): with A = X^T X + tau^{-2}
Lambda^{-2} = L L^T (L lower), the paper's printed transposes are garbled; the
reading used here is the one whose covariance is Sigma = A^{-1}:
    w = L^{-1} X^T z,  s_j = Phi^{-1}(u_j),  beta = L^{-T} (w + s),
so that E[beta] = A^{-1} X^T z and Cov[beta] = L^{-T} L^{-1} = A^{-1}.

Initial state (Sect. 6.1 and 6.2, cold start): beta = 0 and
lambda = nu = tau = xi = 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg
from scipy.special import ndtri

from . import philox
from .gamma import gamma_first_accepted
from .tn import tn_signed


@dataclass
class State:
    beta: np.ndarray
    lam_inv2: np.ndarray
    nu_inv: np.ndarray
    tau_inv2: float
    xi_inv: float
    k: int = 0
    extra: dict = field(default_factory=dict)

    def copy(self):
        return State(self.beta.copy(), self.lam_inv2.copy(), self.nu_inv.copy(),
                     float(self.tau_inv2), float(self.xi_inv), int(self.k))


def init_state(p: int) -> State:
    return State(np.zeros(p), np.ones(p), np.ones(p), 1.0, 1.0, 0)


def gram(X) -> np.ndarray:
    """X^T X in float64 (Sect. 5, beta update, step i)."""
    X = np.asarray(X, dtype=np.float64)
    return X.T @ X


def std_normal_from_uniform(u, uc):
    """Phi^{-1}(u), evaluated on the smaller of u and 1 - u."""
    return np.where(u <= uc, ndtri(np.minimum(u, 0.5)), -ndtri(np.minimum(uc, 0.5)))


def draw_lambda(st: State, seed, k, chain=0, problem=0):
    p = st.beta.size
    u, _, _, _ = philox.uniforms(seed, np.arange(p), k, philox.LAMBDA, chain, problem)
    rate = st.nu_inv + st.tau_inv2 * st.beta ** 2 / 2.0
    return -np.log(u) / rate


def draw_tau(beta_prev, lam_inv2_new, xi_inv_prev, seed, k, chain=0, problem=0):
    p = beta_prev.size
    shape = (p + 1) / 2.0
    rate = xi_inv_prev + 0.5 * float(np.sum(lam_inv2_new * beta_prev ** 2))
    g, r, m = gamma_first_accepted(shape, seed, k, chain, problem)
    return g / rate, (r, m)


def draw_z(beta, X, y, seed, k, chain=0, problem=0):
    N = X.shape[0]
    eta = X @ beta
    ystar = 2.0 * np.asarray(y, dtype=np.float64) - 1.0
    u, uc, _, _ = philox.uniforms(seed, np.arange(N), k, philox.Z, chain, problem)
    return tn_signed(ystar, eta, u, uc), eta


def draw_beta(G, lam_inv2, tau_inv2, xtz, seed, k, chain=0, problem=0):
    p = xtz.size
    A = G + tau_inv2 * np.diag(lam_inv2)
    L = np.linalg.cholesky(A)
    w = scipy.linalg.solve_triangular(L, xtz, lower=True)
    u, uc, _, _ = philox.uniforms(seed, np.arange(p), k, philox.BETA, chain, problem)
    s = std_normal_from_uniform(u, uc)
    beta = scipy.linalg.solve_triangular(L.T, w + s, lower=False)
    return beta, L, s


def draw_nu(lam_inv2_new, seed, k, chain=0, problem=0):
    p = lam_inv2_new.size
    u, _, _, _ = philox.uniforms(seed, np.arange(p), k, philox.NU, chain, problem)
    return -np.log(u) / (1.0 + lam_inv2_new)


def draw_xi(tau_inv2_new, seed, k, chain=0, problem=0):
    u, _, _, _ = philox.uniforms(seed, np.zeros(1), k, philox.XI, chain, problem)
    return float(-np.log(u[0]) / (1.0 + tau_inv2_new))


def sweep_once(st: State, X, y, G, seed, chain=0, problem=0, keep=False) -> State:
    """One sweep k = st.k + 1 from state ``st``; X is float64 N x p."""
    k = st.k + 1
    # (i) z and lambda^{-2} in parallel, then tau^{-2}
    z, eta = draw_z(st.beta, X, y, seed, k, chain, problem)
    lam_inv2 = draw_lambda(st, seed, k, chain, problem)
    tau_inv2, tau_pick = draw_tau(st.beta, lam_inv2, st.xi_inv, seed, k, chain, problem)
    # (ii) beta, nu^{-1}, xi^{-1} in parallel
    xtz = X.T @ z
    beta, L, s = draw_beta(G, lam_inv2, tau_inv2, xtz, seed, k, chain, problem)
    nu_inv = draw_nu(lam_inv2, seed, k, chain, problem)
    xi_inv = draw_xi(tau_inv2, seed, k, chain, problem)
    out = State(beta, lam_inv2, nu_inv, tau_inv2, xi_inv, k)
    if keep:
        out.extra = {"z": z, "eta": eta, "xtz": xtz, "L": L, "s": s, "tau_pick": tau_pick}
    return out


def run(st: State, X, y, G, seed, n, chain=0, problem=0, thin=1):
    """n sweeps; returns the final state and the thinned draws of beta, lambda^{-2}, tau^{-2}."""
    betas, lams, taus = [], [], []
    for _ in range(n):
        st = sweep_once(st, X, y, G, seed, chain, problem)
        if st.k % thin == 0:
            betas.append(st.beta.copy())
            lams.append(st.lam_inv2.copy())
            taus.append(st.tau_inv2)
    return st, np.array(betas), np.array(lams), np.array(taus)
