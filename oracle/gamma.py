"""Gamma draw for tau^{-2} by Cheng (1977) algorithm GB (oracle side).

Eq. 12 gives tau^{-2} | - with shape (p + 1) / 2 and scale parameter
xi^{-1} + (1/2) sum_j lambda_j^{-2} beta_j^2.  The equation labels it "IG"
while the drawing step (Sect. 5, tau^{-2} update, step iii) draws
tau^{-2} ~ G(a, b); the reading taken here is a Gamma with that shape and
*rate* b (tau^2 ~ IG, so tau^{-2} ~ Gamma), i.e. tau^{-2} = G / b with
G ~ Gamma(a, 1).

Algorithm GB (R.C.H. Cheng, "The generation of Gamma variables with
non-integral shape parameter", Applied Statistics 26 (1977) 71-75), written
from the paper's description: with lam = sqrt(2a - 1), the proposal is the
log-logistic X = a (u1 / (1 - u1))^{1/lam}; writing V = ln(u1 / (1 - u1)) / lam,
X = a e^V, and the proposal is accepted when
    (a - ln 4) + (a + lam) V - X >= ln(u1^2 u2).
(This is the exact test; Cheng's squeeze only short-cuts it.)

The paper's kernel makes 32 proposals at once and keeps the first accepted one
(Sect. 5, tau^{-2} update, steps a to c).  Here proposal m of round r uses the
uniform pair (u_a, u_b) of counter (32 r + m, k, TAU, ...); the smallest m of
the first round with any acceptance wins, and rounds repeat while all 32
reject.
"""
from __future__ import annotations

import numpy as np

from . import philox


def cheng_gb_propose(a, u1, uc1, u2):
    """Proposals X and accept flags for shape a >= 1 (vectorised over u)."""
    a = float(a)
    lam = np.sqrt(2.0 * a - 1.0)
    V = (np.log(u1) - np.log(uc1)) / lam
    X = a * np.exp(V)
    accept = (a - np.log(4.0)) + (a + lam) * V - X >= 2.0 * np.log(u1) + np.log(u2)
    return X, accept


def gamma_first_accepted(a, seed, k, chain=0, problem=0, max_rounds=64):
    """G ~ Gamma(a, 1): returns (G, round, lane)."""
    for r in range(max_rounds):
        idx = r * 32 + np.arange(32, dtype=np.uint64)
        u1, uc1, u2, _ = philox.uniforms(seed, idx, k, philox.TAU, chain, problem)
        X, acc = cheng_gb_propose(a, u1, uc1, u2)
        if acc.any():
            m = int(np.argmax(acc))
            return float(X[m]), r, m
    raise RuntimeError("Cheng GB: no proposal accepted in %d rounds" % max_rounds)
