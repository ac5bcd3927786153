"""Philox4x32-10 and the counter map of the sampler (oracle side).

Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror & Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11), which the paper
recommends for its constant-time skip-ahead (Sect. 5, random number
generation).  Here it is used statelessly: every uniform the sweep consumes is
a pure function of (seed, counter), so nothing is skipped ahead and nothing is
stored.

Definition (from the SC'11 paper): a 128-bit counter (c0, c1, c2, c3) and a
64-bit key (k0, k1) go through 10 rounds.  One round maps
    (c0, c1, c2, c3) -> (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),
                         hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
with M0 = 0xD2511F53, M1 = 0xCD9E8D57 and hi/lo the halves of the 64-bit
product; after each round the key is bumped by the Weyl constants
(0x9E3779B9, 0xBB67AE85) modulo 2^32.

Counter map (the CUDA library implements the same map on its own):
    key     = (seed mod 2^32, seed div 2^32)
    counter = (index, sweep k, purpose | chain << 8, problem)
    purpose: Z=1 (latent z_i, index i), LAMBDA=2 (index j), TAU=3 (index
    32 r + m for proposal m of round r), BETA=4 (noise s_j), NU=5 (index j),
    XI=6 (index 0).  k counts sweeps from 1.
Uniforms: words (w0, w1) give u_a and (w2, w3) give u_b through
    m = (w_hi << 20) | (w_lo >> 12)      (52 bits)
    u = (2 m + 1) / 2^53,   1 - u = (2 (2^52 - 1 - m) + 1) / 2^53
both exact in float64, so u is in [2^-53, 1 - 2^-53] and 1 - u is known
without rounding.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)

Z, LAMBDA, TAU, BETA, NU, XI = 1, 2, 3, 4, 5, 6


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10; arguments broadcast, returns four uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK32 for v in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = (np.array(v) for v in (c0, c1, c2, c3))
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for _ in range(10):
        p0 = M0 * c0          # < 2^64: exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)
        k0 = (k0 + W0) & 0xFFFFFFFF
        k1 = (k1 + W1) & 0xFFFFFFFF
    return tuple(v.astype(np.uint32) for v in (c0, c1, c2, c3))


def _to_unit(w_hi, w_lo):
    m = (w_hi.astype(np.uint64) << np.uint64(20)) | (w_lo.astype(np.uint64) >> np.uint64(12))
    mc = np.uint64((1 << 52) - 1) - m
    u = (2.0 * m.astype(np.float64) + 1.0) * 2.0 ** -53
    uc = (2.0 * mc.astype(np.float64) + 1.0) * 2.0 ** -53
    return u, uc


def counter(index, k, purpose, chain=0, problem=0):
    return (np.asarray(index, dtype=np.uint64), k, purpose | (int(chain) << 8), problem)


def uniforms(seed, index, k, purpose, chain=0, problem=0):
    """(u_a, 1-u_a, u_b, 1-u_b) for the counters (index, k, purpose|chain<<8, problem)."""
    c0, c1, c2, c3 = counter(index, k, purpose, chain, problem)
    w0, w1, w2, w3 = philox4x32_10(c0, c1, c2, c3, int(seed) & 0xFFFFFFFF, int(seed) >> 32)
    ua, uca = _to_unit(w0, w1)
    ub, ucb = _to_unit(w2, w3)
    return ua, uca, ub, ucb
