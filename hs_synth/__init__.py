"""Seeded synthetic inputs for the Horseshoe-probit Gibbs sweep.

This module only makes data.  It holds no step of the sampler: both the CUDA
library and the CPU oracle are fed the arrays it returns, byte for byte.

The generative model is the paper's synthetic design (Sect. 6.1, Eq. 13):
x_ij ~ N(0, 1), a sparse true coefficient vector, and y_i = 1{x_i beta + eps_i > 0}
with eps_i ~ N(0, 1), which is the same as y ~ Ber(Phi(X beta)).  The workloads
measured here replace the paper's fixed beta = (1.3, 4, -1, 1.6, 5, -2, 0, ...)
by ``n_nonzero`` coefficients at uniformly chosen positions with magnitude
U[lo, hi] and a random sign; ``paper_beta(p)`` returns the paper's own vector.

Storage formats (what the library is handed):
  * ``f64``  float64 row-major N x p
  * ``f32``  float32 row-major N x p
  * ``bf16`` uint16 bit patterns (round to nearest even from float32)
  * ``fp8``  uint8 e4m3 codes (OCP "FN" variant: bias 7, max 448, no inf)
             with one float32 scale per column, scale_j = max_i |x_ij| / 448

y is generated from the *stored* X (after rounding), so that the sampler's
target is the posterior of the data it is actually given.
"""
from __future__ import annotations

import numpy as np

__all__ = ["make_problem", "paper_beta", "fp8_e4m3_values", "stored_to_float64",
           "counter_uniform_bits", "uneven_sizes"]


def paper_beta(p: int) -> np.ndarray:
    """The paper's synthetic coefficient vector (Sect. 6.1, Eq. 13)."""
    b = np.zeros(p)
    head = np.array([1.3, 4.0, -1.0, 1.6, 5.0, -2.0])
    b[: min(p, 6)] = head[: min(p, 6)]
    return b


def fp8_e4m3_values() -> np.ndarray:
    """Value of every e4m3 code 0..255 (NaN for 0x7f and 0xff)."""
    vals = np.empty(256)
    for c in range(256):
        s = -1.0 if c & 0x80 else 1.0
        e = (c >> 3) & 0xF
        m = c & 0x7
        if e == 0xF and m == 0x7:
            vals[c] = np.nan
        elif e == 0:
            vals[c] = s * (m / 8.0) * 2.0 ** -6
        else:
            vals[c] = s * (1.0 + m / 8.0) * 2.0 ** (e - 7)
    return vals


def _f32_to_bf16_bits(x32: np.ndarray) -> np.ndarray:
    b = x32.view(np.uint32).astype(np.uint64)
    rounding = ((b >> 16) & 1) + 0x7FFF
    return ((b + rounding) >> 16).astype(np.uint16)


def _bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _encode_fp8(v: np.ndarray) -> np.ndarray:
    """Nearest e4m3 code (ties to the even code) of values with |v| <= 448."""
    vals = fp8_e4m3_values()[:0x7F]            # non-negative finite codes, increasing
    a = np.abs(v)
    idx = np.searchsorted(vals, a)             # vals[idx-1] < a <= vals[idx]
    idx = np.clip(idx, 1, len(vals) - 1)
    lo, hi = vals[idx - 1], vals[idx]
    pick_hi = (a - lo > hi - a) | ((a - lo == hi - a) & ((idx % 2) == 0))
    code = np.where(pick_hi, idx, idx - 1).astype(np.uint8)
    code = np.where(a == 0, 0, code).astype(np.uint8)
    return np.where(v < 0, code | 0x80, code).astype(np.uint8)


def stored_to_float64(X, x_dtype: str, scales=None) -> np.ndarray:
    """Value of a stored matrix as float64 (used only to generate y)."""
    if x_dtype in ("f64", "f32"):
        return np.asarray(X, dtype=np.float64)
    if x_dtype == "bf16":
        return _bf16_bits_to_f64(X)
    if x_dtype == "fp8":
        return fp8_e4m3_values()[X] * np.asarray(scales, dtype=np.float64)[None, :]
    raise ValueError(x_dtype)


def _chunk_rng(seed: int, stream: int) -> np.random.Generator:
    # numpy's Philox4x64 keyed by (seed, stream): one independent stream per chunk.
    return np.random.Generator(np.random.Philox(key=(int(seed) & ((1 << 64) - 1)) | (int(stream) << 64)))


def make_problem(N: int, p: int, n_nonzero: int, x_dtype: str = "f64", seed: int = 0,
                 mag=(1.0, 3.0), design: str = "iid", rho: float = 0.5,
                 beta_true=None, chunk_rows: int = 1 << 15, threads: int | None = None) -> dict:
    """Seeded synthetic probit data set.

    Returns a dict with ``X`` (storage array), ``scales`` (fp8 only, else None),
    ``y`` (uint8 in {0,1}), ``beta_true`` (float64), ``x_dtype``, ``N``, ``p``.

    ``design="ar1"`` draws rows from N(0, Toeplitz(rho^|i-j|)) by the recursion
    x_1 = g_1, x_j = rho x_{j-1} + sqrt(1 - rho^2) g_j.
    Stream 0 of numpy's Philox keyed by ``seed`` draws beta_true; row chunk c
    (``chunk_rows`` rows) draws its x's and noise from stream c + 1, so the
    result is the same for any thread count.
    """
    if N < 1 or p < 1:
        raise ValueError("N and p must be positive")
    rng0 = _chunk_rng(seed, 0)
    if beta_true is None:
        beta_true = np.zeros(p)
        k = min(n_nonzero, p)
        pos = rng0.choice(p, size=k, replace=False)
        beta_true[pos] = rng0.uniform(mag[0], mag[1], size=k) * rng0.choice([-1.0, 1.0], size=k)
    beta_true = np.asarray(beta_true, dtype=np.float64)
    if design not in ("iid", "ar1"):
        raise ValueError(design)
    c_ar = np.sqrt(1.0 - rho * rho)

    def rows(rng, n):
        g = rng.standard_normal((n, p), dtype=np.float64)
        if design == "ar1":
            for j in range(1, p):
                g[:, j] = rho * g[:, j - 1] + c_ar * g[:, j]
        return g

    store_dt = {"f64": np.float64, "f32": np.float32, "bf16": np.uint16, "fp8": np.uint8}[x_dtype]
    X = np.empty((N, p), dtype=store_dt)
    y = np.empty(N, dtype=np.uint8)
    starts = list(range(0, N, chunk_rows))
    import concurrent.futures as cf
    import os
    nthr = threads or min(32, os.cpu_count() or 1)

    scales = None
    if x_dtype == "fp8":
        def cmax(ci):
            r0 = starts[ci]
            return np.abs(rows(_chunk_rng(seed, ci + 1), min(chunk_rows, N - r0))).max(axis=0)
        with cf.ThreadPoolExecutor(nthr) as ex:
            colmax = np.max(np.stack(list(ex.map(cmax, range(len(starts))))), axis=0)
        scales = (np.where(colmax > 0, colmax, 1.0) / 448.0).astype(np.float32)

    def fill(ci):
        r0 = starts[ci]
        n = min(chunk_rows, N - r0)
        rng = _chunk_rng(seed, ci + 1)
        blk = rows(rng, n)
        if x_dtype == "f64":
            X[r0:r0 + n] = blk
        elif x_dtype == "f32":
            X[r0:r0 + n] = blk.astype(np.float32)
        elif x_dtype == "bf16":
            X[r0:r0 + n] = _f32_to_bf16_bits(blk.astype(np.float32))
        else:
            X[r0:r0 + n] = _encode_fp8(blk / scales.astype(np.float64)[None, :])
        eta = stored_to_float64(X[r0:r0 + n], x_dtype, scales) @ beta_true
        y[r0:r0 + n] = (eta + rng.standard_normal(n) > 0).astype(np.uint8)

    with cf.ThreadPoolExecutor(nthr) as ex:
        list(ex.map(fill, range(len(starts))))
    return {"X": X, "scales": scales, "y": y, "beta_true": beta_true,
            "x_dtype": x_dtype, "N": N, "p": p}


def uneven_sizes(n: int, N_range=(10_000, 200_000), p_range=(50, 2000), seed: int = 0) -> list:
    """Sizes (N_m, p_m) of n independent problems, each log-uniform on its
    range (rounded to integers), from a Philox stream of its own keyed by seed."""
    rng = _chunk_rng(seed, 1 << 40)
    lo_n, hi_n = np.log(N_range[0]), np.log(N_range[1])
    lo_p, hi_p = np.log(p_range[0]), np.log(p_range[1])
    Ns = np.rint(np.exp(rng.uniform(lo_n, hi_n, size=n))).astype(np.int64)
    ps = np.rint(np.exp(rng.uniform(lo_p, hi_p, size=n))).astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(Ns, ps)]


def counter_uniform_bits(n: int, seed: int) -> np.ndarray:
    """n uint32 words from numpy's Philox stream (test fixtures only)."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    return rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
