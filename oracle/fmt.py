"""Values of the stored X formats, decoded to float64 (oracle side).

bf16: the upper 16 bits of an IEEE float32.
fp8 e4m3 (OCP "FN"): sign, 4 exponent bits with bias 7, 3 mantissa bits;
exponent 0 is subnormal (m/8 * 2^-6); code 0x7f/0xff is NaN; no infinities.
The value used is scale_j * code_value for column j.
"""
from __future__ import annotations

import numpy as np


def bf16_to_f64(bits):
    return (np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _e4m3_table():
    c = np.arange(256)
    sign = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    m = (c & 7).astype(np.float64)
    val = np.where(e == 0, m / 8.0 * 2.0 ** -6, (1.0 + m / 8.0) * np.exp2(e - 7.0))
    val = sign * val
    val[(e == 0xF) & (c & 7 == 7)] = np.nan
    return val


E4M3 = _e4m3_table()


def fp8_to_f64(codes, scales):
    return E4M3[np.asarray(codes, dtype=np.uint8)] * np.asarray(scales, dtype=np.float32).astype(np.float64)[None, :]


def stored_to_f64(X, x_dtype, scales=None):
    if x_dtype in ("f64", "f32"):
        return np.asarray(X, dtype=np.float64)
    if x_dtype == "bf16":
        return bf16_to_f64(X)
    if x_dtype == "fp8":
        return fp8_to_f64(X, scales)
    raise ValueError(x_dtype)
