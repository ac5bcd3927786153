"""The exact-digit arithmetic of the tensor-core Gram matrix (tc_common.cuh
and the windows of gram_tc.cu), compiled for the host: FP32 values cut into
five BF16 digits on a per-column power-of-two grid reconstruct exactly, every
digit is an integer of at most 8 significant bits (|d_1| <= 256, later digits
<= 128), the class sums of a 128-row window stay below 2^24 at every partial
sum (so FP32 accumulation is exact), and folding the classes into FP32 pairs
that are flushed into FP64 every 8 windows gives X^T X within 2e-13 of
sum |x_ri x_rj| (long double reference) over 16384 rows (FP32 data, five
digits, pairs with t + u <= 6), and within 2e-14 for BF16 data with four
digits and every pair (exact products), for
columns scaled from 2^-20 to 2^20 with tiny and zero entries."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not found")


def test_gram_digit_arithmetic(tmp_path):
    exe = str(tmp_path / "digits_check")
    r = subprocess.run([_nvcc(), "-x", "cu", "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1608_04329_gb300", "csrc"),
                        "-I", os.path.join(ROOT, "include"), "-o", exe, os.path.join(ROOT, "tests", "digits_check.cu")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    v = {out[i]: float(out[i + 1]) for i in range(0, len(out), 2)}
    for tag in ("f32", "bf16"):
        assert v[tag + "_digits_exact"] == 1 and v[tag + "_digit_bounds"] == 1
        assert v[tag + "_rest"] <= 0.5
        assert v[tag + "_window_exact"] == 1 and v[tag + "_class_max"] < 2 ** 24
    assert v["f32_gram_err"] <= 2e-13
    # BF16 data with every digit pair: exact products, only the FP32-pair and
    # FP64 accumulation round
    assert v["bf16_gram_err"] <= 2e-14
