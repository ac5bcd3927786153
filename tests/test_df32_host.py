"""The FP32-pair ("double-float") arithmetic of the factorization (df32.cuh),
compiled for the host and checked against long double on random operands
spanning 2^-8 .. 2^8: splitting a double, pair add (relative to |a| + |b|),
multiply, reciprocal and square root within a small multiple of 2^-48, and
32-term dot products accumulated with df_fma within 64 x 2^-48 of sum |a_q b_q|
(the tile products of the factorization are such dot products)."""
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


def test_pair_arithmetic_error_bounds(tmp_path):
    exe = str(tmp_path / "df32_check")
    subprocess.run([_nvcc(), "-x", "cu", "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1608_04329_gb300", "csrc"),
                    "-o", exe, os.path.join(ROOT, "tests", "df32_check.cu")], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    err = {out[i]: float(out[i + 1]) for i in range(0, len(out), 2)}
    u = 2.0 ** -48
    assert err["split"] <= u
    assert err["add"] <= 4 * u
    assert err["mul"] <= 8 * u
    assert err["recip"] <= 8 * u
    assert err["sqrt"] <= 8 * u
    assert err["dot32"] <= 64 * u
