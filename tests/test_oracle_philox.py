"""Pins of the oracle's Philox4x32-10 and uniform map (CPU only)."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
from scipy import stats

from oracle import philox

_TRITON_SCRIPT = textwrap.dedent(r'''
    import os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(out_ptr, cin_ptr, seed, n: tl.constexpr):
        offs = tl.arange(0, n)
        c0 = tl.load(cin_ptr + offs * 4 + 0)
        c1 = tl.load(cin_ptr + offs * 4 + 1)
        c2 = tl.load(cin_ptr + offs * 4 + 2)
        c3 = tl.load(cin_ptr + offs * 4 + 3)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
        tl.store(out_ptr + offs * 4 + 0, a)
        tl.store(out_ptr + offs * 4 + 1, b)
        tl.store(out_ptr + offs * 4 + 2, c)
        tl.store(out_ptr + offs * 4 + 3, d)

    data = np.load(sys.argv[1])
    cin = torch.from_numpy(data["counters"].astype(np.uint32).reshape(-1).copy())
    res = {}
    for seed in data["seeds"].tolist():
        out = torch.zeros_like(cin)
        k[(1,)](out, cin, int(seed), cin.numel() // 4)
        res[str(seed)] = out.numpy().reshape(-1, 4)
    np.savez(sys.argv[2], **res)
''')


def test_philox_matches_triton_library(tmp_path):
    """Philox4x32-10 against an independent library implementation (triton's
    tl.philox, run by triton's CPU interpreter): same words for random
    counters and keys, including all-ones words."""
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    n = 64
    counters = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64)
    counters[0] = 0
    counters[1] = 2 ** 32 - 1
    seeds = [0, 1, 2 ** 32 - 1, 2 ** 32, 0x243F6A8885A308D3, 2 ** 64 - 1]
    inp = tmp_path / "in.npz"
    outp = tmp_path / "out.npz"
    np.savez(inp, counters=counters, seeds=np.array(seeds, dtype=np.uint64))
    script = tmp_path / "tri.py"
    script.write_text(_TRITON_SCRIPT)
    env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, str(script), str(inp), str(outp)], env=env,
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    ref = np.load(outp)
    for seed in seeds:
        w = philox.philox4x32_10(counters[:, 0], counters[:, 1], counters[:, 2], counters[:, 3],
                                 seed & 0xFFFFFFFF, seed >> 32)
        mine = np.stack(w, axis=1).astype(np.uint32)
        np.testing.assert_array_equal(mine, ref[str(seed)].astype(np.uint32))


def test_uniform_map_exact():
    """u = (2m+1) 2^-53 and 1-u are exact, inside (0,1), and sum to 1 exactly."""
    hi = np.array([0, 0, 2 ** 32 - 1, 2 ** 31, 12345], dtype=np.uint32)
    lo = np.array([0, 4095, 2 ** 32 - 1, 0, 2 ** 31], dtype=np.uint32)
    u, uc = philox._to_unit(hi, lo)
    assert u[0] == 2.0 ** -53 and u[1] == 2.0 ** -53
    assert u[2] == 1.0 - 2.0 ** -53 and uc[2] == 2.0 ** -53
    assert np.all(u + uc == 1.0)
    assert u[3] == 0.5 + 2.0 ** -53
    m = (int(hi[4]) << 20) | (int(lo[4]) >> 12)
    assert u[4] == (2 * m + 1) / 2.0 ** 53


def test_uniforms_are_uniform_and_streams_distinct():
    n = 200_000
    idx = np.arange(n)
    ua, uca, ub, ucb = philox.uniforms(12345, idx, 3, philox.Z)
    for u in (ua, ub):
        counts, _ = np.histogram(u, bins=100, range=(0, 1))
        assert stats.chisquare(counts).pvalue > 1e-4
        assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.01
    assert abs(np.corrcoef(ua, ub)[0, 1]) < 0.01
    # different purpose / sweep / chain / problem / seed give different streams
    others = [philox.uniforms(12345, idx[:1000], 3, philox.LAMBDA)[0],
              philox.uniforms(12345, idx[:1000], 4, philox.Z)[0],
              philox.uniforms(12345, idx[:1000], 3, philox.Z, chain=1)[0],
              philox.uniforms(12345, idx[:1000], 3, philox.Z, problem=1)[0],
              philox.uniforms(12346, idx[:1000], 3, philox.Z)[0]]
    for o in others:
        assert not np.any(o == ua[:1000])
