"""The allocation-free X-stream entry point against the FP64 oracle.

hs_probit_xstream_noalloc exists for callers that must not call cudaMalloc
while they run (it can synchronize the device and allocates outside the
caller's own memory pool).  It runs the X-stream kernels with their scratch in
a fixed device array, on buffers the caller owns.  Here its z and X^T z are
compared with the oracle's latent draw from the same beta and counters
(``oracle.sweep.draw_z``) and with X^T z formed from the oracle's z, on two
calls in a row (the second with a different beta and sweep number, so
left-over scratch from the first call would show).  Every buffer handed to the
library is a real device allocation of the size the call reads.  This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from tests.gpu_common import lib_pkg, problem, random_state, x_f64

pytestmark = pytest.mark.gpu

_LD_ELEMS = {"f32": 4, "bf16": 8, "fp8": 16}  # elements per 16 bytes


def _padded(d, ld):
    """X of the problem with rows padded to ld elements (zeros past p)."""
    X = d["X"]
    out = np.zeros((X.shape[0], ld), dtype=X.dtype)
    out[:, : X.shape[1]] = X
    return out.view(np.int16) if out.dtype == np.uint16 else out  # torch holds bf16 bit patterns as int16


@pytest.mark.parametrize("dt,N,p", [("f32", 20003, 301),   # one 16-byte slice per thread, 16-row tiles
                                    ("f32", 3001, 1500),   # two slices per thread, 4-row tiles
                                    ("bf16", 9001, 300),
                                    ("fp8", 7001, 130)])   # column scales folded into beta_c and X^T z
def test_noalloc_xstream_matches_oracle(dt, N, p):
    torch = pytest.importorskip("torch")
    pkg = lib_pkg()
    lib = pkg.load_library()
    seed = 77
    d = problem(N, p, 5, dt, seed=12)
    X64 = x_f64(d)
    ve = _LD_ELEMS[dt]
    ld = (p + ve - 1) // ve * ve
    Xd = torch.from_numpy(_padded(d, ld)).cuda()
    yd = torch.from_numpy(d["y"]).cuda()
    sc = None if d["scales"] is None else torch.from_numpy(np.ascontiguousarray(d["scales"], np.float32)).cuda()
    xtz = torch.empty(p, dtype=torch.float64, device="cuda")
    z = torch.empty(N, dtype=torch.float64, device="cuda")
    for call, (k, sseed) in enumerate(((4, 1), (9, 2))):
        st = random_state(p, k=k, seed=sseed)
        bc = np.zeros(ld, dtype=np.float32)
        bc[:p] = st.beta * (1.0 if d["scales"] is None else d["scales"])
        bcd = torch.from_numpy(bc).cuda()
        xtz.fill_(np.nan)
        z.fill_(np.nan)
        torch.cuda.synchronize()
        status = lib.hs_probit_xstream_noalloc(
            pkg.X_FP8E4M3 if dt == "fp8" else pkg.X_BF16 if dt == "bf16" else pkg.X_F32,
            ctypes.c_void_p(Xd.data_ptr()), ld, ctypes.c_void_p(yd.data_ptr()), N, p,
            ctypes.c_void_p(bcd.data_ptr()), None if sc is None else ctypes.c_void_p(sc.data_ptr()),
            seed, 0, 0, k + 1, ctypes.c_void_p(xtz.data_ptr()), ctypes.c_void_p(z.data_ptr()), None)
        assert status == 0, (call, status)
        got_xtz, got_z = xtz.cpu().numpy(), z.cpu().numpy()
        zt, _ = oracle.sweep.draw_z(st.beta, X64, d["y"], seed, k + 1)
        xtzt = X64.T @ zt
        # FP32 arithmetic on the stored X: the tolerance of every FP32-accumulation path
        assert np.all(np.sign(got_z) == np.sign(zt)), call
        dz = np.abs(got_z - zt) / np.maximum(np.abs(zt), 1.0)
        assert dz.max() <= 1e-4, (call, dz.max())
        assert np.linalg.norm(got_xtz - xtzt) <= 1e-4 * np.linalg.norm(xtzt), call


def test_noalloc_rejects_scales_for_unscaled_types():
    torch = pytest.importorskip("torch")
    pkg = lib_pkg()
    lib = pkg.load_library()
    N, p = 64, 8
    X = torch.zeros((N, p), dtype=torch.float32, device="cuda")
    y = torch.zeros(N, dtype=torch.uint8, device="cuda")
    bc = torch.zeros(p, dtype=torch.float32, device="cuda")
    sc = torch.ones(p, dtype=torch.float32, device="cuda")
    xtz = torch.empty(p, dtype=torch.float64, device="cuda")
    st = lib.hs_probit_xstream_noalloc(pkg.X_F32, ctypes.c_void_p(X.data_ptr()), p, ctypes.c_void_p(y.data_ptr()),
                                       N, p, ctypes.c_void_p(bc.data_ptr()), ctypes.c_void_p(sc.data_ptr()), 0, 0,
                                       0, 1, ctypes.c_void_p(xtz.data_ptr()), None, None)
    assert st == -1


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """FP32 rows of 8192 columns take one row per tile, so the kernel's grid is
    min(SMs - 1, N) blocks, each with one 32 KB row of partial sums: on a GPU
    with more than 129 SMs that exceeds the fixed 4 MiB and the call is refused
    on the host.  The buffers are real allocations of the full size, so on a
    smaller GPU, where the call is accepted, the kernels run on valid memory."""
    torch = pytest.importorskip("torch")
    pkg = lib_pkg()
    lib = pkg.load_library()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    N, p = 4096, 8192
    grid = min(max(sms - 1, 1), N)
    beyond = grid * p * 4 > (4 << 20)
    X = torch.zeros((N, p), dtype=torch.float32, device="cuda")
    y = torch.zeros(N, dtype=torch.uint8, device="cuda")
    bc = torch.zeros(p, dtype=torch.float32, device="cuda")
    xtz = torch.empty(p, dtype=torch.float64, device="cuda")
    st = lib.hs_probit_xstream_noalloc(pkg.X_F32, ctypes.c_void_p(X.data_ptr()), p, ctypes.c_void_p(y.data_ptr()),
                                       N, p, ctypes.c_void_p(bc.data_ptr()), None, 0, 0, 0, 1,
                                       ctypes.c_void_p(xtz.data_ptr()), None, None)
    assert st == (-1 if beyond else 0), (sms, st)
