"""The allocation-free X-stream entry point against the handle's sweep.

hs_probit_xstream_noalloc exists for callers that must not call cudaMalloc
while they run (it can synchronize the device and allocates outside the
caller's own memory pool).  It runs the X-stream kernels with their scratch in
a fixed device array, on buffers the caller owns.  Here it must reproduce the
z and X^T z that hs_probit_sweep computes from the same beta and counters,
on two calls in a row (the second with a different beta and sweep number, so
left-over scratch from the first call would show).  This file is collected
last on purpose.
"""
import ctypes

import numpy as np
import pytest

from tests.gpu_common import lib_pkg, problem, random_state

pytestmark = pytest.mark.gpu


def _handle_reference(pkg, d, st, seed):
    s = pkg.HSProbit(d["X"], d["y"], seed=seed, debug=True)
    try:
        s.set_state(st.beta, st.lam_inv2, st.nu_inv, st.tau_inv2, st.xi_inv, st.k)
        s.sweep(1)
        return s.debug_xtz(), s.debug_z()
    finally:
        s.close()


def test_noalloc_xstream_matches_handle_sweep():
    torch = pytest.importorskip("torch")
    pkg = lib_pkg()
    lib = pkg.load_library()
    N, p, seed = 20003, 301, 77
    d = problem(N, p, 5, "f32", seed=12)
    ld = (p + 3) // 4 * 4                      # rows of 16-byte multiples for FP32
    Xp = np.zeros((N, ld), dtype=np.float32)
    Xp[:, :p] = d["X"]
    Xd = torch.from_numpy(Xp).cuda()
    yd = torch.from_numpy(d["y"]).cuda()
    xtz = torch.empty(p, dtype=torch.float64, device="cuda")
    z = torch.empty(N, dtype=torch.float64, device="cuda")
    for call, (k, sseed) in enumerate(((4, 1), (9, 2))):
        st = random_state(p, k=k, seed=sseed)
        ref_xtz, ref_z = _handle_reference(pkg, d, st, seed)
        bc = np.zeros(ld, dtype=np.float32)
        bc[:p] = st.beta
        bcd = torch.from_numpy(bc).cuda()
        xtz.fill_(np.nan)
        z.fill_(np.nan)
        torch.cuda.synchronize()
        status = lib.hs_probit_xstream_noalloc(
            pkg.X_F32, ctypes.c_void_p(Xd.data_ptr()), ld, ctypes.c_void_p(yd.data_ptr()), N, p,
            ctypes.c_void_p(bcd.data_ptr()), None, seed, 0, 0, k + 1,
            ctypes.c_void_p(xtz.data_ptr()), ctypes.c_void_p(z.data_ptr()), None)
        assert status == 0, (call, status)
        got_xtz, got_z = xtz.cpu().numpy(), z.cpu().numpy()
        # same kernels, same partition, same counters: equal to rounding (1e-4 is the FP32 path tolerance)
        assert np.linalg.norm(got_xtz - ref_xtz) <= 1e-4 * np.linalg.norm(ref_xtz), call
        assert np.all(np.abs(got_z - ref_z) <= 1e-4 * np.maximum(np.abs(ref_z), 1.0)), call
        assert np.array_equal(got_xtz, ref_xtz) and np.array_equal(got_z, ref_z), call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    pkg = lib_pkg()
    lib = pkg.load_library()
    # One row of 8192 FP32 partials per SM (5 MB on 152 SMs) is beyond the
    # fixed 4 MiB: rejected on the host before any launch, so the buffers
    # below (never read) only need to be non-NULL.
    st = lib.hs_probit_xstream_noalloc(pkg.X_F32, ctypes.c_void_p(16), 8192, ctypes.c_void_p(16), 1_000_000,
                                       8192, ctypes.c_void_p(16), None, 0, 0, 0, 1, ctypes.c_void_p(16), None, None)
    assert st == -1
