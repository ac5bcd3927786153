"""The C-ABI library builds, loads and exports every entry point declared in
include/hs_probit.h; host-side argument checks reject bad input before any
CUDA call (CPU only: no kernel runs here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    from paper_1608_04329_gb300 import _build
    import paper_1608_04329_gb300 as pkg
    _build.build()
    return pkg.load_library()


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(hs_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for st in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert lib.hs_probit_status_string(st)


@pytest.mark.parametrize("N,p", [(1, 5), (0, 5), (10, 0), (10, 8193)])
def test_init_rejects_bad_sizes_on_host(lib, N, p):
    X = np.zeros((max(N, 1), max(p, 1)), dtype=np.float32)
    y = np.zeros(max(N, 1), dtype=np.uint8)
    h = lib.hs_probit_init(X.ctypes.data, y.ctypes.data, N, p, 0)
    assert not h
    assert lib.hs_probit_last_error() == -1


def test_init_rejects_bad_y_on_host(lib):
    X = np.zeros((4, 2), dtype=np.float32)
    y = np.array([0, 1, 2, 0], dtype=np.uint8)
    assert not lib.hs_probit_init(X.ctypes.data, y.ctypes.data, 4, 2, 0)
    assert lib.hs_probit_last_error() == -1


def test_null_handle_is_rejected(lib):
    assert lib.hs_probit_sweep(None, 1) == -1
    assert lib.hs_probit_draws_available(None) == -1
    lib.hs_probit_free(None)


def test_config_default(lib):
    import paper_1608_04329_gb300 as pkg
    cfg = pkg._Config()
    lib.hs_probit_config_default(ctypes.byref(cfg))
    assert cfg.x_dtype == pkg.X_F32 and cfg.thin == 1 and cfg.ring_size == 1024 and cfg.use_graph == 0


def test_init_rejects_fp64_rows_beyond_the_kernel(lib):
    import paper_1608_04329_gb300 as pkg
    cfg = pkg._Config()
    lib.hs_probit_config_default(ctypes.byref(cfg))
    cfg.x_dtype = pkg.X_F64
    X = np.zeros((4, 4097), dtype=np.float64)
    y = np.zeros(4, dtype=np.uint8)
    assert not lib.hs_probit_init_ex(ctypes.byref(cfg), X.ctypes.data, y.ctypes.data, 4, 4097, 0)
    assert lib.hs_probit_last_error() == -1


def _no_cuda_device():
    try:
        import torch
        return not torch.cuda.is_available()
    except ImportError:
        return True


# The addresses below are host-side stand-ins that no kernel may ever be given;
# the test runs only where there is no GPU, so even a check that regressed
# could not launch a kernel on them.
@pytest.mark.skipif(not _no_cuda_device(), reason="host-only argument checks; a GPU is present")
def test_noalloc_rejects_bad_arguments_on_host(lib):
    # NULL buffers, a row stride that is not a multiple of 16 bytes, an X that
    # does not start on a 16-byte boundary, misaligned beta_c / xtz / z, and
    # column scales given for a type without them are all rejected before any
    # CUDA call.
    v = ctypes.c_void_p
    assert lib.hs_probit_xstream_noalloc(1, None, 8, None, 10, 8, None, None, 0, 0, 0, 1, None, None, None) == -1
    assert lib.hs_probit_xstream_noalloc(1, v(4096), 5, v(4096), 10, 5, v(4096), None, 0, 0, 0, 1, v(4096), None,
                                         None) == -1
    assert lib.hs_probit_xstream_noalloc(1, v(4096 + 4), 8, v(4096), 10, 8, v(4096), None, 0, 0, 0, 1, v(4096),
                                         None, None) == -1
    assert lib.hs_probit_xstream_noalloc(0, v(4096), 8, v(4096), 10, 8, v(4096 + 4), None, 0, 0, 0, 1, v(4096),
                                         None, None) == -1
    assert lib.hs_probit_xstream_noalloc(1, v(4096), 8, v(4096), 10, 8, v(4096), None, 0, 0, 0, 1, v(4096 + 4),
                                         None, None) == -1
    assert lib.hs_probit_xstream_noalloc(1, v(4096), 8, v(4096), 10, 8, v(4096), None, 0, 0, 0, 1, v(4096),
                                         v(4096 + 4), None) == -1
    assert lib.hs_probit_xstream_noalloc(1, v(4096), 8, v(4096), 10, 8, v(4096), v(4096), 0, 0, 0, 1, v(4096),
                                         None, None) == -1
    assert lib.hs_probit_xstream_noalloc(3, v(4096), 16, v(4096), 10, 16, v(4096), None, 0, 0, 0, 1, v(4096),
                                         None, None) == -1


def test_tn_sample_rejects_bad_arguments_on_host(lib):
    # nothing is launched for these: n < 0, NULL arrays with n > 0, unknown method, chain id too large
    assert lib.hs_tn_sample(None, -1, 0, 0, 1, 0, None, None, None) == -1
    assert lib.hs_tn_sample(None, 5, 0, 0, 1, 0, None, None, None) == -1
    assert lib.hs_tn_sample(None, 0, 0, 0, 1, 7, None, None, None) == -1
    assert lib.hs_tn_sample(None, 0, 0, 1 << 24, 1, 0, None, None, None) == -1
    assert lib.hs_tn_sample(None, 0, 0, 0, 1, 1, None, None, None) == 0  # empty input: nothing to do


@pytest.mark.parametrize("field,value,dtype,p,status", [
    ("num_chains", 33, "bf16", 64, -1),      # more than 32 chains
    ("num_chains", -1, "bf16", 64, -1),
    ("beta_solve", 3, "f32", 64, -1),        # unknown beta form
    ("chol_sched", 4, "f32", 64, -1),        # unknown schedule
])
def test_init_rejects_bad_config_on_host(lib, field, value, dtype, p, status):
    import paper_1608_04329_gb300 as pkg
    cfg = pkg._Config()
    lib.hs_probit_config_default(ctypes.byref(cfg))
    cfg.x_dtype = {"f32": pkg.X_F32, "bf16": pkg.X_BF16}[dtype]
    setattr(cfg, field, value)
    X = np.zeros((4, p), dtype=np.float32 if dtype == "f32" else np.uint16)
    y = np.zeros(4, dtype=np.uint8)
    assert not lib.hs_probit_init_ex(ctypes.byref(cfg), X.ctypes.data, y.ctypes.data, 4, p, 0)
    assert lib.hs_probit_last_error() == status


def test_batch_and_launch_shape_reject_bad_arguments_on_host(lib):
    import paper_1608_04329_gb300 as pkg
    cfg = pkg._Config()
    lib.hs_probit_config_default(ctypes.byref(cfg))
    probs = (pkg._Problem * 2)()
    X = np.zeros((4, 3), dtype=np.float32)
    y = np.zeros(4, dtype=np.uint8)
    probs[0] = pkg._Problem(X.ctypes.data, y.ctypes.data, 4, 3, None)
    probs[1] = pkg._Problem(X.ctypes.data, y.ctypes.data, 1, 3, None)  # N < 2
    for args in ((None, 1, probs), (ctypes.byref(cfg), 0, probs), (ctypes.byref(cfg), 1, None),
                 (ctypes.byref(cfg), 2, probs)):
        assert not lib.hs_probit_batch_init(*args, 0)
        assert lib.hs_probit_last_error() == -1
    assert lib.hs_probit_batch_size(None) == -1
    assert lib.hs_probit_batch_problem(None, 0) is None
    assert lib.hs_probit_batch_sweep(None, 1) == -1
    assert lib.hs_probit_batch_tune(None, 1, None) == -1
    assert lib.hs_probit_batch_tune_trials(None, None, 0) == -1
    lib.hs_probit_batch_free(None)
    ls = pkg._LaunchShape()
    assert lib.hs_probit_get_launch_shape(None, ctypes.byref(ls)) == -1
    assert lib.hs_probit_set_launch_shape(None, ctypes.byref(ls)) == -1
