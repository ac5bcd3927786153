"""GB300 (sm_103a) Gibbs sampler for Horseshoe probit regression.

Python binding of ``lib/libhs_probit.so``, whose C ABI is declared in
``include/hs_probit.h``.  The binding only marshals arguments: every step of a
sweep runs in the library's CUDA kernels.  If the library is missing or cannot
be loaded, every entry point raises; there is no CPU fallback.

Model (Terenin, Dong & Draper, Sect. 5): probit likelihood through latent z
(Eq. 9), horseshoe prior (Eq. 10), full conditionals of Eq. 12, sampled in the
order (i) z and lambda^{-2}, then tau^{-2}; (ii) beta, nu^{-1}, xi^{-1}.

    import numpy as np, paper_1608_04329_gb300 as hs
    s = hs.HSProbit(X.astype(np.float32), y, seed=0)
    s.sweep(1000)
    d = s.draws()            # {"beta": (n, p), "lambda_inv2": (n, p), "tau_inv2": (n,)}
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["HSProbit", "HSProbitError", "load_library", "library_path", "STATUS",
           "X_F64", "X_F32", "X_BF16", "X_FP8E4M3", "CHOL_F64", "CHOL_DF32",
           "SCHED_AUTO", "SCHED_COLUMNS", "SCHED_SINGLE", "SCHED_TENSOR", "BETA_AUTO", "BETA_INVERSE", "BETA_SUBST",
           "TN_INVCDF", "TN_REJECTION", "tn_sample", "HSProbitBatch", "X_ADOPT", "UPD_LAMBDA", "UPD_TAU",
           "UPD_NU", "UPD_XI"]

X_F64, X_F32, X_BF16, X_FP8E4M3 = 0, 1, 2, 3
CHOL_F64, CHOL_DF32 = 0, 1
SCHED_AUTO, SCHED_COLUMNS, SCHED_SINGLE, SCHED_TENSOR = 0, 1, 2, 3
BETA_AUTO, BETA_INVERSE, BETA_SUBST = 0, 1, 2
TN_INVCDF, TN_REJECTION = 0, 1
X_ADOPT = 2
UPD_LAMBDA, UPD_TAU, UPD_NU, UPD_XI = 1, 2, 4, 8
STATUS = {0: "HS_OK", -1: "HS_EINVAL", -2: "HS_ENOMEM", -3: "HS_ECUDA", -4: "HS_ENOTPD",
          -5: "HS_ENONFINITE", -6: "HS_ETIMEOUT", -7: "HS_ESTATE", -8: "HS_EUNSUPPORTED"}
KERNEL_GROUPS = {"xstream": 0, "reduce": 1, "shrink": 2, "cholesky": 3, "tail": 4, "gram": 5}

_PKG = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_PKG, "lib", "libhs_probit.so")


class HSProbitError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: {STATUS.get(int(status), status)} ({int(status)})")


class _Config(ctypes.Structure):
    _fields_ = [("x_dtype", ctypes.c_int32), ("x_is_device", ctypes.c_int32), ("thin", ctypes.c_int32),
                ("ring_size", ctypes.c_int32), ("debug", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("chol_arith", ctypes.c_int32), ("device", ctypes.c_int32), ("chain", ctypes.c_uint32),
                ("problem", ctypes.c_uint32), ("stream", ctypes.c_void_p), ("x_scales", ctypes.c_void_p),
                ("chol_sched", ctypes.c_int32), ("num_chains", ctypes.c_int32), ("beta_solve", ctypes.c_int32),
                ("update_mask", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class _StateView(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_void_p), ("lambda_inv2", ctypes.c_void_p), ("nu_inv", ctypes.c_void_p),
                ("tau_inv2", ctypes.c_double), ("xi_inv", ctypes.c_double), ("k", ctypes.c_int64)]


class _LaunchShape(ctypes.Structure):
    _fields_ = [("xk_chains", ctypes.c_int32), ("xk_stages", ctypes.c_int32), ("xstream_ctas", ctypes.c_int32),
                ("chol_ctas", ctypes.c_int32), ("trail_ctas", ctypes.c_int32), ("xk_ctas_per_sm", ctypes.c_int32),
                ("overlap", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class _Problem(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("y", ctypes.c_void_p), ("N", ctypes.c_int64), ("p", ctypes.c_int64),
                ("x_scales", ctypes.c_void_p)]


class _TuneTrial(ctypes.Structure):
    _fields_ = [("ms_per_sweep", ctypes.c_double), ("oversub", ctypes.c_double), ("chol_oversub", ctypes.c_double),
                ("xk_chains", ctypes.c_int32), ("xk_stages", ctypes.c_int32), ("xk_ctas_per_sm", ctypes.c_int32),
                ("overlap", ctypes.c_int32)]


_LIB = None

# name -> (restype, argtypes)
_PROTOS = {
    "hs_probit_config_default": (None, [ctypes.POINTER(_Config)]),
    "hs_probit_init": (ctypes.c_void_p, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_uint64]),
    "hs_probit_init_ex": (ctypes.c_void_p, [ctypes.POINTER(_Config), ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64]),
    "hs_probit_last_error": (ctypes.c_int, []),
    "hs_probit_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "hs_probit_sweep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "hs_probit_draws": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int64]),
    "hs_probit_draws_available": (ctypes.c_int64, [ctypes.c_void_p]),
    "hs_probit_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_StateView)]),
    "hs_probit_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_StateView)]),
    "hs_probit_debug_z": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hs_probit_debug_xtz": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hs_probit_gram": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "hs_probit_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_void_p)]),
    "hs_probit_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "hs_probit_kernel_time": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_int64)]),
    "hs_probit_launches_per_sweep": (ctypes.c_int64, [ctypes.c_void_p]),
    "hs_probit_debug_wait_timeout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "hs_probit_num_chains": (ctypes.c_int, [ctypes.c_void_p]),
    "hs_probit_draws_available_chain": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_int]),
    "hs_probit_get_state_chain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(_StateView)]),
    "hs_probit_set_state_chain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(_StateView)]),
    "hs_probit_draws_chain": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_int64]),
    "hs_probit_debug_z_chain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "hs_probit_debug_xtz_chain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "hs_probit_free": (None, [ctypes.c_void_p]),
    "hs_chol_task_list": (ctypes.c_int64, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_int64]),
    "hs_probit_debug_factor": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "hs_probit_debug_error_word": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "hs_chol_block_task_list": (ctypes.c_int64, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_void_p, ctypes.c_int64]),
    "hs_tn_sample": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "hs_probit_draws_async": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_int64]),
    "hs_probit_draws_wait": (ctypes.c_int, [ctypes.c_void_p]),
    "hs_probit_get_launch_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_LaunchShape)]),
    "hs_probit_set_launch_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_LaunchShape)]),
    "hs_probit_batch_init": (ctypes.c_void_p, [ctypes.POINTER(_Config), ctypes.c_int32, ctypes.POINTER(_Problem),
                                               ctypes.c_uint64]),
    "hs_probit_batch_size": (ctypes.c_int32, [ctypes.c_void_p]),
    "hs_probit_batch_problem": (ctypes.c_void_p, [ctypes.c_void_p, ctypes.c_int32]),
    "hs_probit_batch_sweep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "hs_probit_batch_tune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "hs_probit_batch_tune_trials": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(_TuneTrial), ctypes.c_int32]),
    "hs_probit_batch_free": (None, [ctypes.c_void_p]),
    "hs_probit_xstream_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                                 ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
}


def load_library(path: str | None = None):
    """Load libhs_probit.so (raises if it is missing: there is no fallback)."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; "
                           "g.build()'` (needs nvcc); this package has no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == library_path():
        _LIB = lib
    return lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def _infer_dtype(X) -> int:
    name = str(getattr(X, "dtype", ""))
    if name.endswith("float64"):
        return X_F64
    if name.endswith("float32"):
        return X_F32
    if name.endswith("bfloat16") or name.endswith("uint16"):
        return X_BF16
    if "float8_e4m3" in name or name.endswith("uint8"):
        return X_FP8E4M3
    raise ValueError(f"unsupported X dtype {name}")


class HSProbit:
    """One Horseshoe-probit Gibbs chain on one GPU.

    X: N x p row-major.  A numpy array (host) or a torch tensor (host or CUDA
    device memory; device tensors are copied by the library on the device).
    Element type: float64, float32, bfloat16 (torch) / uint16 bit patterns, or
    e4m3 (torch float8_e4m3fn / uint8 codes) with ``scales`` (p float32).
    y: N values in {0, 1} (uint8), on the same side (host/device) as X.
    """

    def __init__(self, X, y, seed: int = 0, *, scales=None, thin: int = 1, ring_size: int = 1024,
                 debug: bool = False, use_graph: bool = False, chol_arith: int = CHOL_DF32, chain: int = 0,
                 problem: int = 0, stream=None, device: int = 0, x_dtype: int | None = None,
                 chol_sched: int = SCHED_AUTO, num_chains: int = 1, beta_solve: int = BETA_AUTO,
                 adopt: bool = False, update_mask: int = 0):
        self._lib = load_library()
        self._h = None
        self._adopted = None
        is_dev = hasattr(X, "is_cuda") and bool(X.is_cuda)
        dt = _infer_dtype(X) if x_dtype is None else int(x_dtype)
        self._keep = []
        if hasattr(X, "data_ptr"):
            Xc = X.contiguous()
            yc = y.contiguous()
            self._keep += [Xc, yc]
            xptr, yptr = ctypes.c_void_p(Xc.data_ptr()), ctypes.c_void_p(yc.data_ptr())
            N, p = int(Xc.shape[0]), int(Xc.shape[1])
        else:
            Xc = np.ascontiguousarray(X)
            yc = np.ascontiguousarray(y, dtype=np.uint8)
            self._keep += [Xc, yc]
            xptr, yptr = _ptr(Xc), _ptr(yc)
            N, p = Xc.shape
        cfg = _Config()
        self._lib.hs_probit_config_default(ctypes.byref(cfg))
        cfg.x_dtype = dt
        cfg.x_is_device = (X_ADOPT if adopt else 1) if is_dev else 0
        if adopt and not is_dev:
            raise ValueError("adopt needs X in CUDA device memory")
        cfg.update_mask = update_mask
        cfg.thin = thin
        cfg.ring_size = ring_size
        cfg.debug = 1 if debug else 0
        cfg.use_graph = 1 if use_graph else 0
        cfg.chol_arith = chol_arith
        cfg.chol_sched = chol_sched
        cfg.num_chains = num_chains
        cfg.beta_solve = beta_solve
        cfg.device = device
        cfg.chain = chain
        cfg.problem = problem
        cfg.stream = ctypes.c_void_p(int(stream)) if stream is not None else None
        if scales is not None:
            if hasattr(scales, "data_ptr"):
                sc = scales.contiguous()
                cfg.x_scales = ctypes.c_void_p(sc.data_ptr())
            else:
                sc = np.ascontiguousarray(scales, dtype=np.float32)
                cfg.x_scales = ctypes.c_void_p(sc.ctypes.data)
            self._keep.append(sc)
        h = self._lib.hs_probit_init_ex(ctypes.byref(cfg), xptr, yptr, N, p, ctypes.c_uint64(seed & (2**64 - 1)))
        if not h:
            raise HSProbitError(self._lib.hs_probit_last_error(), "hs_probit_init_ex")
        self._h = ctypes.c_void_p(h)
        if adopt:
            self._adopted = Xc  # the library reads this tensor in place: keep it alive
        self._keep = []
        self.N, self.p, self.seed, self.x_dtype = int(N), int(p), int(seed), dt

    # ---- core ----
    def sweep(self, n: int = 1) -> None:
        st = self._lib.hs_probit_sweep(self._h, int(n))
        if st != 0:
            raise HSProbitError(st, "hs_probit_sweep")

    def sweep_status(self, n: int = 1) -> int:
        return int(self._lib.hs_probit_sweep(self._h, int(n)))

    def num_chains(self) -> int:
        return int(self._lib.hs_probit_num_chains(self._h))

    def draws(self, max_draws: int | None = None, chain: int = 0) -> dict:
        avail = int(self._lib.hs_probit_draws_available_chain(self._h, int(chain)))
        if avail < 0:
            raise HSProbitError(avail, "hs_probit_draws_available_chain")
        n = avail if max_draws is None else min(avail, int(max_draws))
        beta = np.empty((n, self.p))
        lam = np.empty((n, self.p))
        tau = np.empty(n)
        got = self._lib.hs_probit_draws_chain(self._h, int(chain), _ptr(beta), _ptr(lam), _ptr(tau), n)
        if got < 0:
            raise HSProbitError(got, "hs_probit_draws_chain")
        return {"beta": beta[:got], "lambda_inv2": lam[:got], "tau_inv2": tau[:got]}

    def draws_async(self, out: dict, chain: int = 0) -> int:
        """Start copying the chain's unread draws into ``out`` (arrays
        "beta" (n, p), "lambda_inv2" (n, p), "tau_inv2" (n,), float64, ideally
        page-locked) on a side stream; returns how many are being copied.
        Read ``out`` only after ``draws_wait()``."""
        n = min(len(out["beta"]), len(out["lambda_inv2"]), len(out["tau_inv2"]))
        for k in ("beta", "lambda_inv2", "tau_inv2"):
            a = out[k]
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or (k != "tau_inv2" and a.shape[1:] != (self.p,)):
                raise ValueError(f"{k}: C-contiguous float64 with rows of p values expected")
        got = self._lib.hs_probit_draws_async(self._h, int(chain), _ptr(out["beta"]), _ptr(out["lambda_inv2"]),
                                              _ptr(out["tau_inv2"]), n)
        if got < 0:
            raise HSProbitError(got, "hs_probit_draws_async")
        return int(got)

    def draws_wait(self) -> None:
        st = self._lib.hs_probit_draws_wait(self._h)
        if st != 0:
            raise HSProbitError(st, "hs_probit_draws_wait")

    def get_state(self, chain: int = 0) -> dict:
        beta, lam, nu = np.empty(self.p), np.empty(self.p), np.empty(self.p)
        v = _StateView(_ptr(beta).value, _ptr(lam).value, _ptr(nu).value, 0.0, 0.0, 0)
        st = self._lib.hs_probit_get_state_chain(self._h, int(chain), ctypes.byref(v))
        if st != 0:
            raise HSProbitError(st, "hs_probit_get_state_chain")
        return {"beta": beta, "lambda_inv2": lam, "nu_inv": nu, "tau_inv2": v.tau_inv2, "xi_inv": v.xi_inv,
                "k": int(v.k)}

    def set_state(self, beta, lambda_inv2, nu_inv, tau_inv2, xi_inv, k, chain: int = 0) -> None:
        b = np.ascontiguousarray(beta, dtype=np.float64)
        l_ = np.ascontiguousarray(lambda_inv2, dtype=np.float64)
        n_ = np.ascontiguousarray(nu_inv, dtype=np.float64)
        if b.shape != (self.p,) or l_.shape != (self.p,) or n_.shape != (self.p,):
            raise ValueError("state arrays must have length p")
        v = _StateView(_ptr(b).value, _ptr(l_).value, _ptr(n_).value, float(tau_inv2), float(xi_inv), int(k))
        st = self._lib.hs_probit_set_state_chain(self._h, int(chain), ctypes.byref(v))
        if st != 0:
            raise HSProbitError(st, "hs_probit_set_state_chain")

    # ---- debug / inspection ----
    def debug_z(self, chain: int = 0) -> np.ndarray:
        z = np.empty(self.N)
        st = self._lib.hs_probit_debug_z_chain(self._h, int(chain), _ptr(z))
        if st != 0:
            raise HSProbitError(st, "hs_probit_debug_z_chain")
        return z

    def debug_xtz(self, chain: int = 0) -> np.ndarray:
        v = np.empty(self.p)
        st = self._lib.hs_probit_debug_xtz_chain(self._h, int(chain), _ptr(v))
        if st != 0:
            raise HSProbitError(st, "hs_probit_debug_xtz_chain")
        return v

    def gram(self) -> np.ndarray:
        G = np.empty((self.p, self.p))
        st = self._lib.hs_probit_gram(self._h, _ptr(G))
        if st != 0:
            raise HSProbitError(st, "hs_probit_gram")
        return G

    def stream(self) -> int:
        s = ctypes.c_void_p()
        self._lib.hs_probit_info(self._h, None, None, ctypes.byref(s))
        return int(s.value or 0)

    def set_profiling(self, on: bool) -> None:
        self._lib.hs_probit_set_profiling(self._h, 1 if on else 0)

    def kernel_time(self, group: str):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        st = self._lib.hs_probit_kernel_time(self._h, KERNEL_GROUPS[group], ctypes.byref(ms), ctypes.byref(n))
        if st != 0:
            raise HSProbitError(st, "hs_probit_kernel_time")
        return float(ms.value), int(n.value)

    def launches_per_sweep(self) -> int:
        return int(self._lib.hs_probit_launches_per_sweep(self._h))

    def launch_shape(self) -> dict:
        """Grid and tile sizes of the handle's kernels (``hs_probit_get_launch_shape``)."""
        ls = _LaunchShape()
        st = self._lib.hs_probit_get_launch_shape(self._h, ctypes.byref(ls))
        if st != 0:
            raise HSProbitError(st, "hs_probit_get_launch_shape")
        return {f: int(getattr(ls, f)) for f in ("xk_chains", "xk_stages", "xstream_ctas", "chol_ctas", "trail_ctas",
                                                 "xk_ctas_per_sm", "overlap")}

    def set_launch_shape(self, **sizes) -> None:
        """Change launch sizes (keyword per field; omitted fields stay)."""
        ls = _LaunchShape()
        for k, v in sizes.items():
            setattr(ls, k, int(v))
        st = self._lib.hs_probit_set_launch_shape(self._h, ctypes.byref(ls))
        if st != 0:
            raise HSProbitError(st, "hs_probit_set_launch_shape")

    def debug_factor(self, chain: int = 0) -> np.ndarray:
        """The factorization's P x P work matrix of one chain (lower tiles: the factor)."""
        P = (self.p + 31) // 32 * 32
        L = np.empty((P, P))
        st = self._lib.hs_probit_debug_factor(self._h, int(chain), _ptr(L))
        if st != 0:
            raise HSProbitError(st, "hs_probit_debug_factor")
        return L

    def debug_error_word(self) -> int:
        """The raw device error word of the last sweep (status and wait-site bits)."""
        w = ctypes.c_int()
        self._lib.hs_probit_debug_error_word(self._h, ctypes.byref(w))
        return int(w.value)

    def debug_wait_timeout(self, max_spins: int) -> int:
        return int(self._lib.hs_probit_debug_wait_timeout(self._h, int(max_spins)))

    @classmethod
    def _member(cls, lib, handle, N: int, p: int, seed: int, x_dtype: int, owner) -> "HSProbit":
        """A view of a handle another object owns (a batch's problem)."""
        self = cls.__new__(cls)
        self._lib, self._h, self._keep, self._owner = lib, ctypes.c_void_p(handle), [], owner
        self.N, self.p, self.seed, self.x_dtype = int(N), int(p), int(seed), int(x_dtype)
        return self

    def close(self) -> None:
        if getattr(self, "_owner", None) is not None:
            self._h = None  # the owner frees the handle
            return
        if self._h is not None and self._lib is not None:
            self._lib.hs_probit_free(self._h)
        self._h = None
        self._adopted = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class HSProbitBatch:
    """Independent problems of uneven N and p swept together (``hs_probit_batch_*``).

    problems: list of (X, y) or (X, y, scales), host numpy arrays or torch
    tensors (all host or all CUDA), X of one element type.  Problem m uses
    Philox problem id ``problem + m``; each has ``num_chains`` chains.  One
    ``sweep(n)`` replays, n times, one CUDA graph that holds a sweep of every
    problem.  ``problem(m)`` gives problem m's handle as an ``HSProbit``.
    """

    def __init__(self, problems, seed: int = 0, *, num_chains: int = 1, thin: int = 1, ring_size: int = 1024,
                 debug: bool = False, chol_arith: int = CHOL_DF32, chain: int = 0, problem: int = 0, stream=None,
                 device: int = 0, x_dtype: int | None = None, chol_sched: int = SCHED_AUTO,
                 beta_solve: int = BETA_AUTO):
        self._lib = load_library()
        self._b = None
        if not problems:
            raise ValueError("no problems")
        keep, arr = [], (_Problem * len(problems))()
        dts, dev = set(), set()
        for m, pr in enumerate(problems):
            X, y = pr[0], pr[1]
            sc = pr[2] if len(pr) > 2 else None
            dts.add(_infer_dtype(X) if x_dtype is None else int(x_dtype))
            dev.add(bool(getattr(X, "is_cuda", False)))
            if hasattr(X, "data_ptr"):
                Xc, yc = X.contiguous(), y.contiguous()
                xp, yp = Xc.data_ptr(), yc.data_ptr()
            else:
                Xc, yc = np.ascontiguousarray(X), np.ascontiguousarray(y, dtype=np.uint8)
                xp, yp = Xc.ctypes.data, yc.ctypes.data
            keep += [Xc, yc]
            sp = None
            if sc is not None:
                scc = sc.contiguous() if hasattr(sc, "data_ptr") else np.ascontiguousarray(sc, dtype=np.float32)
                keep.append(scc)
                sp = scc.data_ptr() if hasattr(scc, "data_ptr") else scc.ctypes.data
            arr[m] = _Problem(xp, yp, int(Xc.shape[0]), int(Xc.shape[1]), sp)
        if len(dts) != 1 or len(dev) != 1:
            raise ValueError("every problem's X must have one element type and sit on one side (host or device)")
        cfg = _Config()
        self._lib.hs_probit_config_default(ctypes.byref(cfg))
        cfg.x_dtype = dts.pop()
        cfg.x_is_device = 1 if dev.pop() else 0
        cfg.thin, cfg.ring_size, cfg.debug = thin, ring_size, 1 if debug else 0
        cfg.chol_arith, cfg.chol_sched, cfg.num_chains, cfg.beta_solve = chol_arith, chol_sched, num_chains, beta_solve
        cfg.device, cfg.chain, cfg.problem = device, chain, problem
        cfg.stream = ctypes.c_void_p(int(stream)) if stream is not None else None
        b = self._lib.hs_probit_batch_init(ctypes.byref(cfg), len(problems), arr, ctypes.c_uint64(seed & (2**64 - 1)))
        if not b:
            raise HSProbitError(self._lib.hs_probit_last_error(), "hs_probit_batch_init")
        self._b = ctypes.c_void_p(b)
        self._members = [HSProbit._member(self._lib, self._lib.hs_probit_batch_problem(self._b, m),
                                          arr[m].N, arr[m].p, seed, cfg.x_dtype, self)
                         for m in range(len(problems))]
        self.seed = int(seed)

    def __len__(self) -> int:
        return len(self._members)

    def problem(self, m: int) -> HSProbit:
        return self._members[m]

    def sweep(self, n: int = 1) -> None:
        st = self._lib.hs_probit_batch_sweep(self._b, int(n))
        if st != 0:
            raise HSProbitError(st, "hs_probit_batch_sweep")

    def tune(self, sweeps: int = 3) -> float:
        """Run the autotuner; returns the best ms per batch sweep."""
        ms = ctypes.c_double()
        st = self._lib.hs_probit_batch_tune(self._b, int(sweeps), ctypes.byref(ms))
        if st != 0:
            raise HSProbitError(st, "hs_probit_batch_tune")
        return float(ms.value)

    def tune_trials(self) -> list:
        n = int(self._lib.hs_probit_batch_tune_trials(self._b, None, 0))
        arr = (_TuneTrial * max(n, 1))()
        self._lib.hs_probit_batch_tune_trials(self._b, arr, n)
        return [{"ms_per_sweep": t.ms_per_sweep, "oversub": t.oversub, "chol_oversub": t.chol_oversub,
                 "xk_chains": t.xk_chains, "xk_ctas_per_sm": t.xk_ctas_per_sm, "overlap": t.overlap,
                 "xk_stages": t.xk_stages} for t in arr[:n]]

    def close(self) -> None:
        for h in getattr(self, "_members", []):
            h._h = None
        if self._b is not None and self._lib is not None:
            self._lib.hs_probit_batch_free(self._b)
        self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def tn_sample(mu, seed: int = 0, sweep: int = 1, method: int = TN_INVCDF, chain: int = 0, stream=None):
    """z+ ~ N(mu, 1) restricted to (0, inf) for a CUDA float32 tensor mu, by the
    inverse CDF or the paper's rejection sampler (``hs_tn_sample``); returns
    (z, attempts) as CUDA tensors, enqueued on ``stream`` (a torch stream or a
    raw handle; default: torch's current stream)."""
    import torch
    if not (hasattr(mu, "is_cuda") and mu.is_cuda and mu.dtype == torch.float32):
        raise HSProbitError(-1, "tn_sample: mu must be a CUDA float32 tensor")
    mu = mu.contiguous()
    z = torch.empty_like(mu)
    tries = torch.empty(mu.shape, dtype=torch.int32, device=mu.device)
    if stream is None:
        stream = torch.cuda.current_stream(mu.device)
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    st = load_library().hs_tn_sample(ctypes.c_void_p(mu.data_ptr()), mu.numel(), ctypes.c_uint64(seed & (2**64 - 1)),
                                     chain, sweep, method, ctypes.c_void_p(z.data_ptr()),
                                     ctypes.c_void_p(tries.data_ptr()), ctypes.c_void_p(handle))
    if st != 0:
        raise HSProbitError(st, "hs_tn_sample")
    return z, tries
