"""Helpers of the GPU tests: build/load the library, run one transition on the
GPU and in the oracle from the same state and counters."""
import numpy as np

import hs_synth
import oracle
from oracle import fmt

X_DTYPES = {"f64": 0, "f32": 1, "bf16": 2, "fp8": 3}


def lib_pkg():
    from paper_1608_04329_gb300 import _build
    import paper_1608_04329_gb300 as pkg
    _build.build()
    pkg.load_library()
    return pkg


def random_state(p, k=7, seed=0, scale=0.5):
    r = np.random.default_rng(seed)
    return oracle.State(r.normal(0, scale, p), r.exponential(size=p) + 0.05, r.exponential(size=p) + 0.05,
                        float(r.uniform(0.2, 3.0)), float(r.uniform(0.2, 3.0)), k)


def x_f64(d):
    return fmt.stored_to_f64(d["X"], d["x_dtype"], d["scales"])


def gpu_transition(pkg, d, st, seed, **kw):
    s = pkg.HSProbit(d["X"], d["y"], seed=seed, scales=d["scales"], debug=True, **kw)
    try:
        s.set_state(st.beta, st.lam_inv2, st.nu_inv, st.tau_inv2, st.xi_inv, st.k)
        s.sweep(1)
        out = s.get_state()
        out["z"] = s.debug_z()
        out["xtz"] = s.debug_xtz()
    finally:
        s.close()
    return out


def oracle_transition(d, st, seed, G=None):
    X = x_f64(d)
    if G is None:
        G = oracle.gram(X)
    return oracle.sweep_once(st.copy(), X, d["y"], G, seed, keep=True)


def assert_transition_close(got, ref, tol, tol_exact=1e-12):
    """tol: mixed tolerance for z (|dz| <= tol max(|z|,1)) and normwise for
    beta and X^T z; tol_exact: relative tolerance of the variables whose
    inputs are identical on both sides (lambda, tau, nu, xi)."""
    z, zt = got["z"], ref.extra["z"]
    assert np.all(np.sign(z) == np.sign(zt)) and np.all(z != 0)
    dz = np.abs(z - zt) / np.maximum(np.abs(zt), 1.0)
    assert dz.max() <= tol, ("z", dz.max(), int(dz.argmax()))
    xt = ref.extra["xtz"]
    assert np.linalg.norm(got["xtz"] - xt) <= tol * max(np.linalg.norm(xt), 1.0), "xtz"
    db = np.linalg.norm(got["beta"] - ref.beta) / max(np.linalg.norm(ref.beta), 1e-300)
    assert db <= tol, ("beta", db)
    np.testing.assert_allclose(got["lambda_inv2"], ref.lam_inv2, rtol=tol_exact)
    np.testing.assert_allclose(got["tau_inv2"], ref.tau_inv2, rtol=tol_exact)
    np.testing.assert_allclose(got["nu_inv"], ref.nu_inv, rtol=max(tol_exact, 1e-12))
    np.testing.assert_allclose(got["xi_inv"], ref.xi_inv, rtol=max(tol_exact, 1e-12))
    assert got["k"] == ref.k


def problem(N, p, nz, dt, seed=0, **kw):
    return hs_synth.make_problem(N, p, nz, dt, seed=seed, **kw)
