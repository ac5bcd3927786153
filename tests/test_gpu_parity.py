"""GPU vs oracle: one Gibbs transition from an identical state with identical
counters (Eq. 12 and the schedule of Sect. 5), through the C ABI.

Tolerances: FP64-X path relative 1e-10 on z (mixed abs/rel) and on beta and
X^T z (normwise); FP32-accumulation paths (f32, bf16, fp8 X) 1e-4; the
variables whose inputs are identical on both sides (lambda^{-2}, tau^{-2},
nu^{-1}, xi^{-1}) 1e-12 relative.
"""
import numpy as np
import pytest

from tests.gpu_common import (assert_transition_close, gpu_transition, lib_pkg, oracle_transition, problem,
                              random_state, x_f64)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return lib_pkg()


@pytest.mark.parametrize("chol", [0, 1], ids=["chol_f64", "chol_df32"])
@pytest.mark.parametrize("state_kind", ["cold", "mid"])
def test_c0_shape_fp64(pkg, state_kind, chol):
    d = problem(10000, 100, 5, "f64")
    import oracle
    st = oracle.init_state(100) if state_kind == "cold" else random_state(100, k=41)
    got = gpu_transition(pkg, d, st, seed=0, chol_arith=chol)
    ref = oracle_transition(d, st, seed=0)
    assert_transition_close(got, ref, 1e-10)


@pytest.mark.parametrize("chol", [0, 1], ids=["chol_f64", "chol_df32"])
@pytest.mark.parametrize("N,p", [(2, 1), (37, 3), (1001, 33), (5003, 257), (3001, 600), (999, 1100)])
def test_ragged_shapes_fp64(pkg, N, p, chol):
    d = problem(N, p, min(3, p), "f64", seed=N + p)
    st = random_state(p, k=3, seed=p)
    got = gpu_transition(pkg, d, st, seed=99, chol_arith=chol)
    ref = oracle_transition(d, st, seed=99)
    assert_transition_close(got, ref, 1e-10)


@pytest.mark.parametrize("N,p", [(37, 3), (1001, 33), (5003, 257), (3001, 600), (999, 1100), (2, 1)])
def test_beta_by_substitution_fp64(pkg, N, p):
    """beta by block forward and back substitution with the factor (the
    factorization without the inverse factor), FP64 X: same bar as the
    explicit-inverse form."""
    d = problem(N, p, min(3, p), "f64", seed=N + 2 * p)
    st = random_state(p, k=5, seed=p + 1)
    got = gpu_transition(pkg, d, st, seed=17, chol_arith=1, chol_sched=pkg.SCHED_SINGLE, beta_solve=pkg.BETA_SUBST)
    ref = oracle_transition(d, st, seed=17)
    assert_transition_close(got, ref, 1e-10)


@pytest.mark.parametrize("dt,N,p", [("f32", 20003, 200), ("f32", 4099, 1100), ("bf16", 9001, 300),
                                    ("fp8", 7001, 130), ("f32", 3, 2)])
def test_fp32_accumulation_paths(pkg, dt, N, p):
    d = problem(N, p, 5, dt, seed=7)
    st = random_state(p, k=11, seed=5)
    got = gpu_transition(pkg, d, st, seed=2024, chol_arith=1)
    ref = oracle_transition(d, st, seed=2024)
    assert_transition_close(got, ref, 1e-4)


@pytest.mark.parametrize("dt,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_truncated_normal_tails(pkg, dt, tol):
    """Rows with |x_i beta| up to ~90 and random y exercise both tail arms
    (mu* < -30 in FP64, < -9 in FP32) and the far-right main arm."""
    N, p = 4000, 8
    r = np.random.default_rng(3)
    X = r.normal(size=(N, p)) * r.uniform(0.1, 12.0, size=(N, 1))
    y = r.integers(0, 2, N).astype(np.uint8)
    d = {"X": X if dt == "f64" else X.astype(np.float32), "y": y, "scales": None, "x_dtype": dt}
    import oracle
    st = oracle.State(r.choice([-3.0, 3.0], p), np.ones(p), np.ones(p), 1.0, 1.0, 2)
    got = gpu_transition(pkg, d, st, seed=5)
    ref = oracle_transition(d, st, seed=5)
    mu = (2.0 * y - 1) * (X @ st.beta)
    assert (mu < -30).sum() > 50 and (mu < -9).sum() > 100 and (mu > 30).sum() > 50
    assert_transition_close(got, ref, tol)


def test_trajectory_fp64(pkg):
    """30 sweeps from the cold start stay on the oracle's trajectory."""
    import oracle
    d = problem(3000, 20, 3, "f64", seed=11)
    s = pkg.HSProbit(d["X"], d["y"], seed=77)
    s.sweep(30)
    got = s.get_state()
    s.close()
    st, _, _, _ = oracle.run(oracle.init_state(20), d["X"], d["y"], oracle.gram(d["X"]), 77, 30)
    assert np.linalg.norm(got["beta"] - st.beta) <= 1e-8 * np.linalg.norm(st.beta)
    np.testing.assert_allclose(got["lambda_inv2"], st.lam_inv2, rtol=1e-8)
    np.testing.assert_allclose(got["tau_inv2"], st.tau_inv2, rtol=1e-8)
    assert got["k"] == 30


@pytest.mark.parametrize("dt,N,p", [("f32", 5003, 257), ("f32", 2, 1), ("f64", 3001, 100), ("bf16", 4099, 130),
                                    ("fp8", 2999, 200), ("f32", 40000, 64), ("bf16", 300, 1100), ("f64", 37, 33)])
def test_gram_on_tensor_cores_matches_definition(pkg, dt, N, p):
    """X^T X of the stored X from exact BF16 digit products on the tensor
    cores: every entry within 1e-12 of sum_r |x_ri x_rj| of the FP64
    definition (ragged tiles: p not a multiple of 64 or 128, N not a multiple
    of the 32-row stage or the 128-row window), and exactly symmetric."""
    d = problem(N, p, min(3, p), dt, seed=p + N)
    s = pkg.HSProbit(d["X"], d["y"], seed=1, scales=d["scales"])
    G = s.gram()
    s.close()
    X = x_f64(d)
    ref = X.T @ X
    nrm = np.abs(X).T @ np.abs(X)
    err = np.abs(G - ref) / np.maximum(nrm, 1e-300)
    assert err.max() <= 1e-12, (err.max(), np.unravel_index(err.argmax(), err.shape))
    assert np.array_equal(G, G.T)


def test_gram_matches_definition(pkg):
    d = problem(5000, 70, 3, "f32", seed=2)
    s = pkg.HSProbit(d["X"], d["y"], seed=1)
    G = s.gram()
    s.close()
    X = d["X"].astype(np.float64)
    ref = X.T @ X
    assert np.abs(G - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.array_equal(G, G.T)


def test_fp8_correlated_design_large_p(pkg):
    """The shape of the large correlated workload at a size the oracle runs in
    seconds: FP8 e4m3 X with per-column scales, rows from the AR(1) Toeplitz
    design (rho = 0.5), p = 4000 (125 tiles), 20 nonzeros of magnitude
    U[0.5, 2]; FP32 accumulation tolerance."""
    d = problem(20000, 4000, 20, "fp8", seed=4, mag=(0.5, 2.0), design="ar1")
    st = random_state(4000, k=6, seed=8, scale=0.05)
    got = gpu_transition(pkg, d, st, seed=41, chol_arith=1)
    ref = oracle_transition(d, st, seed=41)
    assert_transition_close(got, ref, 1e-4)
