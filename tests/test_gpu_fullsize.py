"""Full-size transition parity: the benchmark workload (N = 1e6, p = 1000,
FP32 X, 10 nonzeros, seed 0) in the benchmark's launch configuration (CUDA
graph, FP32-pair factorization), one sweep from a mid-chain state, against
the oracle's full FP64 sweep from the same state and counters."""
import numpy as np
import pytest

from tests.gpu_common import assert_transition_close, lib_pkg, oracle_transition, problem, random_state

pytestmark = pytest.mark.gpu


def test_c1_full_size_transition():
    pkg = lib_pkg()
    d = problem(1_000_000, 1000, 10, "f32", seed=0)
    st = random_state(1000, k=20, seed=7, scale=0.05)
    st.beta[np.nonzero(d["beta_true"])[0]] = d["beta_true"][d["beta_true"] != 0]
    s = pkg.HSProbit(d["X"], d["y"], seed=0, debug=True, use_graph=True, chol_arith=pkg.CHOL_DF32)
    try:
        s.set_state(st.beta, st.lam_inv2, st.nu_inv, st.tau_inv2, st.xi_inv, st.k)
        s.sweep(1)
        got = s.get_state()
        got["z"] = s.debug_z()
        got["xtz"] = s.debug_xtz()
    finally:
        s.close()
    ref = oracle_transition(d, st, seed=0)
    assert_transition_close(got, ref, 1e-4)


def test_c2_full_size_chains():
    """The batched workload at full size (N = 1e6, p = 1000, BF16 X, K = 32
    chains, CUDA graph, factor-only factorization with block substitution):
    every chain's transition against the oracle's full FP64 sweep for that
    chain id, with the batched form's derived z bound (row bound computed
    in chunks of X)."""
    from tests.test_gpu_batched import assert_batched_close
    import oracle
    from tests.gpu_common import x_f64
    pkg = lib_pkg()
    K = 32
    d = problem(1_000_000, 1000, 10, "bf16", seed=0)
    states = []
    for m in range(K):
        st = random_state(1000, k=20, seed=100 + m, scale=0.05)
        st.beta[np.nonzero(d["beta_true"])[0]] = d["beta_true"][d["beta_true"] != 0]
        states.append(st)
    s = pkg.HSProbit(d["X"], d["y"], seed=0, debug=True, use_graph=True, num_chains=K)
    got = []
    try:
        for m, st in enumerate(states):
            s.set_state(st.beta, st.lam_inv2, st.nu_inv, st.tau_inv2, st.xi_inv, st.k, chain=m)
        s.sweep(1)
        for m in range(K):
            g = s.get_state(chain=m)
            g["z"] = s.debug_z(chain=m)
            g["xtz"] = s.debug_xtz(chain=m)
            got.append(g)
    finally:
        s.close()
    X = x_f64(d)
    G = oracle.gram(X)
    for m, st in enumerate(states):
        ref = oracle.sweep_once(st.copy(), X, d["y"], G, 0, chain=m, keep=True)
        assert_batched_close(got[m], ref, X, st.beta)
