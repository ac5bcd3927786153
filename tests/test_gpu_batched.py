"""K chains on one BF16 X through the C ABI: the tensor-core X-stream (eta = X B
and X^T Z with two-part BF16 operands) and the per-chain factorization and
draws.  Chain m of a K-chain handle must reproduce the oracle's transition
for chain id (chain + m) from the same state (Eq. 12 and the schedule of
Sect. 5).

Tolerance.  X is exact in BF16; beta enters the tensor cores as hi + lo, two
BF16 numbers, so each beta_j carries a relative error of at most 2^-16 (two
roundings to 8 significant bits), and the products accumulate in FP32 over p
terms.  Hence per row |d eta_i| <= (2^-16 + p 2^-24) sum_j |x_ij beta_j|, and
since the truncated-normal quantile moves by at most as much as its mean,
|d z_i| is bounded by the same amount plus the FP32 sampler's own error
(1e-5 max(|z|, 1), as on the single-chain FP32 path).  X^T z (z also split
in two parts) and beta are compared normwise at 1e-4; lambda, tau, nu, xi
have identical inputs on both sides (1e-12).
"""
import numpy as np
import pytest

import oracle
from tests.gpu_common import assert_transition_close, lib_pkg, problem, random_state, x_f64


def row_abs_dot(X, b, chunk=65536):
    """sum_j |x_ij b_j| per row, a chunk of rows at a time (no N x p temporary)."""
    out = np.empty(X.shape[0])
    ab = np.abs(b)
    for s in range(0, X.shape[0], chunk):
        out[s:s + chunk] = np.abs(X[s:s + chunk]) @ ab
    return out


def assert_batched_close(got, ref, X, beta0):
    z, zt = got["z"], ref.extra["z"]
    assert np.all(np.sign(z) == np.sign(zt)) and np.all(z != 0)
    p = X.shape[1]
    bound = (2.0**-16 + p * 2.0**-24) * row_abs_dot(X, beta0) + 1e-5 * np.maximum(np.abs(zt), 1.0)
    excess = np.abs(z - zt) / bound
    assert excess.max() <= 1.0, ("z", excess.max(), int(excess.argmax()))
    xt = ref.extra["xtz"]
    assert np.linalg.norm(got["xtz"] - xt) <= 1e-4 * max(np.linalg.norm(xt), 1.0), "xtz"
    db = np.linalg.norm(got["beta"] - ref.beta) / max(np.linalg.norm(ref.beta), 1e-300)
    assert db <= 1e-4, ("beta", db)
    np.testing.assert_allclose(got["lambda_inv2"], ref.lam_inv2, rtol=1e-12)
    np.testing.assert_allclose(got["tau_inv2"], ref.tau_inv2, rtol=1e-12)
    np.testing.assert_allclose(got["nu_inv"], ref.nu_inv, rtol=1e-12)
    np.testing.assert_allclose(got["xi_inv"], ref.xi_inv, rtol=1e-12)
    assert got["k"] == ref.k

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return lib_pkg()


def _batched_transitions(pkg, d, states, seed, chain0=0, **kw):
    K = len(states)
    s = pkg.HSProbit(d["X"], d["y"], seed=seed, debug=True, num_chains=K, chain=chain0, **kw)
    try:
        assert s.num_chains() == K
        for m, st in enumerate(states):
            s.set_state(st.beta, st.lam_inv2, st.nu_inv, st.tau_inv2, st.xi_inv, st.k, chain=m)
        s.sweep(1)
        out = []
        for m in range(K):
            g = s.get_state(chain=m)
            g["z"] = s.debug_z(chain=m)
            g["xtz"] = s.debug_xtz(chain=m)
            out.append(g)
    finally:
        s.close()
    return out


@pytest.mark.parametrize("N,p,K", [(3001, 200, 5), (1000, 64, 2), (20003, 1000, 32), (257, 1, 3), (4099, 1100, 8),
                                   (9001, 2000, 4), (5003, 3584, 16)])
def test_batched_chains_match_oracle(pkg, N, p, K):
    d = problem(N, p, min(5, p), "bf16", seed=N % 97)
    X = x_f64(d)
    G = oracle.gram(X)
    states = [random_state(p, k=9, seed=100 + m) for m in range(K)]
    got = _batched_transitions(pkg, d, states, seed=321, chain0=7)
    for m, st in enumerate(states):
        ref = oracle.sweep_once(st.copy(), X, d["y"], G, 321, chain=7 + m, keep=True)
        assert_batched_close(got[m], ref, X, st.beta)


@pytest.mark.parametrize("N,p,K", [(3001, 200, 5), (4099, 1100, 3)])
def test_batched_inverse_and_substitution_agree(pkg, N, p, K):
    """The two ways of applying the factor (explicit inverse products, block
    substitution) give the same transition up to rounding: z, X^T z and the
    exact variables identical, beta to 1e-12."""
    d = problem(N, p, 5, "bf16", seed=p)
    states = [random_state(p, k=4, seed=200 + m) for m in range(K)]
    a = _batched_transitions(pkg, d, states, seed=5, beta_solve=pkg.BETA_INVERSE)
    b = _batched_transitions(pkg, d, states, seed=5, beta_solve=pkg.BETA_SUBST)
    for ga, gb in zip(a, b):
        assert np.array_equal(ga["z"], gb["z"]) and np.array_equal(ga["xtz"], gb["xtz"])
        assert np.array_equal(ga["lambda_inv2"], gb["lambda_inv2"]) and ga["tau_inv2"] == gb["tau_inv2"]
        db = np.linalg.norm(ga["beta"] - gb["beta"]) / np.linalg.norm(ga["beta"])
        assert db <= 1e-12, db


def test_batched_graph_equals_eager_and_chains_differ(pkg):
    d = problem(5000, 300, 5, "bf16", seed=3)
    outs = []
    for graph in (False, True):
        s = pkg.HSProbit(d["X"], d["y"], seed=11, num_chains=4, use_graph=graph)
        s.sweep(3)
        outs.append([s.get_state(chain=m)["beta"] for m in range(4)])
        s.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    assert not np.array_equal(outs[0][0], outs[0][1])


def test_batched_draw_rings_per_chain(pkg):
    d = problem(3000, 50, 3, "bf16", seed=5)
    s = pkg.HSProbit(d["X"], d["y"], seed=2, num_chains=3, ring_size=8)
    s.sweep(5)
    for m in range(3):
        dr = s.draws(chain=m)
        assert dr["beta"].shape == (5, 50)
        assert np.array_equal(dr["beta"][-1], s.get_state(chain=m)["beta"])
    s.close()


@pytest.mark.parametrize("dt,N,p,K,tol", [("f32", 3001, 200, 3, 1e-4), ("f64", 2001, 130, 2, 1e-10),
                                           ("f32", 1000, 1, 2, 1e-4)])
def test_chains_without_tensor_core_xstream_match_oracle(pkg, dt, N, p, K, tol):
    """K chains on F32 or F64 X: one pass of the one-chain X-stream per chain,
    the rest batched; each chain reproduces the oracle's transition at the
    one-chain path's tolerance for that X type."""
    d = problem(N, p, min(5, p), dt, seed=N % 89)
    X = x_f64(d)
    G = oracle.gram(X)
    states = [random_state(p, k=3, seed=300 + m) for m in range(K)]
    got = _batched_transitions(pkg, d, states, seed=77, chain0=2)
    for m, st in enumerate(states):
        ref = oracle.sweep_once(st.copy(), X, d["y"], G, 77, chain=2 + m, keep=True)
        assert_transition_close(got[m], ref, tol)


@pytest.mark.parametrize("N,p,K", [(3001, 1600, 20), (4099, 4000, 4), (1000, 2048, 32)])
def test_bf16_chains_past_the_fused_kernels_tmem_budget_match_oracle(pkg, N, p, K):
    """Past the fused kernel's TMEM budget (p = 1536 at 32 chain columns,
    3584 at 16) the tensor-core X-stream runs as two kernels, pass 1 writing
    Z^T for pass 2; each chain stays within the batched form's BF16 bound."""
    d = problem(N, p, 5, "bf16", seed=p % 13)
    X = x_f64(d)
    G = oracle.gram(X)
    states = [random_state(p, k=2, seed=400 + m, scale=0.2) for m in range(K)]
    s = pkg.HSProbit(d["X"], d["y"], seed=1, num_chains=K)
    assert s.launch_shape()["xk_chains"] == (16 if K <= 16 else 32)
    s.close()
    got = _batched_transitions(pkg, d, states, seed=13)
    for m, st in enumerate(states):
        ref = oracle.sweep_once(st.copy(), X, d["y"], G, 13, chain=m, keep=True)
        assert_batched_close(got[m], ref, X, st.beta)


def test_batched_long_run_moments_match_oracle_within_mc_error(pkg):
    """Long run of the batched form (16 chains, BF16 X) against a long oracle
    chain on the same stored X: posterior means of beta agree within Monte
    Carlo error (GPU: between-chain standard error of 16 independent chains;
    oracle: batch means), and so do the posterior variances."""
    d = problem(2000, 10, 3, "bf16", seed=22)
    X = x_f64(d)
    K, n, burn = 16, 500, 100
    s = pkg.HSProbit(d["X"], d["y"], seed=3, num_chains=K, ring_size=n)
    try:
        s.sweep(n)
        draws = [s.draws(chain=m)["beta"][burn:] for m in range(K)]
        per_chain = np.stack([b.mean(0) for b in draws])
        # the chain's variance about its own mean; 400 draws make the
        # n/(n-1) factor and the autocorrelation bias negligible next to the error
        per_chain_var = np.stack([b.var(0, ddof=1) for b in draws])
    finally:
        s.close()
    mg, sg = per_chain.mean(0), per_chain.std(0, ddof=1) / np.sqrt(K)
    vg_chain = per_chain_var
    vg, svg = vg_chain.mean(0), vg_chain.std(0, ddof=1) / np.sqrt(K)
    _, ob, _, _ = oracle.run(oracle.init_state(10), X, d["y"], oracle.gram(X), 5, 4000)
    ob = ob[500:]
    nb = 25
    bmeans = ob[: len(ob) // nb * nb].reshape(nb, -1, ob.shape[1]).mean(1)
    mo, so = bmeans.mean(0), bmeans.std(0, ddof=1) / np.sqrt(nb)
    zs = (mg - mo) / np.sqrt(sg ** 2 + so ** 2 + 1e-12)
    assert np.all(np.abs(zs) < 5.0), (zs, np.abs(mg - mo).max())
    # posterior variances: each GPU chain's sample variance (between-chain error)
    # against the oracle's (batch means of the squared deviations)
    sq = (ob - ob.mean(0)) ** 2
    vbm = sq[: len(sq) // nb * nb].reshape(nb, -1, sq.shape[1]).mean(1)
    vo, svo = vbm.mean(0), vbm.std(0, ddof=1) / np.sqrt(nb)
    zv = (vg - vo) / np.sqrt(svg ** 2 + svo ** 2 + 1e-24)
    assert np.all(np.abs(zv) < 5.0), ("variances", zv)


def test_batched_posterior_mean_error_vs_fp64_oracle():
    """The batched form's accuracy target: the posterior mean of beta that it
    estimates (32 chains, BF16 X, beta and z split into two BF16 parts on the
    tensor cores, FP32 accumulation) is within 1e-3 of the FP64 oracle's.

    Both sides run chains 0..7 (same seed and chain ids, so the same uniforms)
    for 250 sweeps from one warm state, on a problem shaped like the paper's
    synthetic one but small enough for the oracle: N = 2e4, p = 200, 5 nonzeros,
    X stored in BF16.  With common random numbers the two runs stay coupled
    (a 1e-6 relative perturbation of X moves the trajectory by ~1e-7 over 300
    sweeps), so the difference of the two estimates is the effect of the
    arithmetic on the posterior mean rather than Monte Carlo noise.  The
    oracle's estimate on the unrounded X (same y, same uniforms, four chains)
    shows the effect of storing X in BF16; it is printed, not bounded."""
    pkg = lib_pkg()
    N, p, nz, seed, n = 20000, 200, 5, 5, 250
    d = problem(N, p, nz, "bf16", seed=31)
    X = x_f64(d)
    G = oracle.gram(X)
    warm = oracle.init_state(p)
    for _ in range(400):
        warm = oracle.sweep_once(warm, X, d["y"], G, seed, chain=100)
    warm.k = 0
    s = pkg.HSProbit(d["X"], d["y"], seed=seed, num_chains=32, ring_size=n)
    try:
        for m in range(32):
            s.set_state(warm.beta, warm.lam_inv2, warm.nu_inv, warm.tau_inv2, warm.xi_inv, 0, chain=m)
        s.sweep(n)
        gpu = [s.draws(chain=m)["beta"] for m in range(32)]
    finally:
        s.close()
    chains = range(8)
    ora = [oracle.run(warm.copy(), X, d["y"], G, seed, n, chain=m)[1] for m in chains]
    m_gpu = np.mean([gpu[m].mean(0) for m in chains], axis=0)
    m_ora = np.mean([o.mean(0) for o in ora], axis=0)
    err = np.abs(m_gpu - m_ora).max()
    # Monte Carlo scale of the estimate, for context: between-chain standard error of the 32 GPU chains
    se = (np.stack([g.mean(0) for g in gpu]).std(0, ddof=1) / np.sqrt(32)).max()
    X_unrounded = problem(N, p, nz, "f64", seed=31)["X"]
    Gu = oracle.gram(X_unrounded)
    m_unr = np.mean([oracle.run(warm.copy(), X_unrounded, d["y"], Gu, seed, n, chain=m)[1].mean(0)
                     for m in range(4)], axis=0)
    m_ora4 = np.mean([o.mean(0) for o in ora[:4]], axis=0)
    m_gpu4 = np.mean([gpu[m].mean(0) for m in range(4)], axis=0)
    print(f"posterior-mean error of the batched BF16 form: max |dbeta| = {err:.3e} against the FP64 oracle on "
          f"the stored X (8 coupled chains x {n} sweeps); {np.abs(m_gpu4 - m_unr).max():.3e} against the oracle on "
          f"the unrounded X, of which BF16 storage of X alone accounts for {np.abs(m_ora4 - m_unr).max():.3e}; "
          f"Monte Carlo standard error of the 32-chain estimate {se:.3e}")
    assert err <= 1e-3, err


@pytest.mark.parametrize("dt,N,p,K", [("bf16", 3001, 200, 4),    # 7 tiles: two block columns, the last ragged
                                      ("bf16", 2000, 520, 2),    # 17 tiles: five block columns
                                      ("bf16", 4099, 1000, 8),
                                      ("f32", 3001, 300, 1)])    # one chain
def test_tensor_core_trailing_updates_match_pair_arithmetic(pkg, dt, N, p, K):
    """The block-column schedule (HS_SCHED_TENSOR: tile tasks in FP32-pair
    arithmetic inside each 128-column block, the rank-128 updates to its right
    as exact products of BF16 digits on the tensor cores) against the
    single-launch schedule that applies every tile update in FP32-pair
    arithmetic; both factor only, beta by substitution, from the same state
    per chain.  The factor's updates carry about 48 bits either way, so beta
    agrees to 1e-11 relative; lambda^{-2} and tau^{-2} (drawn before the
    factorization) agree exactly."""
    d = problem(N, p, 5, dt, seed=p)
    states = [random_state(p, k=3, seed=40 + m) for m in range(K)]
    out = {}
    for sched in (pkg.SCHED_SINGLE, pkg.SCHED_TENSOR):
        s = pkg.HSProbit(d["X"], d["y"], seed=7, num_chains=K, chol_sched=sched, beta_solve=pkg.BETA_SUBST)
        try:
            for m, st in enumerate(states):
                s.set_state(st.beta, st.lam_inv2, st.nu_inv, st.tau_inv2, st.xi_inv, st.k, chain=m)
            s.sweep(1)
            out[sched] = [s.get_state(chain=m) for m in range(K)]
        finally:
            s.close()
    for m in range(K):
        a, b = out[pkg.SCHED_SINGLE][m], out[pkg.SCHED_TENSOR][m]
        assert np.array_equal(a["lambda_inv2"], b["lambda_inv2"]) and a["tau_inv2"] == b["tau_inv2"]
        db = np.linalg.norm(a["beta"] - b["beta"]) / np.linalg.norm(a["beta"])
        assert db <= 1e-11, (m, db)


@pytest.mark.parametrize("K", [1, 4])
def test_tensor_core_trailing_updates_after_a_large_jump_of_tau(pkg, K):
    """The digit planes of the tensor-core trailing updates represent factor
    entries in [-1, 1] exactly; a unit diagonal of the equilibrated precision
    matrix (S formed from the new tau^{-2} on that schedule) bounds every
    entry by its row norm, 1, for any design.  From a state whose tau^{-2} is
    far below its conditional (tau^{-2} = 1e-4, small beta, large
    lambda^{-2}) the new tau^{-2} is over 1e3 times the current one and
    tau lambda^{-2} dominates the diagonal; the single-launch schedule (whose
    pair arithmetic needs only range, so it equilibrates with the current
    tau^{-2}) and the block-column schedule must still agree to the pair
    arithmetic's precision."""
    N, p = 2000, 520
    d = problem(N, p, 5, "bf16", seed=p + 1)
    r = np.random.default_rng(5)
    states = [oracle.State(r.normal(0, 0.01, p), np.full(p, 1e3) * r.uniform(0.5, 2.0, p), r.exponential(size=p) + 0.05,
                           1e-4, 1.0, 3) for _ in range(K)]
    out = {}
    for sched in (pkg.SCHED_SINGLE, pkg.SCHED_TENSOR):
        s = pkg.HSProbit(d["X"], d["y"], seed=9, num_chains=K, chol_sched=sched, beta_solve=pkg.BETA_SUBST)
        try:
            for m, st in enumerate(states):
                s.set_state(st.beta, st.lam_inv2, st.nu_inv, st.tau_inv2, st.xi_inv, st.k, chain=m)
            s.sweep(1)
            out[sched] = [s.get_state(chain=m) for m in range(K)]
        finally:
            s.close()
    for m in range(K):
        a, b = out[pkg.SCHED_SINGLE][m], out[pkg.SCHED_TENSOR][m]
        assert a["tau_inv2"] == b["tau_inv2"] and a["tau_inv2"] > 1e3 * states[m].tau_inv2
        db = np.linalg.norm(a["beta"] - b["beta"]) / np.linalg.norm(a["beta"])
        assert db <= 1e-11, (m, db)


def test_eight_chains_on_fp8_correlated_design_at_p_4000(pkg):
    """The large correlated workload's shape with its K = 8 chains at a size
    the oracle runs in seconds: FP8 e4m3 X with column scales, AR(1) rows,
    p = 4000, 20 nonzeros U[0.5, 2].  The X-stream runs on the tensor cores
    as two kernels, the FP8 codes converted to BF16 in shared memory (exact)
    and the column scales folded into B^T and X^T Z; every chain must stay
    within the batched form's BF16 bound of the oracle's transition."""
    N, p, K = 3000, 4000, 8
    d = problem(N, p, 20, "fp8", seed=5, mag=(0.5, 2.0), design="ar1")
    X = x_f64(d)
    G = oracle.gram(X)
    states = [random_state(p, k=3, seed=600 + m, scale=0.05) for m in range(K)]
    s = pkg.HSProbit(d["X"], d["y"], seed=29, scales=d["scales"], debug=True, num_chains=K)
    try:
        for m, st in enumerate(states):
            s.set_state(st.beta, st.lam_inv2, st.nu_inv, st.tau_inv2, st.xi_inv, st.k, chain=m)
        s.sweep(1)
        got = []
        for m in range(K):
            g = s.get_state(chain=m)
            g["z"] = s.debug_z(chain=m)
            g["xtz"] = s.debug_xtz(chain=m)
            got.append(g)
    finally:
        s.close()
    for m, st in enumerate(states):
        ref = oracle.sweep_once(st.copy(), X, d["y"], G, 29, chain=m, keep=True)
        assert_batched_close(got[m], ref, X, st.beta)


@pytest.mark.parametrize("N,p,K", [(3001, 300, 4), (2000, 1000, 24)])
def test_fp8_chains_on_the_tensor_cores_match_oracle(pkg, N, p, K):
    """FP8 X with column scales and K chains at sizes the fused kernel would
    take for BF16: the split form at 16 and 32 chain columns."""
    d = problem(N, p, 5, "fp8", seed=K)
    X = x_f64(d)
    G = oracle.gram(X)
    states = [random_state(p, k=4, seed=700 + m, scale=0.2) for m in range(K)]
    s = pkg.HSProbit(d["X"], d["y"], seed=31, scales=d["scales"], debug=True, num_chains=K)
    try:
        assert s.launch_shape()["xk_chains"] == (16 if K <= 16 else 32)
        for m, st in enumerate(states):
            s.set_state(st.beta, st.lam_inv2, st.nu_inv, st.tau_inv2, st.xi_inv, st.k, chain=m)
        s.sweep(1)
        for m, st in enumerate(states):
            g = s.get_state(chain=m)
            g["z"] = s.debug_z(chain=m)
            g["xtz"] = s.debug_xtz(chain=m)
            ref = oracle.sweep_once(st.copy(), X, d["y"], G, 31, chain=m, keep=True)
            assert_batched_close(g, ref, X, st.beta)
    finally:
        s.close()


def _posterior_means(pkg, X_store, y, scales, warm, seed, n, K, **kw):
    s = pkg.HSProbit(X_store, y, seed=seed, scales=scales, num_chains=K, ring_size=n, **kw)
    try:
        for m in range(K):
            s.set_state(warm["beta"], warm["lambda_inv2"], warm["nu_inv"], warm["tau_inv2"], warm["xi_inv"], 0,
                        chain=m)
        s.sweep(n)
        return [s.draws(chain=m)["beta"] for m in range(K)]
    finally:
        s.close()


def test_fp8_chains_posterior_mean_error_vs_fp64_oracle():
    """The large correlated workload's form (FP8 X with column scales, AR(1)
    rows, K = 8 chains on the two-pass tensor-core X-stream) at a size the
    oracle runs in seconds (N = 2e4, p = 300): coupled chains (same seed and
    chain ids) from one warm state, 250 sweeps; the posterior mean of beta is
    within 1e-3 of the FP64 oracle's on the same stored X."""
    pkg = lib_pkg()
    N, p, seed, n, K = 20000, 300, 9, 250, 8
    d = problem(N, p, 5, "fp8", seed=41, mag=(0.5, 2.0), design="ar1")
    X = x_f64(d)
    G = oracle.gram(X)
    w = oracle.init_state(p)
    for _ in range(400):
        w = oracle.sweep_once(w, X, d["y"], G, seed, chain=100)
    warm = {"beta": w.beta, "lambda_inv2": w.lam_inv2, "nu_inv": w.nu_inv, "tau_inv2": w.tau_inv2,
            "xi_inv": w.xi_inv}
    w.k = 0
    gpu = _posterior_means(pkg, d["X"], d["y"], d["scales"], warm, seed, n, K)
    ora = [oracle.run(w.copy(), X, d["y"], G, seed, n, chain=m)[1] for m in range(K)]
    m_gpu = np.mean([g.mean(0) for g in gpu], axis=0)
    m_ora = np.mean([o.mean(0) for o in ora], axis=0)
    err = np.abs(m_gpu - m_ora).max()
    se = (np.stack([g.mean(0) for g in gpu]).std(0, ddof=1) / np.sqrt(K)).max()
    print(f"posterior-mean error of {K} FP8 chains: max |dbeta| = {err:.3e} against the FP64 oracle on the stored "
          f"X ({n} coupled sweeps); Monte Carlo standard error of the estimate {se:.3e}")
    assert err <= 1e-3, err


def test_fp8_chains_posterior_mean_error_vs_fp64_x_at_p_4000():
    """At the large workload's p = 4000 (N = 2e5, where the oracle is too slow
    for long runs) the reference is the library's FP64-X path, itself held to
    the oracle's transition at 1e-10: the same stored values as FP64 X (one
    FP64 X-stream pass per chain), the same seed, chain ids and warm state.
    The posterior means of the K = 8 FP8 chains over 150 coupled sweeps stay
    within 1e-3 of it."""
    pkg = lib_pkg()
    N, p, seed, n, K = 200_000, 4000, 3, 150, 8
    d = problem(N, p, 20, "fp8", seed=5, mag=(0.5, 2.0), design="ar1")
    X = x_f64(d)
    ref0 = pkg.HSProbit(X, d["y"], seed=seed, chain=100)
    try:
        ref0.sweep(100)
        warm = ref0.get_state()
    finally:
        ref0.close()
    fp64 = _posterior_means(pkg, X, d["y"], None, warm, seed, n, K)
    fp8 = _posterior_means(pkg, d["X"], d["y"], d["scales"], warm, seed, n, K)
    m64 = np.mean([g.mean(0) for g in fp64], axis=0)
    m8 = np.mean([g.mean(0) for g in fp8], axis=0)
    err = np.abs(m8 - m64).max()
    se = (np.stack([g.mean(0) for g in fp64]).std(0, ddof=1) / np.sqrt(K)).max()
    print(f"posterior-mean error of {K} FP8 chains at N = {N}, p = {p}: max |dbeta| = {err:.3e} against the "
          f"FP64-X path ({n} coupled sweeps); Monte Carlo standard error {se:.3e}")
    assert err <= 1e-3, err
