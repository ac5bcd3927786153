"""The rest of the C boundary: an adopted (zero-copy) device X, the
update-mask test hook, draws downloaded on a side stream, and the FP32-pair
factorization on an ill-conditioned design.

The update-mask check is pinned to the closed form, not to the oracle: with
lambda and tau held fixed, beta | z is N(Sigma X^T z, Sigma) with
Sigma = (X^T X + tau^{-2} Lambda^{-2})^{-1} (Sect. 5, beta update), so
L^T (beta_k - Sigma X^T z_k), A = L L^T, must be independent standard
normals over the sweeps k.
"""
import numpy as np
import pytest

import hs_synth
import oracle
from tests.gpu_common import assert_transition_close, gpu_transition, lib_pkg, problem, random_state, x_f64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return lib_pkg()


def test_adopted_device_x_gives_the_copied_transition(pkg):
    import torch
    d = problem(5003, 64, 5, "f32", seed=2)
    st = random_state(64, k=4, seed=1)
    outs = []
    for adopt in (False, True):
        X = torch.from_numpy(d["X"]).cuda()
        y = torch.from_numpy(d["y"]).cuda()
        s = pkg.HSProbit(X, y, seed=9, debug=True, adopt=adopt)
        try:
            if adopt:
                del X  # the handle keeps the adopted tensor alive
            s.set_state(st.beta, st.lam_inv2, st.nu_inv, st.tau_inv2, st.xi_inv, st.k)
            s.sweep(2)
            g = s.get_state()
            g["z"] = s.debug_z()
            outs.append(g)
        finally:
            s.close()
    for key in ("beta", "lambda_inv2", "nu_inv", "z"):
        assert np.array_equal(outs[0][key], outs[1][key]), key


def test_adopt_rejects_rows_or_bases_off_16_bytes(pkg):
    import torch
    d = problem(300, 63, 3, "f32", seed=2)  # 63 * 4 = 252-byte rows
    with pytest.raises(pkg.HSProbitError) as ei:
        pkg.HSProbit(torch.from_numpy(d["X"]).cuda(), torch.from_numpy(d["y"]).cuda(), adopt=True)
    assert ei.value.status == -1
    flat = torch.zeros(300 * 64 + 1, device="cuda")
    X = flat[1:].view(300, 64)  # base 4 bytes past a 16-byte boundary
    with pytest.raises(pkg.HSProbitError) as ei:
        pkg.HSProbit(X, torch.from_numpy(d["y"]).cuda(), adopt=True)
    assert ei.value.status == -1


def test_frozen_lambda_tau_one_sweep_matches_oracle_beta_draw(pkg):
    """Held lambda and tau: beta is the oracle's beta draw from the same
    lambda, tau and X^T z (same counters), nu and xi still move."""
    d = problem(3001, 40, 4, "f64", seed=6)
    X = x_f64(d)
    G = oracle.gram(X)
    st = random_state(40, k=11, seed=3)
    s = pkg.HSProbit(d["X"], d["y"], seed=21, debug=True, update_mask=pkg.UPD_NU | pkg.UPD_XI)
    try:
        s.set_state(st.beta, st.lam_inv2, st.nu_inv, st.tau_inv2, st.xi_inv, st.k)
        s.sweep(1)
        g = s.get_state()
        xtz = s.debug_xtz()
    finally:
        s.close()
    assert np.array_equal(g["lambda_inv2"], st.lam_inv2) and g["tau_inv2"] == st.tau_inv2
    assert not np.array_equal(g["nu_inv"], st.nu_inv) and g["xi_inv"] != st.xi_inv
    beta, _, _ = oracle.sweep.draw_beta(G, st.lam_inv2, st.tau_inv2, xtz, 21, st.k + 1, 0, 0)
    assert np.linalg.norm(g["beta"] - beta) <= 1e-10 * np.linalg.norm(beta)


def test_frozen_lambda_tau_beta_conditional_is_the_closed_form_gaussian(pkg):
    N, p, M = 400, 6, 1500
    d = problem(N, p, 2, "f64", seed=12)
    X = x_f64(d)
    st = random_state(p, k=0, seed=5, scale=0.3)
    s = pkg.HSProbit(d["X"], d["y"], seed=33, debug=True, update_mask=pkg.UPD_NU | pkg.UPD_XI)
    A = X.T @ X + st.tau_inv2 * np.diag(st.lam_inv2)
    L = np.linalg.cholesky(A)
    w = np.empty((M, p))
    try:
        s.set_state(st.beta, st.lam_inv2, st.nu_inv, st.tau_inv2, st.xi_inv, st.k)
        for k in range(M):
            s.sweep(1)
            z = s.debug_z()
            g = s.get_state()
            mu = np.linalg.solve(A, X.T @ z)
            w[k] = L.T @ (g["beta"] - mu)
        assert np.array_equal(g["lambda_inv2"], st.lam_inv2) and g["tau_inv2"] == st.tau_inv2
    finally:
        s.close()
    flat = w.ravel()
    n = flat.size
    assert abs(flat.mean()) < 4.0 / np.sqrt(n)
    assert abs(flat.var() - 1.0) < 4.0 * np.sqrt(2.0 / n)
    C = np.corrcoef(w.T)
    assert np.abs(C - np.eye(p)).max() < 4.0 / np.sqrt(M)
    from scipy import stats
    assert stats.kstest(flat, "norm").pvalue > 1e-4


@pytest.mark.parametrize("ring", [64, 8])
def test_draws_downloaded_on_a_side_stream_equal_the_synchronous_copy(pkg, ring):
    """Eight draws copied asynchronously while the next eight sweeps run; with
    an 8-slot ring those sweeps must first wait for the copy."""
    import torch
    d = problem(20000, 100, 5, "f32", seed=4)
    a = pkg.HSProbit(d["X"], d["y"], seed=8, ring_size=ring)
    b = pkg.HSProbit(d["X"], d["y"], seed=8, ring_size=ring)
    try:
        out = {"beta": torch.empty((8, 100), dtype=torch.float64).pin_memory().numpy(),
               "lambda_inv2": torch.empty((8, 100), dtype=torch.float64).pin_memory().numpy(),
               "tau_inv2": torch.empty(8, dtype=torch.float64).pin_memory().numpy()}
        a.sweep(8)
        assert a.draws_async(out) == 8
        a.sweep(8)  # runs while the copy is in flight (or after it, for the 8-slot ring)
        a.draws_wait()
        b.sweep(8)
        ref = b.draws()
        for k in out:
            assert np.array_equal(out[k], ref[k]), k
        b.sweep(8)
        assert np.array_equal(a.draws()["beta"], b.draws()["beta"])
    finally:
        a.close()
        b.close()


def test_pair_factorization_on_an_ill_conditioned_design(pkg):
    """Rows N(0, Toeplitz 0.99^|i-j|): the Gram matrix's condition number is
    about 4e4 times that of the iid design; the FP32-pair factorization
    (2^-48 per operation) still gives the FP64 oracle's transition to 1e-10."""
    N, p = 20000, 200
    d = hs_synth.make_problem(N, p, 5, "f64", seed=3, design="ar1", rho=0.99)
    X = x_f64(d)
    G = oracle.gram(X)
    assert np.linalg.cond(G) > 1e4
    st = random_state(p, k=2, seed=9, scale=0.2)
    got = gpu_transition(pkg, d, st, 17)
    ref = oracle.sweep_once(st.copy(), X, d["y"], G, 17, keep=True)
    assert_transition_close(got, ref, 1e-10)


@pytest.mark.parametrize("dt,p,K", [("bf16", 304, 4), ("bf16", 2000, 4), ("fp8", 512, 3)])  # rows of 16-byte slices
def test_adopted_x_with_chains_on_the_tensor_cores_gives_the_copied_transition(pkg, dt, p, K):
    """K chains on an adopted device X (the tensor-core X-streams read the
    caller's buffer through their tensor maps): the same transition bit for
    bit as on the library's copy (fused form at p = 304, two-pass form at
    p = 2000 and for FP8 with column scales)."""
    import torch
    d = problem(3001, p, 5, dt, seed=p)
    sts = [random_state(p, k=3, seed=40 + m) for m in range(K)]
    outs = []
    for adopt in (False, True):
        X = torch.from_numpy(d["X"]).cuda()
        y = torch.from_numpy(d["y"]).cuda()
        sc = torch.from_numpy(d["scales"]).cuda() if d["scales"] is not None else None
        s = pkg.HSProbit(X, y, seed=12, debug=True, num_chains=K, adopt=adopt, scales=sc)
        try:
            for m, st in enumerate(sts):
                s.set_state(st.beta, st.lam_inv2, st.nu_inv, st.tau_inv2, st.xi_inv, st.k, chain=m)
            s.sweep(2)
            outs.append([(s.get_state(chain=m)["beta"], s.debug_z(chain=m)) for m in range(K)])
        finally:
            s.close()
    for (b0, z0), (b1, z1) in zip(*outs):
        assert np.array_equal(z0, z1) and np.array_equal(b0, b1)
