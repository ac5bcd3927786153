"""GPU runtime behaviour through the C ABI: graph replay, determinism,
checkpoint/resume, the draw ring, device-side error reporting and the
bounded-wait failure path."""
import numpy as np
import pytest

import oracle
from tests.gpu_common import lib_pkg, problem, random_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return lib_pkg()


@pytest.fixture(scope="module")
def data():
    return problem(6000, 50, 4, "f32", seed=4)


def _state(s):
    st = s.get_state()
    return np.concatenate([st["beta"], st["lambda_inv2"], st["nu_inv"], [st["tau_inv2"], st["xi_inv"], st["k"]]])


def test_graph_replay_equals_eager(pkg, data):
    a = pkg.HSProbit(data["X"], data["y"], seed=3, use_graph=False)
    b = pkg.HSProbit(data["X"], data["y"], seed=3, use_graph=True)
    a.sweep(7)
    b.sweep(7)
    assert np.array_equal(_state(a), _state(b))
    a.close()
    b.close()


@pytest.mark.parametrize("N,p", [(300, 1), (500, 33), (900, 64), (2000, 257), (3001, 600), (2500, 1100),
                                 (3000, 2500)])
@pytest.mark.parametrize("graph", [False, True], ids=["eager", "graph"])
def test_single_launch_factorization_equals_column_launches(pkg, N, p, graph):
    """The FP32-pair factorization scheduled by tile readiness in one
    cooperative launch performs the same operations on every tile as the
    one-launch-per-block-column schedule, so whole chains agree bit for bit."""
    d = problem(N, p, min(4, p), "f32", seed=p)
    a = pkg.HSProbit(d["X"], d["y"], seed=5, use_graph=graph, chol_sched=pkg.SCHED_COLUMNS)
    b = pkg.HSProbit(d["X"], d["y"], seed=5, use_graph=graph, chol_sched=pkg.SCHED_SINGLE,
                     beta_solve=pkg.BETA_INVERSE)  # the same beta form as the column schedule
    assert a.launches_per_sweep() - b.launches_per_sweep() == (p + 31) // 32 - 1
    a.sweep(4)
    b.sweep(4)
    assert np.array_equal(_state(a), _state(b))
    a.close()
    b.close()


def test_deterministic_and_seed_sensitive(pkg, data):
    a = pkg.HSProbit(data["X"], data["y"], seed=3)
    b = pkg.HSProbit(data["X"], data["y"], seed=3)
    c = pkg.HSProbit(data["X"], data["y"], seed=4)
    for s in (a, b, c):
        s.sweep(5)
    assert np.array_equal(_state(a), _state(b))
    assert not np.array_equal(_state(a), _state(c))


def test_checkpoint_resume_bit_exact(pkg, data):
    a = pkg.HSProbit(data["X"], data["y"], seed=9)
    a.sweep(20)
    b = pkg.HSProbit(data["X"], data["y"], seed=9)
    b.sweep(10)
    st = b.get_state()
    b.close()
    c = pkg.HSProbit(data["X"], data["y"], seed=9)
    c.set_state(st["beta"], st["lambda_inv2"], st["nu_inv"], st["tau_inv2"], st["xi_inv"], st["k"])
    c.sweep(10)
    assert np.array_equal(_state(a), _state(c))


def test_draw_ring_thinning(pkg, data):
    s = pkg.HSProbit(data["X"], data["y"], seed=5, thin=2, ring_size=4)
    ref = pkg.HSProbit(data["X"], data["y"], seed=5)
    states = []
    for _ in range(11):
        ref.sweep(1)
        states.append(ref.get_state())
    s.sweep(11)
    d = s.draws()
    # sweeps 2,4,6,8,10 recorded; ring of 4 keeps 4,6,8,10
    assert d["beta"].shape == (4, 50)
    for i, k in enumerate((4, 6, 8, 10)):
        assert np.array_equal(d["beta"][i], states[k - 1]["beta"])
        assert np.array_equal(d["lambda_inv2"][i], states[k - 1]["lambda_inv2"])
        assert d["tau_inv2"][i] == states[k - 1]["tau_inv2"]
    assert s.draws()["beta"].shape == (0, 50)
    s.sweep(2)
    d2 = s.draws()
    assert d2["beta"].shape == (1, 50) and np.array_equal(d2["beta"][0], _ref_after(ref, 12)["beta"])


def _ref_after(ref, k):
    while ref.get_state()["k"] < k:
        ref.sweep(1)
    return ref.get_state()


def test_not_positive_definite_is_reported_and_state_kept(pkg, data):
    s = pkg.HSProbit(data["X"], data["y"], seed=1)
    s.sweep(2)
    before = _state(s)
    p = 50
    # A negative nu^{-1} makes the Exp rate of lambda^{-2} negative, so
    # lambda^{-2} ~ -1e12 and A = G + tau^{-2} Lambda^{-2} is indefinite.
    s.set_state(np.zeros(p), np.ones(p), np.full(p, -1e-12), 1.0, 1.0, 2)
    st = s.sweep_status(1)
    assert st == -4  # HS_ENOTPD
    assert s.sweep_status(1) == -7  # HS_ESTATE until set_state
    after = s.get_state()
    assert after["k"] == 2 and np.all(after["nu_inv"] == -1e-12)
    s.set_state(before[:p], before[p:2 * p], before[2 * p:3 * p], before[-3], before[-2], int(before[-1]))
    s.sweep(1)
    assert s.get_state()["k"] == 3


def test_non_finite_is_reported(pkg, data):
    s = pkg.HSProbit(data["X"], data["y"], seed=1)
    p = 50
    b = np.zeros(p)
    b[3] = np.nan
    s.set_state(b, np.ones(p), np.ones(p), 1.0, 1.0, 0)
    assert s.sweep_status(1) == -5  # HS_ENONFINITE
    assert s.get_state()["k"] == 0


def test_bounded_wait_times_out_and_context_survives(pkg, data):
    s = pkg.HSProbit(data["X"], data["y"], seed=1)
    assert s.debug_wait_timeout(20000) == -6  # HS_ETIMEOUT
    s.sweep(2)
    assert s.get_state()["k"] == 2


def test_device_inputs_and_bad_device_y(pkg, data):
    torch = pytest.importorskip("torch")
    Xd = torch.from_numpy(data["X"]).cuda()
    yd = torch.from_numpy(data["y"]).cuda()
    a = pkg.HSProbit(Xd, yd, seed=8)
    b = pkg.HSProbit(data["X"], data["y"], seed=8)
    a.sweep(3)
    b.sweep(3)
    assert np.array_equal(_state(a), _state(b))
    ybad = yd.clone()
    ybad[17] = 3
    with pytest.raises(pkg.HSProbitError) as ei:
        pkg.HSProbit(Xd, ybad, seed=8)
    assert ei.value.status == -1


def _batch_means(v, nb=25):
    """Mean over the draws (rows of v) and its batch-means standard error."""
    m = v[: len(v) // nb * nb].reshape(nb, -1, v.shape[1]).mean(1)
    return m.mean(0), m.std(0, ddof=1) / np.sqrt(nb)


def _moment_zscores(a, b):
    """z-scores of the differences of the posterior means and of the posterior
    variances of two chains' draws (rows), with batch-means errors; the
    variance of each chain is the batch mean of (v - mean of v)^2."""
    ma, sa = _batch_means(a)
    mb, sb = _batch_means(b)
    va, sva = _batch_means((a - a.mean(0)) ** 2)
    vb, svb = _batch_means((b - b.mean(0)) ** 2)
    zm = (ma - mb) / np.sqrt(sa ** 2 + sb ** 2 + 1e-12)
    zv = (va - vb) / np.sqrt(sva ** 2 + svb ** 2 + 1e-24)
    return zm, zv


def test_long_run_moments_match_oracle_within_mc_error(pkg):
    """Different seeds: posterior means and variances of beta (and of
    log lambda^{-2} and log tau^{-2}) from the GPU chain and the oracle chain
    agree within Monte Carlo error (batch means, 5 standard errors)."""
    d = problem(2000, 10, 3, "f64", seed=21)
    n, burn = 3000, 500
    s = pkg.HSProbit(d["X"], d["y"], seed=1, ring_size=n)
    s.sweep(n)
    g = s.draws()
    _, ob, ol, ot = oracle.run(oracle.init_state(10), d["X"], d["y"], oracle.gram(d["X"]), 2, n)
    gv = np.column_stack([g["beta"], np.log(g["lambda_inv2"]), np.log(g["tau_inv2"])])[burn:]
    ov = np.column_stack([ob, np.log(ol), np.log(ot)])[burn:]
    zm, zv = _moment_zscores(gv, ov)
    assert np.all(np.abs(zm) < 5.0), ("means", zm)
    assert np.all(np.abs(zv) < 5.0), ("variances", zv)


def test_profiling_in_graph_and_eager_modes(pkg, data):
    """Per-kernel CUDA events work with and without graph replay and do not
    change the trajectory."""
    out = {}
    for graph in (False, True):
        s = pkg.HSProbit(data["X"], data["y"], seed=6, use_graph=graph)
        s.set_profiling(True)
        s.sweep(4)
        for g in ("xstream", "reduce", "shrink", "cholesky", "tail"):
            ms, n = s.kernel_time(g)
            assert n == 4 and ms > 0.0, (graph, g, ms, n)
        out[graph] = _state(s)
        s.close()
    assert np.array_equal(out[False], out[True])
