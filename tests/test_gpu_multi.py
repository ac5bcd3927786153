"""Many problems in one launch (Sect. 4: the sweep serves any exchangeable
data-augmented model; here several independent Horseshoe probit problems of
uneven N and p) and the launch shapes the batch tuner chooses between.

Problem m of a batch is the handle that hs_probit_init_ex would make with
problem id (problem + m), so each of its chains must reproduce the oracle's
transition for that (chain, problem) counter pair from the same state, at
the tolerance of its X type (the BF16 bound of the batched form; 1e-4 for
F32).  Launch shapes spread the same work differently, so every shape is
held to the same oracle bound.
"""
import numpy as np
import pytest

import oracle
from tests.gpu_common import assert_transition_close, lib_pkg, problem, random_state, x_f64
from tests.test_gpu_batched import assert_batched_close

pytestmark = pytest.mark.gpu

# uneven sizes: small and large N, p from 1 to 2000 (the 1% nonzero recipe of the uneven batch)
UNEVEN = [(3001, 50), (20000, 700), (1000, 1), (6007, 1900), (12000, 300)]


@pytest.fixture(scope="module")
def pkg():
    return lib_pkg()


def _make(sizes, dt, seed0):
    return [problem(N, p, max(1, round(0.01 * p)), dt, seed=seed0 + m) for m, (N, p) in enumerate(sizes)]


def _batch_transitions(b, ds, K, seed_state):
    states = []
    for m, d in enumerate(ds):
        h = b.problem(m)
        sts = [random_state(d["X"].shape[1], k=5, seed=seed_state + 50 * m + c) for c in range(K)]
        for c, st in enumerate(sts):
            h.set_state(st.beta, st.lam_inv2, st.nu_inv, st.tau_inv2, st.xi_inv, st.k, chain=c)
        states.append(sts)
    b.sweep(1)
    got = []
    for m in range(len(ds)):
        h = b.problem(m)
        outs = []
        for c in range(K):
            g = h.get_state(chain=c)
            g["z"] = h.debug_z(chain=c)
            g["xtz"] = h.debug_xtz(chain=c)
            outs.append(g)
        got.append(outs)
    return states, got


def test_uneven_batch_matches_oracle_per_problem_and_chain(pkg):
    K, seed, prob0, chain0 = 4, 19, 3, 5
    ds = _make(UNEVEN, "bf16", 40)
    b = pkg.HSProbitBatch([(d["X"], d["y"]) for d in ds], seed=seed, num_chains=K, debug=True, problem=prob0,
                          chain=chain0)
    try:
        assert len(b) == len(ds)
        states, got = _batch_transitions(b, ds, K, 700)
    finally:
        b.close()
    for m, d in enumerate(ds):
        X = x_f64(d)
        G = oracle.gram(X)
        for c in range(K):
            ref = oracle.sweep_once(states[m][c].copy(), X, d["y"], G, seed, chain=chain0 + c,
                                    problem=prob0 + m, keep=True)
            assert_batched_close(got[m][c], ref, X, states[m][c].beta)


def test_one_chain_f32_batch_matches_oracle(pkg):
    """K = 1 per problem: each factorization is the single-launch schedule as
    an ordinary (not cooperative) launch sharing the GPU with the others."""
    sizes = [(4000, 100), (2001, 1000), (3000, 2100), (500, 3)]
    ds = _make(sizes, "f32", 90)
    b = pkg.HSProbitBatch([(d["X"], d["y"]) for d in ds], seed=3, debug=True)
    try:
        states, got = _batch_transitions(b, ds, 1, 900)
    finally:
        b.close()
    for m, d in enumerate(ds):
        X = x_f64(d)
        ref = oracle.sweep_once(states[m][0].copy(), X, d["y"], oracle.gram(X), 3, chain=0, problem=m, keep=True)
        assert_transition_close(got[m][0], ref, 1e-4)


def test_batch_member_shape_change_and_free_are_safe(pkg):
    """A launch-shape change on one problem makes the batch recapture its
    graph and keep sweeping; hs_probit_free on a problem's handle is ignored
    (the batch owns it)."""
    ds = _make([(3000, 200), (2500, 90)], "bf16", 3)
    outs = []
    for change_after in (True, False):
        b = pkg.HSProbitBatch([(d["X"], d["y"]) for d in ds], seed=2, num_chains=2)
        try:
            h = b.problem(0)
            if not change_after:
                h.set_launch_shape(xstream_ctas=5)
            b.sweep(2)
            if change_after:
                h.set_launch_shape(xstream_ctas=5)
            b.sweep(2)
            pkg.load_library().hs_probit_free(h._h)  # ignored: the handle still works
            outs.append(h.get_state(chain=1))
            assert outs[-1]["k"] == 4
        finally:
            b.close()
    assert np.all(np.isfinite(outs[0]["beta"])) and np.all(np.isfinite(outs[1]["beta"]))


def test_fp8_batch_with_column_scales_matches_oracle(pkg):
    """Uneven FP8 problems, each with its own column scales (hs_problem.x_scales),
    two chains each: the two-pass tensor-core X-stream per problem."""
    sizes = [(3001, 130), (5000, 700), (700, 16)]
    ds = _make(sizes, "fp8", 60)
    b = pkg.HSProbitBatch([(d["X"], d["y"], d["scales"]) for d in ds], seed=7, num_chains=2, debug=True)
    try:
        states, got = _batch_transitions(b, ds, 2, 1100)
    finally:
        b.close()
    for m, d in enumerate(ds):
        X = x_f64(d)
        G = oracle.gram(X)
        for c in range(2):
            ref = oracle.sweep_once(states[m][c].copy(), X, d["y"], G, 7, chain=c, problem=m, keep=True)
            assert_batched_close(got[m][c], ref, X, states[m][c].beta)


def test_batch_runs_many_sweeps_and_tuner_restores_state(pkg):
    ds = _make(UNEVEN, "bf16", 7)
    b = pkg.HSProbitBatch([(d["X"], d["y"]) for d in ds], seed=5, num_chains=4, ring_size=16)
    try:
        b.sweep(4)
        before = [[b.problem(m).get_state(chain=c) for c in range(4)] for m in range(len(ds))]
        best = b.tune(2)
        trials = b.tune_trials()
        assert best > 0 and len(trials) >= 4
        assert best == pytest.approx(min(t["ms_per_sweep"] for t in trials))
        for m in range(len(ds)):
            for c in range(4):
                after = b.problem(m).get_state(chain=c)
                for key in ("beta", "lambda_inv2", "nu_inv"):
                    assert np.array_equal(before[m][c][key], after[key])
                assert before[m][c]["tau_inv2"] == after["tau_inv2"] and before[m][c]["k"] == after["k"] == 4
        b.sweep(3)
        for m in range(len(ds)):
            h = b.problem(m)
            assert h.get_state(chain=0)["k"] == 7
            dr = h.draws(chain=1)
            assert np.array_equal(dr["beta"][-1], h.get_state(chain=1)["beta"])
            assert np.all(np.isfinite(dr["beta"]))
    finally:
        b.close()


@pytest.mark.parametrize("kc,stages,per_sm", [(16, 4, 1), (16, 6, 1), (16, 8, 1), (16, 4, 2), (32, 4, 1),
                                              (32, 6, 1), (32, 8, 1)])
def test_every_tensor_core_xstream_shape_matches_oracle(pkg, kc, stages, per_sm):
    N, p, K = 4099, 700, 6
    d = problem(N, p, 5, "bf16", seed=kc + stages)
    X = x_f64(d)
    G = oracle.gram(X)
    states = [random_state(p, k=8, seed=500 + m) for m in range(K)]
    s = pkg.HSProbit(d["X"], d["y"], seed=23, debug=True, num_chains=K)
    try:
        s.set_launch_shape(xk_chains=kc, xk_stages=stages, xk_ctas_per_sm=per_sm, xstream_ctas=17)  # of 33 tiles
        sh = s.launch_shape()
        assert (sh["xk_chains"], sh["xk_stages"], sh["xk_ctas_per_sm"], sh["xstream_ctas"]) == (kc, stages, per_sm, 17)
        for m, st in enumerate(states):
            s.set_state(st.beta, st.lam_inv2, st.nu_inv, st.tau_inv2, st.xi_inv, st.k, chain=m)
        s.sweep(1)
        for m, st in enumerate(states):
            g = s.get_state(chain=m)
            g["z"] = s.debug_z(chain=m)
            g["xtz"] = s.debug_xtz(chain=m)
            ref = oracle.sweep_once(st.copy(), X, d["y"], G, 23, chain=m, keep=True)
            assert_batched_close(g, ref, X, st.beta)
    finally:
        s.close()


def test_factorization_grid_does_not_change_the_transition(pkg):
    """The factorization applies each tile's updates in a fixed order whatever
    the number of blocks, so smaller grids give the identical factor."""
    d = problem(3000, 1000, 5, "bf16", seed=8)
    outs = []
    for shrink in (False, True):
        s = pkg.HSProbit(d["X"], d["y"], seed=4, num_chains=4)
        try:
            if shrink:
                sh = s.launch_shape()
                s.set_launch_shape(chol_ctas=max(5, sh["chol_ctas"] // 3), trail_ctas=max(1, sh["trail_ctas"] // 4))
            s.sweep(2)
            outs.append([s.get_state(chain=m)["beta"] for m in range(4)])
        finally:
            s.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_factorization_beside_the_xstream_gives_the_same_transition(pkg):
    d = problem(5000, 600, 5, "bf16", seed=9)
    outs = []
    for overlap in (2, 1):
        s = pkg.HSProbit(d["X"], d["y"], seed=6, num_chains=4, use_graph=True)
        try:
            assert s.launch_shape()["overlap"] == 2
            s.set_launch_shape(overlap=overlap)
            assert s.launch_shape()["overlap"] == overlap
            s.sweep(3)
            outs.append([s.get_state(chain=m)["beta"] for m in range(4)])
        finally:
            s.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_launch_shape_rejects_out_of_range_sizes(pkg):
    d = problem(2000, 300, 5, "bf16", seed=1)
    s = pkg.HSProbit(d["X"], d["y"], seed=1, num_chains=4)
    try:
        sh = s.launch_shape()
        for bad in ({"xk_chains": 8}, {"xk_stages": 5}, {"xstream_ctas": sh["xstream_ctas"] + 1},
                    {"chol_ctas": 4}, {"xstream_ctas": -1}, {"xk_ctas_per_sm": 2, "xk_stages": 8},
                    {"xk_ctas_per_sm": 3}, {"overlap": 3}):
            with pytest.raises(pkg.HSProbitError):
                s.set_launch_shape(**bad)
        assert s.launch_shape() == sh
    finally:
        s.close()
    d = problem(2000, 40, 5, "f32", seed=1)
    s = pkg.HSProbit(d["X"], d["y"], seed=1)
    try:
        with pytest.raises(pkg.HSProbitError):
            s.set_launch_shape(xk_chains=16)  # no tensor-core X-stream on this handle
    finally:
        s.close()
