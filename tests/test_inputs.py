"""The seeded synthetic inputs (hs_synth) against their recipe: rows of the
correlated design follow N(0, Toeplitz(rho^|i-j|)); BF16 and FP8 storage
round the drawn values as stated (FP8: e4m3 codes times a per-column scale
max|x_j| / 448); y comes from the stored X; the data do not depend on the
number of generator threads; the two decoders (generator and oracle) agree."""
import numpy as np
import pytest

import hs_synth
from oracle import fmt


def test_ar1_design_has_the_toeplitz_correlation():
    d = hs_synth.make_problem(40000, 12, 3, "f64", seed=2, design="ar1", rho=0.5)
    X = d["X"]
    C = np.corrcoef(X, rowvar=False)
    lags = [np.mean(np.diag(C, k)) for k in range(4)]
    np.testing.assert_allclose(lags, [1.0, 0.5, 0.25, 0.125], atol=0.01)
    np.testing.assert_allclose(X.var(axis=0), 1.0, atol=0.03)


def test_iid_design_is_standard_normal_and_uncorrelated():
    X = hs_synth.make_problem(40000, 8, 2, "f64", seed=3)["X"]
    C = np.corrcoef(X, rowvar=False)
    assert np.abs(C - np.eye(8)).max() < 0.02
    np.testing.assert_allclose(X.mean(axis=0), 0.0, atol=0.02)


@pytest.mark.parametrize("dt", ["f32", "bf16", "fp8"])
def test_storage_rounds_the_f64_draws(dt):
    ref = hs_synth.make_problem(3000, 20, 4, "f64", seed=7)
    d = hs_synth.make_problem(3000, 20, 4, dt, seed=7)
    Xs = fmt.stored_to_f64(d["X"], dt, d["scales"])
    rel = {"f32": 2.0 ** -24, "bf16": 2.0 ** -8, "fp8": 2.0 ** -3}[dt]
    if dt == "fp8":
        np.testing.assert_allclose(d["scales"], np.abs(ref["X"]).max(axis=0) / 448.0, rtol=1e-6)
        # e4m3 with the column scale: relative error 2^-4 on normal codes, plus the subnormal floor
        floor = d["scales"][None, :].astype(np.float64) * 2.0 ** -10
        assert np.all(np.abs(Xs - ref["X"]) <= rel / 2 * np.abs(ref["X"]) + floor)
    else:
        assert np.all(np.abs(Xs - ref["X"]) <= rel * np.abs(ref["X"]) + 1e-300)
    # the generator's own decoder and the oracle's agree bit for bit
    np.testing.assert_array_equal(hs_synth.stored_to_float64(d["X"], dt, d["scales"]), Xs)


@pytest.mark.parametrize("dt", ["f64", "bf16", "fp8"])
def test_y_is_generated_from_the_stored_x(dt):
    d = hs_synth.make_problem(20000, 10, 3, dt, seed=9)
    Xs = fmt.stored_to_f64(d["X"], dt, d["scales"])
    eta = Xs @ d["beta_true"]
    # y = 1{eta + eps > 0}: agreement with sign(eta) wherever |eta| is large
    big = np.abs(eta) > 5.0
    assert big.sum() > 100
    assert np.all(d["y"][big] == (eta[big] > 0))
    # and P(y = 1 | eta) = Phi(eta) in aggregate
    from scipy.stats import norm
    assert abs(d["y"].mean() - norm.cdf(eta).mean()) < 0.01


def test_generation_does_not_depend_on_thread_count():
    a = hs_synth.make_problem(70000, 6, 2, "bf16", seed=4, threads=1, design="ar1")
    b = hs_synth.make_problem(70000, 6, 2, "bf16", seed=4, threads=7, design="ar1")
    np.testing.assert_array_equal(a["X"], b["X"])
    np.testing.assert_array_equal(a["y"], b["y"])
