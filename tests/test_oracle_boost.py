"""Pins for the oracle's SLR Boost (Sec. V: the boosting ensemble of SLR
trees; the rule is least-squares gradient boosting on residuals).

* closed form: on a target that one split fits exactly (a step in a feature,
  with a gap around the step so every bin edge in the gap separates the two
  sides), every round's tree predicts the residuals exactly, so the training
  MSE after m rounds is (1 - eta)^(2m) times the MSE of the mean;
* eta = 1 and one round: the predictions of one SLR tree grown on y;
* the training MSE never rises; the reported MSE is the mean squared
  residual of the returned F; prediction on the training rows reproduces F
  bit for bit; zero rounds predict the float mean;
* each round rebuilt from its definition: the residuals y - F in float and a
  tree grown with the key seed + m give that round's tree;
* bad arguments are refused.
"""
import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W


def step_data(n=2000, seed=1):
    rng = np.random.default_rng(seed)
    x0 = np.where(rng.random(n) < 0.5, -1.0, 1.0) * (1.0 + rng.random(n))
    X = np.stack([x0, rng.standard_normal(n)], 1).astype(np.float32)
    y = (3.0 * (x0 > 0) + 1.0).astype(np.float32)
    return X, y


@pytest.mark.parametrize("eta", [1.0, 0.5, 0.3])
def test_step_target_contracts_by_one_minus_eta_squared(eta):
    X, y = step_data()
    p = O.make_params("mse", 0, 16, 10, 32, min_leaf=5, max_depth=1)
    b = O.train_boost(p, X, y, 5, eta)
    mse0 = np.mean((y.astype(np.float64) - b.base) ** 2)
    want = np.array([mse0 * (1 - eta) ** (2 * m) for m in range(1, 6)])
    assert np.allclose(b.train_mse, want, rtol=1e-5, atol=1e-9)
    assert b.base == pytest.approx(np.mean(y.astype(np.float64)), rel=1e-7)


def test_one_round_with_eta_one_is_one_tree():
    wl = W.tanh_regression(3000, 6, seed=4)
    p = O.make_params("mse", 0, 16, 10, 64, min_leaf=10, max_depth=3, seed=2)
    b = O.train_boost(p, wl.X, wl.y, 1, 1.0)
    q = O.make_params("mse", 0, 16, 10, 64, min_leaf=10, max_depth=3, seed=3)  # seed + 1
    t = O.train_tree(q, wl.X, None, wl.y)
    assert np.array_equal(b.trees[0].kind, t.kind)
    _, v, _ = O.predict(q, t, wl.X)
    assert np.allclose(b.F, v, rtol=1e-5, atol=1e-5)


def test_training_mse_never_rises_and_matches_f():
    wl = W.tanh_regression(4000, 8, seed=3)
    p = O.make_params("mse", 0, 16, 10, 64, min_leaf=10, max_depth=4)
    b = O.train_boost(p, wl.X, wl.y, 8, 0.3)
    mse0 = np.mean((wl.y.astype(np.float64) - b.base) ** 2)
    assert np.all(np.diff(np.concatenate([[mse0], b.train_mse])) <= 0)
    assert b.train_mse[-1] < 0.5 * mse0
    r = wl.y.astype(np.float64) - b.F.astype(np.float64)
    assert b.train_mse[-1] == pytest.approx(np.mean(r * r), rel=1e-12)
    assert np.array_equal(O.boost_predict(p, b, wl.X), b.F)
    b0 = O.train_boost(p, wl.X, wl.y, 0, 0.3)
    assert np.all(O.boost_predict(p, b0, wl.X) == np.float32(np.mean(wl.y.astype(np.float64))))


def test_rounds_rebuilt_from_their_definition():
    wl = W.tanh_regression(2500, 5, seed=6)
    eta = np.float32(0.4)
    p = O.make_params("mse", 0, 12, 8, 32, min_leaf=10, max_depth=3, seed=11)
    b = O.train_boost(p, wl.X, wl.y, 3, float(eta))
    F = np.full(wl.y.shape, np.float32(b.base), np.float32)
    for m in range(1, 4):
        r = (wl.y - F).astype(np.float32)
        q = O.make_params("mse", 0, 12, 8, 32, min_leaf=10, max_depth=3, seed=11 + m)
        t = O.train_tree(q, wl.X, None, r)
        assert np.array_equal(t.kind, b.trees[m - 1].kind)
        assert np.array_equal(t.dir, b.trees[m - 1].dir)
        _, v, _ = O.predict(q, t, wl.X)
        F = (F + eta * v.astype(np.float32)).astype(np.float32)
    assert np.array_equal(F, b.F)


def test_bad_arguments():
    X, y = step_data(200)
    with pytest.raises(ValueError):
        O.train_boost(O.make_params("gini", 2, 8, 2, 16), X, y, 2, 0.5)
    for eta in (0.0, -0.1, 1.5):
        with pytest.raises(ValueError):
            O.train_boost(O.make_params("mse", 0, 8, 2, 16), X, y, 2, eta)
