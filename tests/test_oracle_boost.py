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

SLM Boost (K-class softmax gradient boosting with least-squares SLR trees):
* closed form on separable classes (K = 2 and 3): every sample keeps the
  same margin g, which grows by eta (1 - p) K / (K - 1), and the loss is
  log(1 + (K - 1) e^-g) (after the first round log(1 + (K - 1) e^-eta));
* on a mixture the loss falls every round, the reported loss is the mean
  cross-entropy of the returned scores, prediction reproduces them and the
  class is their argmax; bad arguments are refused;
* each round rebuilt from its definition: the softmax residuals of the
  scores so far and class k's tree grown with the round's key seed + m and
  tree id k give that round's trees.
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


# ---- SLM Boost (K-class softmax gradient boosting with least-squares trees) ----

def clusters(K, n=2400, seed=2):
    """K classes in separated intervals of feature 0 (gaps of width 1), and a
    noise feature: trees of depth >= ceil(log2 K) fit every residual exactly."""
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, K, n).astype(np.int32)
    x0 = 3.0 * lab + 2.0 * rng.random(n)
    X = np.stack([x0, rng.standard_normal(n)], 1).astype(np.float32)
    return X, lab


@pytest.mark.parametrize("K,depth", [(2, 1), (3, 2)])
@pytest.mark.parametrize("eta", [1.0, 0.5])
def test_cls_separable_closed_form(K, depth, eta):
    # every round's trees predict the residuals exactly, and by symmetry every
    # sample has the same margin g = F_true - F_other: the softmax gives
    # p = e^g / (e^g + K - 1), the true class gains eta (1 - p), each other
    # class loses eta (1 - p) / (K - 1), so g grows by eta (1 - p) K / (K - 1)
    # and the cross-entropy is log(1 + (K - 1) e^-g)
    X, lab = clusters(K)
    p = O.make_params("mse", 0, 16, 10, 32, min_leaf=5, max_depth=depth)
    b = O.train_boost_cls(p, X, lab, K, 4, eta)
    g, want = 0.0, []
    for _ in range(4):
        pm = np.exp(g) / (np.exp(g) + K - 1)
        g += eta * (1 - pm) * K / (K - 1)
        want.append(np.log1p((K - 1) * np.exp(-g)))
    assert np.allclose(b.train_loss, want, rtol=1e-6)
    assert b.train_loss[0] == pytest.approx(np.log1p((K - 1) * np.exp(-eta)), rel=1e-6)
    F, cls = O.boost_predict_cls(p, b, X)
    assert np.array_equal(F, b.F) and np.array_equal(cls, lab)


def test_cls_boosting_on_mixture():
    wl = W.gmm(3000, 6, 4, seed=5)
    p = O.make_params("mse", 0, 16, 10, 32, min_leaf=10, max_depth=3, seed=4)
    b = O.train_boost_cls(p, wl.X, wl.labels, 4, 6, 0.3)
    assert np.all(np.diff(b.train_loss) <= 0)
    assert b.train_loss[0] < np.log(4)
    F, cls = O.boost_predict_cls(p, b, wl.X)
    assert np.array_equal(F, b.F)
    assert np.array_equal(cls, np.argmax(F, axis=1))
    assert np.mean(cls == wl.labels) > 0.5
    # the reported loss is the mean cross-entropy of the returned scores
    Fd = b.F.astype(np.float64)
    lse = Fd.max(1) + np.log(np.exp(Fd - Fd.max(1, keepdims=True)).sum(1))
    ce = np.mean(lse - Fd[np.arange(len(wl.labels)), wl.labels])
    assert b.train_loss[-1] == pytest.approx(ce, rel=1e-12)


def test_cls_rounds_rebuilt_from_their_definition():
    # round m: the softmax residuals of the scores so far, then class k's
    # tree grown with the round's key seed + m and tree id k (the K trees of
    # a round are one forest), then F_k += eta v_k in class order
    wl = W.gmm(2000, 5, 3, seed=12)
    eta = np.float32(0.5)
    p = O.make_params("mse", 0, 12, 6, 32, min_leaf=10, max_depth=2, seed=5)
    b = O.train_boost_cls(p, wl.X, wl.labels, 3, 2, float(eta))
    F = np.zeros((len(wl.labels), 3), np.float32)
    for m in range(1, 3):
        R = O.softmax_residuals(F, wl.labels, 3)
        q = O.make_params("mse", 0, 12, 6, 32, min_leaf=10, max_depth=2, seed=5 + m)
        for k in range(3):
            t = O.train_tree(q, wl.X, None, R[k], tree_id=k)
            bt = b.trees[(m - 1) * 3 + k]
            assert np.array_equal(t.kind, bt.kind) and np.array_equal(t.dir, bt.dir)
            assert np.array_equal(t.bin, bt.bin)
            _, v, _ = O.predict(q, t, wl.X)
            F[:, k] = (F[:, k] + eta * v.astype(np.float32)).astype(np.float32)
    assert np.array_equal(F, b.F)
    # the class trees of one round draw distinct streams: grown as tree 0
    # instead, class 1's first tree differs from the boosting run's
    R = O.softmax_residuals(np.zeros_like(F), wl.labels, 3)
    q = O.make_params("mse", 0, 12, 6, 32, min_leaf=10, max_depth=2, seed=6)
    t0 = O.train_tree(q, wl.X, None, R[1], tree_id=0)
    assert not (np.array_equal(t0.dir, b.trees[1].dir))


def test_cls_bad_arguments():
    X, lab = clusters(3, 200)
    p = O.make_params("mse", 0, 8, 2, 16)
    with pytest.raises(ValueError):
        O.train_boost_cls(p, X, lab, 2, 2, 0.5)     # a label out of range
    with pytest.raises(ValueError):
        O.train_boost_cls(p, X, lab * 0, 1, 2, 0.5)  # K < 2
    with pytest.raises(ValueError):
        O.train_boost_cls(p, X, lab, 3, 2, 0.0)


def test_degenerate_targets():
    # a constant target: every residual is 0, every tree a single leaf of
    # value 0, F stays the mean and the training MSE is 0
    rng = np.random.default_rng(8)
    X = rng.standard_normal((500, 4)).astype(np.float32)
    y = np.full(500, 2.5, np.float32)
    p = O.make_params("mse", 0, 8, 4, 16, min_leaf=5, max_depth=3)
    b = O.train_boost(p, X, y, 3, 0.5)
    assert b.base == 2.5 and np.all(b.F == np.float32(2.5)) and np.all(b.train_mse == 0)
    assert all(t.kind[0] == 0 and (t.kind[1:] == -1).all() for t in b.trees)
    # one class present among K = 3: each round's residuals are constant per
    # class, so the trees are single leaves and every row gets the same scores
    lab = np.zeros(500, np.int32)
    c = O.train_boost_cls(p, X, lab, 3, 3, 0.5)
    assert all(t.kind[0] == 0 for t in c.trees)
    assert np.all(c.F == c.F[0]) and np.all(np.diff(c.train_loss) < 0)
    assert c.train_loss[0] == pytest.approx(np.log1p(2 * np.exp(-0.5)), rel=1e-6)
    # zero rounds: every score 0, every class tied: the lowest class
    z = O.train_boost_cls(p, X, lab, 3, 0, 0.5)
    F, cls = O.boost_predict_cls(p, z, X)
    assert np.all(F == 0) and np.all(cls == 0)
