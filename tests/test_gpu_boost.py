"""GPU parity of SLR Boost (Sec. V; least-squares gradient boosting of SLR
trees on residuals, in float) against the oracle.

* base, every round's tree (identical nodes, except below a node where the
  two searches part after a near-tie the oracle logged), training MSE and
  the predictions, round by round while no tree has parted;
* the boost's prediction of the training rows is the training F: its MSE is
  the last reported training MSE; host and device inputs give one model;
* with one round and learning rate 1 the predictions are one tree's on the
  residuals of the mean; zero rounds predict the mean;
* bad arguments are refused.
"""
import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W
from tests.gpu_util import context, gpu_params, oracle_params
from tests.test_gpu_parity import _check_tree_up_to_near_ties

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = context()
    yield c
    c.close()


@pytest.mark.parametrize("n,d,depth,M,eta,seed", [
    (4000, 6, 3, 5, 0.4, 12),
    (6000, 10, 4, 4, 1.0, 13),
    (3001, 5, 2, 6, 0.25, 14),   # ragged tail of tiles
])
def test_boost_matches_oracle(ctx, n, d, depth, M, eta, seed):
    from paper_2208_07023_gb300 import binding as S
    wl = W.tanh_regression(n, d, seed=seed)
    gp = gpu_params(S, "mse", 0, 16, 10, 32, min_leaf=10, max_depth=depth, seed=2)
    b = ctx.train_boost(gp, wl.X, wl.y, M, eta)
    op = oracle_params(O, "mse", 0, 16, 10, 32, min_leaf=10, max_depth=depth, seed=2)
    r = O.train_boost(op, wl.X, wl.y, M, eta)
    info = b.info()
    assert info["n_rounds"] == M and info["base"] == np.float32(r.base)
    F = np.full(n, np.float32(r.base), np.float32)
    matched = 0
    for m in range(M):
        q = oracle_params(O, "mse", 0, 16, 10, 32, min_leaf=10, max_depth=depth, seed=2 + m + 1)
        res = (wl.y - F).astype(np.float32)
        g = b.tree(m).export(0)
        if _check_tree_up_to_near_ties(g, r.trees[m], q, wl.X, None, res):
            break  # later rounds fit other residuals
        present = r.trees[m].kind >= 0
        assert np.allclose(g["leaf_value"][present], r.trees[m].leaf_value[present],
                           rtol=1e-12, atol=1e-12)
        assert b.train_mse[m] == pytest.approx(r.train_mse[m], rel=1e-12)
        _, v, _ = O.predict(q, r.trees[m], wl.X)
        F = (F + np.float32(eta) * v.astype(np.float32)).astype(np.float32)
        matched += 1
    assert matched >= 1
    if matched == M:
        assert np.array_equal(F, r.F)
        assert np.array_equal(b.predict(wl.X), r.F)
    b.free()


def test_prediction_is_the_training_f_and_host_equals_device(ctx):
    import torch
    from paper_2208_07023_gb300 import binding as S
    wl = W.tanh_regression(5000, 8, seed=21)
    gp = gpu_params(S, "mse", 0, 16, 8, 64, min_leaf=20, max_depth=4, seed=5)
    b = ctx.train_boost(gp, wl.X, wl.y, 6, 0.3)
    pred = b.predict(wl.X)
    mse = np.mean((wl.y.astype(np.float64) - pred.astype(np.float64)) ** 2)
    assert mse == pytest.approx(b.train_mse[-1], rel=1e-12)
    assert np.all(np.diff(b.train_mse) <= 0)
    Xd, yd = torch.from_numpy(wl.X).cuda(), torch.from_numpy(wl.y).cuda()
    b2 = ctx.train_boost(gp, Xd, yd, 6, 0.3)
    assert np.array_equal(b2.predict(Xd), pred)
    assert np.array_equal(b2.train_mse, b.train_mse)
    for m in range(6):
        for k, v in b.tree(m).export(0).items():
            assert np.array_equal(v, b2.tree(m).export(0)[k]), k
    b.free()
    b2.free()


def test_degenerate_rounds(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.tanh_regression(2000, 4, seed=22)
    gp = gpu_params(S, "mse", 0, 8, 5, 32, min_leaf=10, max_depth=3, seed=1)
    b0 = ctx.train_boost(gp, wl.X, wl.y, 0, 0.5)
    mean = np.float32(np.mean(wl.y.astype(np.float64)))
    assert np.all(b0.predict(wl.X) == mean)
    with pytest.raises(IndexError):
        b0.tree(0)
    # one round at learning rate 1: the tree's leaf values (means of y - mean)
    b1 = ctx.train_boost(gp, wl.X, wl.y, 1, 1.0)
    t = b1.tree(0)
    _, v, _ = ctx.predict(t, wl.X)
    want = (mean + np.float32(1.0) * v.astype(np.float32)).astype(np.float32)
    assert np.array_equal(b1.predict(wl.X), want)


def test_bad_boost_arguments(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.tanh_regression(500, 4, seed=23)
    gp = gpu_params(S, "mse", 0, 8, 2, 16, min_leaf=5, max_depth=2)
    for eta in (0.0, -1.0, 1.5):
        with pytest.raises(S.SlmError) as e:
            ctx.train_boost(gp, wl.X, wl.y, 2, eta)
        assert e.value.status == S.SLM_EINVAL
    with pytest.raises(S.SlmError) as e:
        ctx.train_boost(gpu_params(S, "gini", 2, 8, 2, 16), wl.X, wl.y, 2, 0.5)
    assert e.value.status == S.SLM_EINVAL
    with pytest.raises(S.SlmError) as e:
        ctx.train_boost(gpu_params(S, "mse", 0, 8, 2, 16, n_trees=2, bootstrap=True),
                        wl.X, wl.y, 2, 0.5)
    assert e.value.status == S.SLM_EUNSUPPORTED
