"""GPU parity of SLR Boost and SLM Boost (Sec. V; gradient boosting of SLR
trees on residuals, in float) against the oracle. SLR Boost:

* base, every round's tree (identical nodes, except below a node where the
  two searches part after a near-tie the oracle logged), training MSE and
  the predictions, round by round while no tree has parted;
* the boost's prediction of the training rows is the training F: its MSE is
  the last reported training MSE; host and device inputs give one model;
* with one round and learning rate 1 the predictions are one tree's on the
  residuals of the mean; zero rounds predict the mean;
* bad arguments are refused.

SLM Boost (K-class softmax gradient boosting with least-squares SLR trees):
* every tree of every round as the oracle's (up to a logged near-tie), the
  residuals of each round taken from the oracle's scores, the training
  cross-entropy, the scores and the classes;
* the scores' cross-entropy is the reported loss, the class their argmax;
  two targets, a label outside [0, K) and K < 2 are refused.
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


# ---- SLM Boost ----------------------------------------------------------------------

@pytest.mark.parametrize("n,d,K,depth,M,eta,seed", [
    (3000, 6, 3, 3, 3, 0.5, 31),
    (2500, 8, 4, 2, 2, 1.0, 32),
])
def test_cls_boost_matches_oracle(ctx, n, d, K, depth, M, eta, seed):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(n, d, K, seed=seed)
    gp = S.make_params("mse", K, n_particles=16, n_iters=10, n_bins=32, min_leaf=10,
                       max_depth=depth, seed=2)
    b = ctx.train_boost(gp, wl.X, labels=wl.labels, n_classes=K, n_rounds=M,
                        learning_rate=eta)
    op = oracle_params(O, "mse", 0, 16, 10, 32, min_leaf=10, max_depth=depth, seed=2)
    r = O.train_boost_cls(op, wl.X, wl.labels, K, M, eta)
    assert b.info()["n_outputs"] == K and b.info()["n_rounds"] == M
    # the first round's residuals take two values (1 - 1/K, -1/K), so
    # partitions with equal counts have exactly equal SSE: the GPU's exact
    # fixed-point sums keep the tie (lower index wins) while the oracle's
    # double sums part them by rounding and log a near-tie; below such a node
    # the checker only requires the GPU's choice to be valid, and the later
    # trees then fit other residuals
    F = np.zeros((n, K), np.float32)
    matched, compared = True, 0
    for m in range(M):
        R = O.softmax_residuals(F, wl.labels, K)
        for k in range(K):
            t = m * K + k
            # the round's key seed + m, tree id k (the K trees of a round are
            # one forest)
            q = oracle_params(O, "mse", 0, 16, 10, 32, min_leaf=10, max_depth=depth,
                              seed=2 + m + 1)
            g = b.tree(t).export(0)
            compared += 1
            if _check_tree_up_to_near_ties(g, r.trees[t], q, wl.X, None, R[k], tree_id=k):
                matched = False
                break
            _, v, _ = O.predict(q, r.trees[t], wl.X)
            F[:, k] = (F[:, k] + np.float32(eta) * v.astype(np.float32)).astype(np.float32)
        if not matched:
            break
        assert b.train_loss[m] == pytest.approx(r.train_loss[m], rel=1e-12)
    assert compared >= 1
    if matched:
        assert np.array_equal(F, r.F)
        scores, cls = b.predict(wl.X, want_class=True)
        assert np.array_equal(scores, r.F)
        _, rcls = O.boost_predict_cls(op, r, wl.X)
        assert np.array_equal(cls, rcls)
    b.free()


def test_cls_boost_predictions_and_errors(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.gmm(4000, 8, 3, seed=33)
    gp = S.make_params("mse", 3, n_particles=16, n_iters=8, n_bins=32, min_leaf=10,
                       max_depth=3, seed=4)
    b = ctx.train_boost(gp, wl.X, labels=wl.labels, n_classes=3, n_rounds=4,
                        learning_rate=0.3)
    scores, cls = b.predict(wl.X, want_class=True)
    assert scores.shape == (4000, 3) and np.array_equal(cls, np.argmax(scores, axis=1))
    assert np.all(np.diff(b.train_loss) <= 0) and b.train_loss[0] < np.log(3)
    Fd = scores.astype(np.float64)
    lse = Fd.max(1) + np.log(np.exp(Fd - Fd.max(1, keepdims=True)).sum(1))
    ce = np.mean(lse - Fd[np.arange(4000), wl.labels])
    assert b.train_loss[-1] == pytest.approx(ce, rel=1e-12)
    assert np.mean(cls == wl.labels) > 0.5
    b.free()
    with pytest.raises(S.SlmError) as e:  # both targets
        ctx.train_boost(gp, wl.X, y=wl.X[:, 0].copy(), labels=wl.labels, n_rounds=1)
    assert e.value.status == S.SLM_EINVAL
    bad = wl.labels.copy()
    bad[7] = 3
    with pytest.raises(S.SlmError) as e:  # a label outside [0, K)
        ctx.train_boost(gp, wl.X, labels=bad, n_classes=3, n_rounds=1)
    assert e.value.status == S.SLM_EINVAL
    with pytest.raises(S.SlmError) as e:
        ctx.train_boost(S.make_params("mse", 1, n_particles=8, n_iters=2, n_bins=16), wl.X,
                        labels=wl.labels * 0, n_classes=1, n_rounds=1)
    assert e.value.status == S.SLM_EINVAL


def test_degenerate_targets(ctx):
    from paper_2208_07023_gb300 import binding as S
    rng = np.random.default_rng(8)
    X = rng.standard_normal((500, 4)).astype(np.float32)
    p = gpu_params(S, "mse", 0, 8, 4, 16, min_leaf=5, max_depth=3)
    b = ctx.train_boost(p, X, np.full(500, 2.5, np.float32), 3, 0.5)
    assert b.info()["base"] == 2.5 and np.all(b.predict(X) == np.float32(2.5))
    assert np.all(b.train_mse == 0)
    for m in range(3):
        k = b.tree(m).export(0)["kind"]
        assert k[0] == 0 and (k[1:] == -1).all()
    c = ctx.train_boost(S.make_params("mse", 3, n_particles=8, n_iters=4, n_bins=16, min_leaf=5,
                                      max_depth=3),
                        X, labels=np.zeros(500, np.int32), n_classes=3, n_rounds=3,
                        learning_rate=0.5)
    r = O.train_boost_cls(oracle_params(O, "mse", 0, 8, 4, 16, min_leaf=5, max_depth=3), X,
                          np.zeros(500, np.int32), 3, 3, 0.5)
    scores, cls = c.predict(X, want_class=True)
    assert np.array_equal(scores, r.F) and np.all(cls == 0)
    assert np.allclose(c.train_loss, r.train_loss, rtol=1e-12)


def test_boost_with_adaptive_pso_trees_matches_oracle(ctx):
    from paper_2208_07023_gb300 import binding as S
    wl = W.tanh_regression(3000, 6, seed=15)
    M, eta = 3, 0.5
    gp = S.make_params("mse", 0, n_particles=16, n_iters=10, n_bins=32, min_leaf=10,
                       max_depth=3, seed=2, apso=True)
    b = ctx.train_boost(gp, wl.X, wl.y, M, eta)
    op = oracle_params(O, "mse", 0, 16, 10, 32, min_leaf=10, max_depth=3, seed=2)
    op.apso = 1
    r = O.train_boost(op, wl.X, wl.y, M, eta)
    F = np.full(len(wl.y), np.float32(r.base), np.float32)
    for m in range(M):
        q = oracle_params(O, "mse", 0, 16, 10, 32, min_leaf=10, max_depth=3, seed=2 + m + 1)
        q.apso = 1
        if _check_tree_up_to_near_ties(b.tree(m).export(0), r.trees[m], q, wl.X, None,
                                       (wl.y - F).astype(np.float32)):
            break
        assert b.train_loss[m] == pytest.approx(r.train_mse[m], rel=1e-12)
        _, v, _ = O.predict(q, r.trees[m], wl.X)
        F = (F + np.float32(eta) * v.astype(np.float32)).astype(np.float32)
    b.free()


def test_boost_with_bf16_trees(ctx):
    # the tensor-core form's trees: every split is scored in FP32, the loss
    # falls every round and prediction reproduces the reported loss
    from paper_2208_07023_gb300 import binding as S
    wl = W.tanh_regression(20000, 32, seed=16)
    gp = S.make_params("mse", 0, n_particles=32, n_iters=10, n_bins=64, min_leaf=20,
                       max_depth=4, seed=3, proj=S.SLM_PROJ_BF16_TOPK, topk=8)
    b = ctx.train_boost(gp, wl.X, wl.y, 4, 0.5)
    assert np.all(np.diff(b.train_loss) < 0)
    pred = b.predict(wl.X)
    mse = np.mean((wl.y.astype(np.float64) - pred.astype(np.float64)) ** 2)
    assert mse == pytest.approx(b.train_loss[-1], rel=1e-12)
    b.free()


def test_cls_boost_round_forest_views(ctx):
    """Each round's K class trees are grown as one forest; every tree the
    boosting object returns is a one-tree view of it: tree ids 0..K-1 (node
    uids (k << 16) | h) under the round's key, its own evaluations (the
    searched entries of its internal nodes x P x (T + 1)), and it predicts
    on its own like the oracle's tree of that round and class."""
    from paper_2208_07023_gb300 import binding as S
    K, M, P, T = 3, 2, 16, 6
    wl = W.gmm(2500, 6, K, seed=41)
    gp = S.make_params("mse", K, n_particles=P, n_iters=T, n_bins=32, min_leaf=10,
                       max_depth=3, seed=9)
    b = ctx.train_boost(gp, wl.X, labels=wl.labels, n_classes=K, n_rounds=M,
                        learning_rate=0.5)
    r = O.train_boost_cls(oracle_params(O, "mse", 0, P, T, 32, min_leaf=10, max_depth=3,
                                        seed=9), wl.X, wl.labels, K, M, 0.5)
    F = np.zeros((len(wl.labels), K), np.float32)
    for m in range(M):
        R = O.softmax_residuals(F, wl.labels, K)
        for k in range(K):
            t = b.tree(m * K + k)
            inf = t.info()
            assert inf["n_trees"] == 1
            g = t.export(0)
            # searched nodes: every internal node, and at most every node
            # above the last level (a searched node may become a leaf)
            H = len(g["kind"])
            depth = np.floor(np.log2(np.arange(H) + 1)).astype(int)
            lo = int(g["weight"][g["kind"] == 1].sum())
            hi = int(g["weight"][(g["kind"] >= 0) & (depth < 3)].sum())
            ev = inf["evaluations"]
            assert ev % (P * (T + 1)) == 0 and lo <= ev // (P * (T + 1)) <= hi
            q = oracle_params(O, "mse", 0, P, T, 32, min_leaf=10, max_depth=3, seed=9 + m + 1)
            if _check_tree_up_to_near_ties(g, r.trees[m * K + k], q, wl.X, None, R[k],
                                          tree_id=k):
                b.free()
                return  # a logged near-tie: the rest of the run fits other residuals
            _, vg, _ = ctx.predict(t, wl.X)
            _, vo, _ = O.predict(q, r.trees[m * K + k], wl.X)
            assert np.allclose(vg, vo, rtol=1e-12, atol=1e-12)
            F[:, k] = (F[:, k] + np.float32(0.5) * vo.astype(np.float32)).astype(np.float32)
    b.free()
