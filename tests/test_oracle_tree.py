"""Pins for the oracle's tree growth (Algorithm 2) and prediction."""
import numpy as np
import pytest

import oracle as O
from paper_2208_07023_gb300 import workloads as W


def _params(crit, K, depth, **kw):
    base = dict(n_particles=16, n_iters=20, n_bins=32, max_depth=depth, min_leaf=5,
                precision=O.F32_MIRROR)
    base.update(kw)
    return O.make_params(crit, K, **base)


def _check_structure(t, p, n_total):
    H = len(t.kind)
    assert t.kind[0] != -1 and t.weight[0] == n_total
    for h in range(H):
        if t.kind[h] == 1:
            l, r = 2 * h + 1, 2 * h + 2
            assert t.kind[l] != -1 and t.kind[r] != -1
            assert t.n_left[h] == t.weight[l] and t.n_right[h] == t.weight[r]
            assert t.weight[l] + t.weight[r] == t.weight[h]
            assert t.weight[l] >= p.min_leaf and t.weight[r] >= p.min_leaf
        elif t.kind[h] == 0 and 2 * h + 1 < H:
            assert t.kind[2 * h + 1] == -1 and t.kind[2 * h + 2] == -1


@pytest.mark.parametrize("precision", [O.F64, O.F32_MIRROR])
def test_classification_tree_structure_and_training_fit(precision):
    wl = W.gmm(3000, 6, 4, seed=2)
    p = _params("gini", 4, 5, precision=precision)
    t = O.train_tree(p, wl.X, wl.labels)
    _check_structure(t, p, wl.n)
    cls, _, leaf = O.predict(p, t, wl.X)
    # predict sends each training sample to the leaf the partition gave it
    assert np.array_equal(np.bincount(leaf, minlength=len(t.kind)).astype(float)[t.kind == 0],
                          t.weight[t.kind == 0])
    # leaves predict their majority class
    for h in np.nonzero(t.kind == 0)[0]:
        m = leaf == h
        assert t.leaf_class[h] == np.argmax(np.bincount(wl.labels[m], minlength=4))
    # training error never rises as the depth limit grows
    errs = []
    for depth in range(0, 6):
        td = O.train_tree(_params("gini", 4, depth, precision=precision), wl.X, wl.labels)
        errs.append(np.mean(O.predict(_params("gini", 4, depth), td, wl.X)[0] != wl.labels))
    assert all(b <= a + 1e-12 for a, b in zip(errs, errs[1:]))
    assert errs[-1] < errs[0]


def test_separable_data_is_fit_exactly():
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (2000, 3)).astype(np.float32)
    lab = ((X[:, 0] + 0.5 * X[:, 1] > 0.1).astype(np.int32)
           + 2 * (X[:, 2] - 0.3 * X[:, 0] > 0.0).astype(np.int32))
    p = _params("gini", 4, 8, n_particles=32, n_iters=60, n_bins=256, min_leaf=1)
    t = O.train_tree(p, X, lab)
    err = np.mean(O.predict(p, t, X)[0] != lab)
    assert err < 0.01


def test_pure_and_tiny_nodes_are_leaves():
    X = np.random.default_rng(0).standard_normal((50, 3)).astype(np.float32)
    t = O.train_tree(_params("gini", 2, 4), X, np.zeros(50, np.int32))
    assert t.kind[0] == 0 and t.leaf_class[0] == 0 and np.all(t.kind[1:] == -1)
    t = O.train_tree(_params("gini", 2, 4, min_leaf=30), X, (np.arange(50) % 2).astype(np.int32))
    assert t.kind[0] == 0


def test_regression_tree():
    wl = W.tanh_regression(4000, 8, seed=4)
    p = _params("mse", 0, 6, min_leaf=10)
    t = O.train_tree(p, wl.X, None, wl.y)
    _check_structure(t, p, wl.n)
    _, val, leaf = O.predict(p, t, wl.X)
    for h in np.nonzero(t.kind == 0)[0]:
        assert t.leaf_value[h] == pytest.approx(wl.y[leaf == h].astype(np.float64).mean(), rel=1e-12)
    mse = np.mean((val - wl.y) ** 2)
    assert mse < 0.6 * np.var(wl.y)


def test_bootstrap_tree_uses_its_bag():
    wl = W.gmm(2000, 4, 3, seed=5)
    p = _params("gini", 3, 4)
    t = O.train_tree(p, wl.X, wl.labels, tree_id=7, bootstrap=True)
    w = O.bootstrap(p.seed, 7, wl.n)
    _check_structure(t, p, wl.n)
    assert t.weight[0] == w.sum()
    # the root's class counts are the bag's
    _, _, leaf = O.predict(p, t, wl.X)
    for h in np.nonzero(t.kind == 0)[0]:
        assert t.weight[h] == w[leaf == h].sum()


def test_majority_tie_goes_to_lowest_class():
    # Sec. II-A: leaves predict their majority class; equal counts -> lowest id.
    X = np.random.default_rng(1).standard_normal((40, 2)).astype(np.float32)
    lab = np.array([2, 1] * 20, np.int32)
    t = O.train_tree(_params("gini", 3, 3, min_leaf=25), X, lab)
    assert t.kind[0] == 0 and t.leaf_class[0] == 1


def _clusters(values_per_cluster):
    """1-D rows at x = 0, 1, 2, ...: cluster c holds values_per_cluster[c]."""
    xs, vs = [], []
    for c, vals in enumerate(values_per_cluster):
        xs += [float(c)] * len(vals)
        vs += list(vals)
    return np.array(xs, np.float32)[:, None], np.array(vs)


def test_split_that_keeps_the_class_mix_is_not_made():
    # Algorithm 2 grows a node only when its children are purer (Sec. II-A,
    # Eq. 4). Four clusters on a line, each with 10 samples of class 0 and 10
    # of class 1: with 4 bins every admissible edge leaves both children at
    # the parent's 50/50 mix, so the best split has zero gain and the root
    # must stay a leaf.
    X, lab = _clusters([[0] * 10 + [1] * 10] * 4)
    lab = lab.astype(np.int32)
    p = _params("gini", 2, 3, n_bins=4, min_leaf=5)
    sp = O.node_split(p, X, lab).split
    # there is an admissible split, and it scores the parent's impurity
    assert sp["valid"] == 1 and sp["loss"] == pytest.approx(0.5, abs=1e-15)
    t = O.train_tree(p, X, lab)
    assert t.kind[0] == 0 and np.all(t.kind[1:] == -1)
    assert t.weight[0] == 80 and t.leaf_class[0] == 0


def test_mse_split_that_does_not_lower_the_loss_is_not_made():
    # Regression form of the same rule: every cluster has mean 0 and the
    # same spread, so every admissible split keeps the parent's MSE (1.0).
    X, y = _clusters([[-1.0, 1.0] * 10] * 4)
    y = y.astype(np.float32)
    p = _params("mse", 0, 3, n_bins=4, min_leaf=5)
    sp = O.node_split(p, X, None, y).split
    assert sp["valid"] == 1 and sp["loss"] == pytest.approx(1.0, abs=1e-15)
    t = O.train_tree(p, X, None, y)
    assert t.kind[0] == 0 and np.all(t.kind[1:] == -1)
    assert t.leaf_value[0] == pytest.approx(0.0, abs=1e-15)


@pytest.mark.parametrize("flip", [False, True])
def test_right_child_holds_the_samples_at_or_above_the_threshold(flip):
    # Eqs. 3-4: the "+" side a^T x >= t_b, i.e. bin(z) >= b*, is the right
    # child 2h+2. Sides are computed here from the stored gB, zmin, inv_w and
    # b* with the float32 binning (one rounding per operation), not through
    # the oracle's prediction. 30 samples of one class below 0, 70 of the
    # other above, so the two children differ in size and class.
    rng = np.random.default_rng(11)
    neg = -rng.uniform(1.0, 2.0, 30)
    pos = rng.uniform(1.0, 2.0, 70)
    X = np.concatenate([neg, pos]).astype(np.float32)[:, None]
    lab = np.array([1] * 30 + [0] * 70, np.int32)
    if flip:
        lab = 1 - lab
    p = _params("gini", 2, 2, n_bins=16, min_leaf=5)
    t = O.train_tree(p, X, lab)
    assert t.kind[0] == 1
    a = np.float32(t.dir[0, 0])
    z = X[:, 0] * a  # d = 1: the fused multiply-add with 0 is one rounding
    off = (z - np.float32(t.zmin[0])).astype(np.float32)
    b = np.floor((off * np.float32(t.inv_w[0])).astype(np.float32)).astype(np.int64)
    b = np.clip(b, 0, p.n_bins - 1)
    right = b >= t.bin[0]
    assert 0 < right.sum() < len(X)
    assert t.weight[2] == right.sum() and t.weight[1] == (~right).sum()
    assert t.n_right[0] == right.sum() and t.n_left[0] == (~right).sum()
    # both children are pure: each predicts the class its own side holds
    assert t.kind[1] == 0 and t.kind[2] == 0
    assert t.leaf_class[2] == np.bincount(lab[right], minlength=2).argmax()
    assert t.leaf_class[1] == np.bincount(lab[~right], minlength=2).argmax()
    assert t.leaf_class[1] != t.leaf_class[2]
